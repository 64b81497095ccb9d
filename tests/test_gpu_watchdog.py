"""The bounded-wait watchdog of the tcgen05 kernels, made to fire without any GPU fault: a
wait on an mbarrier that nothing arrives on must give up after its limit (2 s of the GPU's
global timer), report LADDER_ERR_TIMEOUT through the status word, and leave the context
usable for the next call."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import make_inputs
from conftest import rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def test_lost_arrival_times_out_and_the_context_survives():
    status, waited_ms = lad.ladder_watchdog_selftest()
    assert status == lad.LADDER_ERR_TIMEOUT
    assert 1900.0 <= waited_ms <= 10000.0
    # the context still works: a full emulated ladder call right after
    L, t2, _, _ = make_inputs(3, 20, 30, seed=9)
    plan = lad.ladder_plan(3, 20, 30, lad.LADDER_EMU_BF16)
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda(), R)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    assert rel_fro(R.cpu().numpy(), oracle.ladder(L, t2)) <= 1e-10


def test_shorter_wait_limit_is_honoured():
    # the same device wait with a 0.3 s limit gives up after ~0.3 s
    status, waited_ms = lad.ladder_watchdog_selftest(0.3)
    assert status == lad.LADDER_ERR_TIMEOUT
    assert 290.0 <= waited_ms <= 5000.0
    assert lad.ladder_watchdog_selftest(-1.0)[0] == lad.LADDER_ERR_ARG
    assert lad.ladder_watchdog_selftest(120.0)[0] == lad.LADDER_ERR_ARG


def test_plan_wait_limit_is_a_plan_parameter():
    L, t2, _, _ = make_inputs(4, 33, 40, seed=19)
    plan = lad.ladder_plan(4, 33, 40, lad.LADDER_EMU_BF16)
    assert plan.wait_limit() == pytest.approx(2.0)
    plan.set_wait_limit(30.0)
    assert plan.wait_limit() == pytest.approx(30.0)
    for bad in (-1.0, 1e-4, 4000.0):
        with pytest.raises(lad.LadderError) as e:
            plan.set_wait_limit(bad)
        assert e.value.status == lad.LADDER_ERR_ARG
    assert plan.wait_limit() == pytest.approx(30.0)
    # a call under a short (but ample) limit is unaffected
    plan.set_wait_limit(0.25)
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda(), R)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    assert rel_fro(R.cpu().numpy(), oracle.ladder(L, t2)) <= 1e-10
    plan.set_wait_limit(0.0)
    assert plan.wait_limit() == pytest.approx(2.0)
