"""GPU parity of the host-buffer entry point ladder_apply_host (Eq. vfunction-chol): host L and
t2 in, host R out, through the plan's two device staging sets with the host-to-device copies of
one call on the library's copy stream during the previous call's contraction.  Checked against
the CPU oracle at the path's tolerance (FP64 1e-12, emulated 1e-10), bit for bit against
ladder_apply on device copies of the same inputs, and with several calls in flight on different
inputs (each result must be its own)."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs
from conftest import rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EMU = lad.LADDER_EMU_BF16


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def pinned(x):
    return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()


@pytest.mark.parametrize("precision,tol", [(lad.LADDER_FP64, 1e-12), (EMU, 1e-10)])
def test_host_call_matches_the_oracle_and_the_device_call(precision, tol):
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    plan = lad.ladder_plan(s.no, s.nv, s.nchol, precision)
    ws = plan.workspace()
    Rh = torch.full(t2.shape, 7.0, dtype=torch.float64).pin_memory()   # overwritten, not accumulated
    lad.ladder_apply_host(plan, pinned(L), pinned(t2), Rh, ws=ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    R = Rh.numpy()
    assert rel_fro(R, oracle.ladder(L, t2)) <= tol
    Rd = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda(), Rd, ws)
    assert np.array_equal(Rd.cpu().numpy(), R)


@pytest.mark.parametrize("precision,tol", [(lad.LADDER_FP64, 1e-12), (EMU, 1e-10)])
def test_calls_in_flight_keep_their_own_inputs(precision, tol):
    no, nv, nchol = 4, 33, 40
    inputs = [make_inputs(no, nv, nchol, seed=100 + k)[:2] for k in range(5)]
    plan = lad.ladder_plan(no, nv, nchol, precision)
    ws, stage = plan.workspace(), plan.host_staging()
    assert plan.host_staging_bytes() >= 2 * 8 * (nchol * nv * nv + 2 * no * no * nv * nv)
    hosts = [(pinned(L), pinned(t)) for L, t in inputs]
    outs = [torch.empty(t.shape, dtype=torch.float64).pin_memory() for _, t in inputs]
    for (Lh, th), Rh in zip(hosts, outs):   # five calls enqueued back to back, no host wait
        lad.ladder_apply_host(plan, Lh, th, Rh, stage, ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    for (L, t), Rh in zip(inputs, outs):
        assert rel_fro(Rh.numpy(), oracle.ladder(L, t)) <= tol


def test_pageable_host_memory_and_argument_checks():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    plan = lad.ladder_plan(s.no, s.nv, s.nchol, EMU)
    Rh = torch.empty(t2.shape, dtype=torch.float64)           # pageable
    lad.ladder_apply_host(plan, torch.from_numpy(L), torch.from_numpy(t2), Rh)
    torch.cuda.synchronize()
    assert rel_fro(Rh.numpy(), oracle.ladder(L, t2)) <= 1e-10
    with pytest.raises(TypeError):
        lad.ladder_apply_host(plan, torch.from_numpy(L).cuda(), torch.from_numpy(t2), Rh)
    lib = lad.lib()
    stage, ws = plan.host_staging(), plan.workspace()
    vp = ctypes.c_void_p
    args = [vp(torch.from_numpy(L).data_ptr()), vp(torch.from_numpy(t2).data_ptr()), vp(Rh.data_ptr())]
    misaligned = vp(stage.data_ptr() + 8)
    stream = vp(torch.cuda.current_stream().cuda_stream)
    assert lib.ladder_apply_host(plan.handle, *args, misaligned, vp(ws.data_ptr()), stream) == lad.LADDER_ERR_ARG
    assert lib.ladder_apply_host(plan.handle, *args, None, vp(ws.data_ptr()), stream) == lad.LADDER_ERR_ARG
