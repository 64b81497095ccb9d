"""Cholesky vectors sliced in batches (emulated path): each batch's L^T digit planes are sliced
per block pair and its ERI adds exact int64 sums into V, rounded onto the pair's grid after the
last batch.  Checked against the CPU oracle (Eq. vfunction-chol) within the emulated tolerance,
against the unbatched plan, and bit-exactly on integer inputs."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import make_inputs, make_integer_inputs
from conftest import rel_fro
from test_gpu_fp64 import dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EMU = lad.LADDER_EMU_BF16
TOL_R = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def run(L, t2, pb=None, budget=0, blocks=None, form=None):
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(no, nv, nchol, EMU, ws_budget_bytes=budget)
    if form is not None:
        plan.set_form(form)
    if pb is not None:
        plan.set_pbatch(pb)
    if blocks is not None:
        plan.set_blocks(*blocks)
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, dev(L), dev(t2), R, plan.workspace())
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R.cpu().numpy(), plan


def test_batches_of_cholesky_vectors_match_the_oracle_and_the_unbatched_plan():
    L, t2, _, _ = make_inputs(4, 40, 2600, seed=71)
    ref = oracle.ladder(L, t2)
    R1, p1 = run(L, t2, pb=1024)                      # three batches: 1024, 1024, 552
    assert p1.pbatch() == 1024 and p1.form() == 1
    assert rel_fro(R1, ref) <= TOL_R
    R0, p0 = run(L, t2, pb=0, form=1)                 # all vectors at once, same ladder form
    assert p0.pbatch() == 0
    # the exact levels are the same; only the shared tail level's rounding may differ
    assert rel_fro(R1, R0) <= 1e-13
    Rb, pbk = run(L, t2, pb=640, blocks=(13, 7))      # batches and a blocking together
    assert pbk.pbatch() == 640
    assert rel_fro(Rb, ref) <= TOL_R


def test_integer_grid_is_bit_exact_with_batches():
    L, t2 = make_integer_inputs(3, 21, 2100, seed=5)
    R, plan = run(L, t2, pb=1024)
    assert plan.pbatch() == 1024
    assert np.array_equal(R, oracle.ladder(L, t2))


def test_planner_batches_when_the_planes_of_all_vectors_do_not_fit():
    no, nv, nchol = 3, 32, 6000
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=72)
    planes = 12 * nv * 32 * 6000                      # L^T digit planes of all vectors (S = 6)
    budget = int(planes * 0.7)
    with pytest.raises(lad.LadderError):             # all vectors at once cannot fit
        lad.ladder_plan_dry(no, nv, nchol, EMU, ws_budget_bytes=budget, force_n_a=1, force_n_b=1)
    R, plan = run(L, t2, budget=budget)
    assert plan.pbatch() > 0 and plan.workspace_bytes() <= budget
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL_R


def test_batches_need_the_split_form():
    plan = lad.ladder_plan(3, 20, 2000, EMU)
    plan.set_pbatch(1024)
    assert plan.form() == 1
    with pytest.raises(lad.LadderError):
        plan.set_form(0)
    for bad in (-64, 100):
        with pytest.raises(lad.LadderError):
            plan.set_pbatch(bad)
    plan.set_pbatch(0)
    assert plan.pbatch() == 0
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan(3, 20, 2000, lad.LADDER_FP64).set_pbatch(1024)
    assert e.value.status == lad.LADDER_ERR_UNSUPPORTED
