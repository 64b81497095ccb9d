"""GPU parity of the factorised evaluation order R_ij = sum_P L_P T_ij L_P^T (native FP64, two
DMMA GEMMs per batch of Cholesky vectors, amplitude pairs i <= j with R_ji = R_ij^T) against the
CPU oracle's plain loops (Eq. vfunction-chol), through the C ABI.  Tolerance as for the FP64
path: ||R - R_oracle||_F / ||R_oracle||_F <= 1e-12; integer inputs bit-exact."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs, make_integer_inputs
from conftest import rel_fro
from test_gpu_fp64 import dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-12
FP64 = lad.LADDER_FP64


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def assert_ij_symmetry(R):
    """R_ji^ba = R_ij^ab: exact for i != j (R_ji is written as the transpose of the R_ij the
    order computes for i < j); for i == j the entries (a, b) and (b, a) are two separate sums of
    the same products in another order, equal to rounding (nv 2^-50 relative)."""
    no, nv = R.shape[0], R.shape[2]
    Rt = R.transpose(1, 0, 3, 2)
    off = ~np.eye(no, dtype=bool)
    assert np.array_equal(R[off], Rt[off])
    d = np.arange(no)
    assert rel_fro(R[d, d], Rt[d, d]) <= nv * 2.0 ** -50


def run(L, t2, path=None, budget=0, R0=None):
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(no, nv, nchol, FP64, ws_budget_bytes=budget)
    if path is not None:
        plan.set_path(path)
    Ld, td = dev(L), dev(t2)
    R = dev(R0) if R0 is not None else torch.zeros_like(td)
    lad.ladder_apply(plan, Ld, td, R, plan.workspace())
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R.cpu().numpy(), plan


def test_planner_picks_the_factorised_order_where_it_is_cheaper():
    no, nv, nchol = 12, 64, 8          # few Cholesky vectors, many amplitude pairs
    assert lad.ladder_path_model(no, nv, nchol, FP64) == 1
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=3)
    R, plan = run(L, t2)
    assert plan.path() == lad.LADDER_PATH_FACTORISED
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL
    assert_ij_symmetry(R)


@pytest.mark.parametrize("no,nv,nchol", [(5, 19, 72), (1, 1, 1), (3, 17, 5), (2, 70, 9), (7, 33, 130)])
def test_forced_factorised_order_matches_the_oracle(no, nv, nchol):
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=no * 100 + nv)
    R, plan = run(L, t2, path=lad.LADDER_PATH_FACTORISED)
    assert plan.path() == 1
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL


def test_batches_of_cholesky_vectors_and_accumulation():
    no, nv, nchol = 4, 40, 11
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=8)
    npij = no * (no + 1) // 2
    budget = 8 * npij * nv * nv * 3 + 4096       # three Cholesky vectors per batch: 4 batches
    R0 = np.random.default_rng(2).standard_normal(t2.shape)
    R, plan = run(L, t2, path=lad.LADDER_PATH_FACTORISED, budget=budget, R0=R0)
    assert plan.workspace_bytes() <= budget
    assert rel_fro(R - R0, oracle.ladder(L, t2)) <= TOL


def test_integer_grid_is_bit_exact():
    L, t2 = make_integer_inputs(3, 21, 6, seed=4)
    R, _ = run(L, t2, path=lad.LADDER_PATH_FACTORISED)
    assert np.array_equal(R, oracle.ladder(L, t2))


def test_switching_orders_and_emulated_rejection():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R0, plan = run(L, t2)
    assert plan.path() == lad.LADDER_PATH_FUSED   # the planner's choice at this shape
    plan.set_path(lad.LADDER_PATH_FACTORISED)
    assert plan.path() == 1
    plan.set_blocks(7, 5)                      # a forced blocking is the rebuild order
    assert plan.path() == 0
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan(s.no, s.nv, s.nchol, lad.LADDER_EMU_BF16).set_path(1)
    assert e.value.status == lad.LADDER_ERR_UNSUPPORTED
    R1, _ = run(L, t2, path=lad.LADDER_PATH_FACTORISED)
    assert rel_fro(R1, R0) <= TOL
