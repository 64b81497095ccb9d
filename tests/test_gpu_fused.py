"""GPU parity of the fused evaluation (native FP64): (ac|bd) built chunk by chunk in shared memory
and contracted with t2 at once (the two C-split steps of a batch kept on the chip, Sec. "An
Asymmetric and Dynamic Splitting Protocol", Table 1), against the CPU oracle's plain loops
(Eq. vfunction-chol), through the C ABI.

Tolerance as for the FP64 path: ||R - R_oracle||_F / ||R_oracle||_F <= 1e-12; integer inputs
bit-exact.  Every (a, b) pair sums its (c, d) chunks in one fixed order whatever tile or block
pair holds it, so any blocking or sharding gives the same bits."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs, make_integer_inputs
from conftest import rel_fro
from test_gpu_fp64 import _golden, assert_pair_symmetry, check_sampled, dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-12
FP64 = lad.LADDER_FP64
FUSED = lad.LADDER_PATH_FUSED


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def run(L, t2, plan=None, R0=None, budget=0):
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    torch.cuda.empty_cache()
    if plan is None:
        plan = lad.ladder_plan(no, nv, nchol, FP64, ws_budget_bytes=budget)
        plan.set_path(FUSED)
    assert plan.path() == FUSED
    Ld, td = dev(L), dev(t2)
    R = dev(R0) if R0 is not None else torch.zeros_like(td)
    lad.ladder_apply(plan, Ld, td, R, plan.workspace())
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R.cpu().numpy(), plan


def test_c1_parity_symmetry_and_no_workspace():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = run(L, t2)
    assert plan.workspace_bytes() <= 256
    assert plan.describe()["n_block_pairs"] == 1
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL
    assert_pair_symmetry(R)


# Shapes: ragged nv and nchol against the 4x4 pair tiles, 16x16 (c,d) chunks and 16-vector
# staging steps; no^2 in each accumulator variant (8-row tiles per warp: 1, 2, 4, 8, 16,
# up to no^2 = 1024).
@pytest.mark.parametrize("no,nv,nchol", [(1, 1, 1), (3, 17, 5), (2, 70, 9), (7, 33, 130), (9, 37, 17),
                                         (12, 50, 40), (20, 23, 33), (32, 21, 20), (5, 19, 72)])
def test_edge_shapes_match_the_oracle(no, nv, nchol):
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=no * 1000 + nv)
    R, _ = run(L, t2)
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL
    assert_pair_symmetry(R)


def test_accumulates_into_nonzero_R():
    L, t2, _, _ = make_inputs(6, 29, 21, seed=11)
    R0 = np.random.default_rng(5).standard_normal(t2.shape)
    R, _ = run(L, t2, R0=R0)
    assert rel_fro(R - R0, oracle.ladder(L, t2)) <= TOL


def test_integer_grid_is_bit_exact():
    L, t2 = make_integer_inputs(4, 26, 7, seed=9)
    R, _ = run(L, t2)
    assert np.array_equal(R, oracle.ladder(L, t2))


def test_same_bits_as_its_shards_and_any_blocking():
    no, nv, nchol = 5, 45, 24
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=21)
    R_whole, _ = run(L, t2)
    acc = np.zeros_like(R_whole)
    world = 3
    for rank in range(world):
        plan = lad.ladder_plan(no, nv, nchol, FP64)
        plan.set_path(FUSED)
        plan.shard(rank, world)
        assert plan.path() == FUSED
        R, _ = run(L, t2, plan=plan)
        written = R != 0
        assert not np.any(written & (acc != 0))     # the shards write disjoint entries
        acc += R
    assert np.array_equal(acc, R_whole)


def test_path_rules_and_rejections():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    plan = lad.ladder_plan(s.no, s.nv, s.nchol, FP64)
    plan.set_path(FUSED)
    assert plan.path() == FUSED
    plan.set_path(lad.LADDER_PATH_ERI)                 # back to the rebuild order, with a V block
    assert plan.path() == 0 and plan.workspace_bytes() > 256
    plan.set_path(FUSED)
    plan.set_blocks(7, 5)                               # a forced blocking is path 0
    assert plan.path() == 0
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan(s.no, s.nv, s.nchol, lad.LADDER_EMU_BF16).set_path(FUSED)
    assert e.value.status == lad.LADDER_ERR_UNSUPPORTED
    big = lad.ladder_plan(33, 8, 4, FP64)               # no^2 = 1089 > 1024 accumulator rows
    with pytest.raises(lad.LadderError) as e:
        big.set_path(FUSED)
    assert e.value.status == lad.LADDER_ERR_UNSUPPORTED
    assert big.path() != FUSED


def test_planner_takes_the_fused_path_when_no_workspace_fits():
    no, nv, nchol = 4, 48, 30
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=31)
    # 4 KB: no V block (one pair row is 8 nv^2 = 18 KB) and no factorised batch fits
    plan = lad.ladder_plan(no, nv, nchol, FP64, ws_budget_bytes=4096)
    assert plan.path() == FUSED
    R, _ = run(L, t2, plan=plan)
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL


def test_c3_sampled_parity():
    # about 40 s on GB300 (FP64 DMMA ~1.1 TFLOP/s): 48 (a,b) pairs against the oracle's pair
    # mode, the whole array through ||R||_F and E_L against the oracle's stored values.
    s = CONFIGS["c3"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = run(L, t2)
    check_sampled(R, L, t2, TOL)
    assert_pair_symmetry(R)
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    Eg, Fg = _golden("c3", "E_L"), _golden("c3", "R_fro")
    if Eg is not None:
        assert abs(E - Eg) <= 1e-10 * abs(Eg)
    if Fg is not None:
        assert abs(float(np.linalg.norm(R.ravel())) - Fg) <= 1e-12 * Fg
