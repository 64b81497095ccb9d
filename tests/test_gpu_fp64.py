"""GPU parity of the native FP64 path against the CPU oracle (through the C ABI).

Tolerance: ||R_gpu - R_oracle||_F / ||R_oracle||_F <= 1e-12 (FP64 path).
Integer-valued inputs must agree bit for bit (every partial sum is an exact
integer below 2^53).
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs, make_integer_inputs
from conftest import rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
TOL_FP64 = 1e-12
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def assert_pair_symmetry(R, diag_tol=None):
    """R_ij^ab = R_ji^ba: exact for a != b (both written from one value); for a == b
    R_ij^aa and R_ji^aa are separate evaluations (FP64: the same nv^2 products summed in
    another order, a rounding difference growing like sqrt(nv^2) u, so the default is
    nv 2^-50; emulated: digits taken in different exponent groups), equal to diag_tol."""
    Rt = R.transpose(1, 0, 3, 2)
    nv = R.shape[2]
    if diag_tol is None:
        diag_tol = nv * 2.0 ** -50
    off = ~np.eye(nv, dtype=bool)
    assert np.array_equal(R[:, :, off], Rt[:, :, off])
    d = np.arange(nv)
    assert rel_fro(R[:, :, d, d], Rt[:, :, d, d]) <= diag_tol


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_ladder(L, t2, precision=lad.LADDER_FP64, R0=None, blocks=None, budget=0, nslices=0,
               path=lad.LADDER_PATH_ERI):
    """R from one ladder_apply.  FP64 plans are held to the given evaluation order (default:
    rebuild (ac|bd) per block pair; the factorised order has its own tests)."""
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    # the default budget is a fraction of the free memory: hand torch's cached blocks back first
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(no, nv, nchol, precision, nslices=nslices, ws_budget_bytes=budget)
    if precision == lad.LADDER_FP64 and path is not None:
        plan.set_path(path)
    if blocks is not None:
        plan.set_blocks(*blocks)
    Ld, td = dev(L), dev(t2)
    R = dev(R0) if R0 is not None else torch.zeros_like(td)
    ws = plan.workspace()
    lad.ladder_apply(plan, Ld, td, R, ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R.cpu().numpy(), plan


def test_c1_parity_and_pair_symmetry():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, _ = gpu_ladder(L, t2)
    ref = oracle.ladder(L, t2)
    assert rel_fro(R, ref) <= TOL_FP64
    assert_pair_symmetry(R)


def test_accumulates_into_nonzero_R():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R0 = np.random.default_rng(3).standard_normal(t2.shape)
    R, _ = gpu_ladder(L, t2, R0=R0)
    ref = oracle.ladder(L, t2, R0)
    assert rel_fro(R, ref) <= TOL_FP64


@pytest.mark.parametrize("blocks", [(1, 1), (3, 7), (7, 3), (19, 19), (5, 19), (19, 1), (2, 2), (10, 4)])
def test_forced_blockings_match_single_batch(blocks):
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R1, plan1 = gpu_ladder(L, t2)
    assert plan1.describe()["n_block_pairs"] == 1
    Rb, planb = gpu_ladder(L, t2, blocks=blocks)
    d = planb.describe()
    assert (d["n_a"], d["n_b"]) == blocks
    assert rel_fro(Rb, R1) <= TOL_FP64
    assert rel_fro(Rb, oracle.ladder(L, t2)) <= TOL_FP64


def test_small_budget_forces_split():
    no, nv, nchol = 3, 37, 45   # ragged against every tile size
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=21)
    ref = oracle.ladder(L, t2)
    one = lad.ladder_plan(no, nv, nchol)
    one.set_path(lad.LADDER_PATH_ERI)
    full = one.workspace_bytes()
    R, plan = gpu_ladder(L, t2, budget=full // 6)
    d = plan.describe()
    assert d["n_block_pairs"] > 1 and plan.workspace_bytes() <= full // 6
    assert rel_fro(R, ref) <= TOL_FP64


def test_budget_too_small_is_an_error():
    # no V block, no factorised batch, and no^2 = 1089 rows are more than the fused kernel holds
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan(33, 37, 45, ws_budget_bytes=512)
    assert e.value.status == lad.LADDER_ERR_BUDGET
    # with no^2 <= 1024 the fused path needs no workspace and takes the plan
    plan = lad.ladder_plan(3, 37, 45, ws_budget_bytes=512)
    assert plan.path() == lad.LADDER_PATH_FUSED and plan.workspace_bytes() <= 512


@pytest.mark.parametrize("no,nv,nchol", [(1, 1, 1), (1, 2, 3), (2, 1, 5), (4, 9, 1), (6, 65, 17), (9, 33, 130)])
def test_edge_shapes(no, nv, nchol):
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=no * 1000 + nv)
    R, _ = gpu_ladder(L, t2)
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL_FP64


def test_integer_inputs_bit_exact():
    L, t2 = make_integer_inputs(4, 23, 40, seed=5)
    R, _ = gpu_ladder(L, t2)
    assert np.array_equal(R, oracle.ladder(L, t2))
    Rb, _ = gpu_ladder(L, t2, blocks=(4, 9))
    assert np.array_equal(Rb, oracle.ladder(L, t2))


def test_nonsymmetric_t2_violates_packing_precondition():
    no, nv, nchol = 3, 11, 13
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=31, symmetric_t2=False)
    R, _ = gpu_ladder(L, t2)
    assert rel_fro(R, oracle.ladder(L, t2)) > 1e-3


def test_deterministic():
    no, nv, nchol = 4, 45, 60
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=41)
    R1, _ = gpu_ladder(L, t2)
    R2, _ = gpu_ladder(L, t2)
    assert np.array_equal(R1, R2)


def test_energy_kernel():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = gpu_ladder(L, t2)
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    assert E == pytest.approx(oracle.energy(t2, R), rel=1e-13, abs=1e-15)
    E_ref = oracle.energy(t2, oracle.ladder(L, t2))
    assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    lad.ladder_energy(plan, dev(t2), dev(R), E_dev=Ed)
    torch.cuda.synchronize()
    assert float(Ed.item()) == E


def test_misaligned_pointer_is_rejected():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    plan = lad.ladder_plan(s.no, s.nv, s.nchol)
    Ld = torch.zeros(L.size + 1, dtype=torch.float64, device="cuda")[1:]
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_apply(plan, Ld, dev(t2), torch.zeros_like(dev(t2)))
    assert e.value.status == lad.LADDER_ERR_ARG


def _sample_pairs(nv, n, seed):
    rng = np.random.default_rng(seed)
    fixed = [(0, 0), (0, nv - 1), (nv - 1, nv - 1), (nv // 2, nv // 2), (1, 2), (nv - 2, nv - 1)]
    rnd = [tuple(sorted(rng.integers(0, nv, 2))) for _ in range(n - len(fixed))]
    return fixed + rnd


def check_sampled(R, L, t2, tol, nsample=48, seed=0):
    nv = L.shape[1]
    pairs = _sample_pairs(nv, nsample, seed)
    a = [p[0] for p in pairs]
    b = [p[1] for p in pairs]
    ref = oracle.ladder_pairs(L, t2, a, b)            # [k, i, j]
    got = np.stack([R[:, :, x, y] for x, y in pairs])
    assert rel_fro(got, ref) <= tol
    # mirrors R[j,i,b,a] = R[i,j,a,b]
    mir = np.stack([R[:, :, y, x].T for x, y in pairs])
    assert rel_fro(mir, ref) <= tol


def _golden(name, key):
    if not os.path.exists(GOLDEN):
        return None
    with open(GOLDEN) as f:
        g = json.load(f)
    return g.get(name, {}).get(key)


def _golden_energy(name):
    return _golden(name, "E_L")


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_full_size_sampled_parity(name):
    # c3 in FP64 takes ~40 s on GB300 (FP64 ~1.1 TFLOP/s); the whole array is checked through
    # its Frobenius norm and E_L against the oracle's stored values, and 48 (a,b) pairs directly.
    s = CONFIGS[name]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = gpu_ladder(L, t2)
    check_sampled(R, L, t2, TOL_FP64)
    assert_pair_symmetry(R)
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    assert E == pytest.approx(oracle.energy(t2, R), rel=1e-12)
    Eg, Fg = _golden_energy(name), _golden(name, "R_fro")
    if Eg is not None:
        assert abs(E - Eg) <= 1e-10 * abs(Eg)
    if Fg is not None:
        assert abs(float(np.linalg.norm(R.ravel())) - Fg) <= 1e-12 * Fg
