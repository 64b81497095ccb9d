"""GPU parity of the emulated-FP64 path (BF16 digit slices on tcgen05) against
the CPU oracle, through the C ABI.

Tolerances (stated for the emulated path): ||R - R_oracle||_F / ||R_oracle||_F
<= 1e-10 and |E_L - E_L(oracle)| <= 1e-8 Eh at the default 6 slices.
Every cross-chunk and cross-block sum of the path is an exact integer, so the
result must not depend on the blocking or on the split-K partition at all:
those tests compare bit for bit.
"""
import json
import os
import sys

import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs, make_integer_inputs
from conftest import rel_fro

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from emu_model import emulated_ladder  # noqa: E402
from test_gpu_fp64 import check_sampled, dev, gpu_ladder, assert_pair_symmetry, _golden, _golden_energy  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EMU = lad.LADDER_EMU_BF16
TOL_R = 1e-10
TOL_E = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def test_c1_parity_energy_and_symmetry():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = gpu_ladder(L, t2, EMU)
    ref = oracle.ladder(L, t2)
    assert rel_fro(R, ref) <= TOL_R
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    assert abs(E - oracle.energy(t2, ref)) <= TOL_E
    assert_pair_symmetry(R, diag_tol=TOL_R)


def test_c1_matches_cpu_model_of_the_scheme():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, _ = gpu_ladder(L, t2, EMU)
    model = emulated_ladder(L, t2, S=6)
    # The model computes every (a, b) from its own V row; the library forms a > b from the
    # mirror R_ji^ba, so compare the a <= b half, where both evaluate the same digits.  The only
    # difference left is the FP32 rounding of the levels >= 6 (weight <= 2^-28).
    iu = np.triu_indices(s.nv)
    assert rel_fro(R[:, :, iu[0], iu[1]], model[:, :, iu[0], iu[1]]) <= 1e-13


@pytest.mark.parametrize("no,nv,nchol", [(3, 32, 50), (2, 47, 40), (4, 80, 33)])
def test_sector_paired_layouts_match_the_model(no, nv, nchol):
    # vp (nv rounded up to 16): the ERI epilogue stores V in whole
    # 32-byte sectors.  Same digits as the model, and blocking-independent bit for bit.
    # With K = nv^2 near a full 1024 chunk the FP32 accumulator of the levels >= 6 is no
    # longer exact (the model keeps it in FP64); modelling it as FP32 with truncation moves
    # the result by ~2e-13 here, so the bound is 2e-12 (a wrong digit plane gives >= 1e-9).
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=nv)
    R, _ = gpu_ladder(L, t2, EMU)
    model = emulated_ladder(L, t2, S=6)
    iu = np.triu_indices(nv)
    assert rel_fro(R[:, :, iu[0], iu[1]], model[:, :, iu[0], iu[1]]) <= 2e-12
    Rb, _ = gpu_ladder(L, t2, EMU, blocks=(5, 3))
    assert np.array_equal(Rb, R)


@pytest.mark.parametrize("S,tol", [(5, 1e-8), (6, 1e-10), (7, 1e-11), (8, 5e-12)])
def test_slice_count_controls_the_error(S, tol):
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = gpu_ladder(L, t2, EMU, nslices=S)
    assert plan.describe()["nslices"] == S
    assert rel_fro(R, oracle.ladder(L, t2)) <= tol


def test_integer_grid_is_bit_exact():
    L, t2 = make_integer_inputs(4, 23, 40, seed=5)
    R, _ = gpu_ladder(L, t2, EMU)
    assert np.array_equal(R, oracle.ladder(L, t2))


@pytest.mark.parametrize("blocks", [(1, 1), (3, 7), (7, 3), (5, 19), (19, 2), (10, 4)])
def test_blocking_does_not_change_a_single_bit(blocks):
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R1, _ = gpu_ladder(L, t2, EMU)
    Rb, plan = gpu_ladder(L, t2, EMU, blocks=blocks)
    d = plan.describe()
    assert (d["n_a"], d["n_b"]) == blocks
    assert np.array_equal(Rb, R1)


def test_small_budget_split_and_accumulation():
    no, nv, nchol = 3, 37, 45
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=21)
    R0 = np.random.default_rng(4).standard_normal(t2.shape)
    full = lad.ladder_plan(no, nv, nchol, EMU).workspace_bytes()
    R, plan = gpu_ladder(L, t2, EMU, R0=R0, budget=int(full * 0.6))
    assert plan.describe()["n_block_pairs"] > 1
    assert rel_fro(R - R0, oracle.ladder(L, t2)) <= TOL_R


@pytest.mark.parametrize("no,nv,nchol", [(1, 1, 1), (1, 2, 3), (2, 1, 5), (4, 9, 1), (6, 65, 17), (9, 33, 130),
                                         (12, 20, 70), (3, 130, 200)])
def test_edge_shapes(no, nv, nchol):
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=no * 1000 + nv)
    R, _ = gpu_ladder(L, t2, EMU)
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL_R


def test_nonsymmetric_L_violates_the_emulated_precondition():
    # The emulated path multiplies only the rows (a <= c) of L^T (L[P] symmetric in (a, c)).
    L, t2 = make_integer_inputs(3, 11, 13, seed=7, symmetric_L=False)
    R, _ = gpu_ladder(L, t2, EMU)
    assert rel_fro(R, oracle.ladder(L, t2)) > 1e-3


def test_deterministic():
    L, t2, _, _ = make_inputs(5, 45, 60, seed=41)
    R1, _ = gpu_ladder(L, t2, EMU)
    R2, _ = gpu_ladder(L, t2, EMU)
    assert np.array_equal(R1, R2)


def test_zero_inputs_give_zero():
    L = np.zeros((7, 11, 11))
    t2 = np.zeros((3, 3, 11, 11))
    R, _ = gpu_ladder(L, t2, EMU)
    assert np.all(R == 0.0)


def test_rejects_unsupported_requests():
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan(5, 19, 72, lad.LADDER_EMU_INT8)
    assert e.value.status == lad.LADDER_ERR_UNSUPPORTED
    for bad in (4, 9):
        with pytest.raises(lad.LadderError) as e:
            lad.ladder_plan(5, 19, 72, EMU, nslices=bad)
        assert e.value.status == lad.LADDER_ERR_ARG


def test_nchol_spanning_several_exact_chunks():
    # nchol > 1024: the ERI accumulates two exact chunks in int64 registers.
    L, t2, _, _ = make_inputs(3, 23, 1500, seed=55)
    R, _ = gpu_ladder(L, t2, EMU)
    assert rel_fro(R, oracle.ladder(L, t2)) <= TOL_R


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_full_size_sampled_parity(name):
    s = CONFIGS[name]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = gpu_ladder(L, t2, EMU)
    check_sampled(R, L, t2, TOL_R, nsample=32)
    assert_pair_symmetry(R, diag_tol=TOL_R)
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    assert E == pytest.approx(oracle.energy(t2, R), rel=1e-12)
    Eg, Fg = _golden_energy(name), _golden(name, "R_fro")
    if Eg is not None:
        assert abs(E - Eg) <= TOL_E
    if Fg is not None:
        assert abs(float(np.linalg.norm(R.ravel())) - Fg) <= TOL_R * Fg


def test_c3_planner_split_is_bitwise_identical():
    # A budget far below the one-batch workspace forces asymmetric a/b blocks at full size.
    s = CONFIGS["c3"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R1, plan1 = gpu_ladder(L, t2, EMU)
    one_block = lad.ladder_plan_dry(s.no, s.nv, s.nchol, EMU, force_n_a=s.nv, force_n_b=s.nv)["ws_bytes"]
    budget = one_block // 5
    Rb, planb = gpu_ladder(L, t2, EMU, budget=budget)
    d = planb.describe()
    assert d["n_block_pairs"] > 1 and planb.workspace_bytes() <= budget
    assert np.array_equal(Rb, R1)


def _emu_run(L, t2, chunk_blocks=None, form=None):
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(no, nv, nchol, EMU)
    if form is not None:
        plan.set_form(form)
    if chunk_blocks is not None:
        plan.set_eri_chunk(chunk_blocks)
    ws = plan.workspace()
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, dev(L), dev(t2), R, ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R.cpu().numpy(), plan.eri_chunk(ws)


@pytest.mark.parametrize("form", [0, 1])
def test_exact_chunk_from_digit_norms_is_bit_identical(form):
    # nchol = 1500 spans two blocks of 1024: the digit-norm bound admits one chunk for the whole
    # K; forcing chunks of 1024 gives the same bits (the exact levels are the same either way, and
    # the per-chunk rounding of the shared tail accumulator stays below the V grid here)
    L, t2, _, _ = make_inputs(4, 40, 1500, seed=61)
    R_long, chunk = _emu_run(L, t2, form=form)
    assert chunk >= 1500
    R_1024, chunk1 = _emu_run(L, t2, chunk_blocks=1, form=form)
    assert chunk1 == 1024
    assert np.array_equal(R_long, R_1024)
    assert rel_fro(R_long, oracle.ladder(L, t2)) <= TOL_R


def test_worst_case_digits_keep_chunks_of_1024():
    # L = 3 everywhere: the top digit of every entry is 48, so two blocks of 1024 would reach
    # 48^2 * 2048 > 2^22 at level 2: the bound must refuse the longer chunk; integer inputs make
    # the result exact, so it must equal the oracle bit for bit
    no, nv, nchol = 2, 9, 2100
    L = np.full((nchol, nv, nv), 3.0)
    rng = np.random.default_rng(9)
    x = rng.integers(-3, 4, size=(no, no, nv, nv)).astype(np.float64)
    t2 = np.ascontiguousarray(x + x.transpose(1, 0, 3, 2))
    R, chunk = _emu_run(L, t2)
    assert chunk == 1024
    assert np.array_equal(R, oracle.ladder(L, t2))


def test_eri_chunk_rejects_bad_limits():
    plan = lad.ladder_plan(3, 20, 30, EMU)
    for bad in (0, 5, -1):
        with pytest.raises(lad.LadderError):
            plan.set_eri_chunk(bad)
