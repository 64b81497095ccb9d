"""Whole-R parity at the one-batch workload (no=10, nv=200, nchol=630, seed 1236): every
element of R from the GPU against the CPU oracle's plain FP64 loops (Eq. vfunction-chol), for
the native FP64 path (rebuild order through HBM and the fused on-chip kernel) and for both forms
of the emulated path.

The oracle's R is computed once per module (about 2.3e12 flops: a minute or two on a
many-core host) and pinned first to its own stored E_L and ||R||_F (tests/golden, written by
oracle/make_golden.py).  Tolerances: ||R - R_oracle||_F / ||R_oracle||_F <= 1e-12 (FP64),
<= 1e-10 (emulated), |E_L - E_L(oracle)| <= 1e-8 Eh; a <= b mirror symmetry exact.
"""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs
from conftest import rel_fro
from test_gpu_fp64 import _golden, assert_pair_symmetry, dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def c2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()
    s = CONFIGS["c2"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    ref = oracle.ladder(L, t2)
    E_ref = oracle.energy(t2, ref)
    assert E_ref == pytest.approx(_golden("c2", "E_L"), abs=1e-9)
    assert float(np.linalg.norm(ref.ravel())) == pytest.approx(_golden("c2", "R_fro"), rel=1e-13)
    return s, L, t2, ref, E_ref


def _run(s, L, t2, precision, form=None, path=None):
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(s.no, s.nv, s.nchol, precision)
    if path is not None:
        plan.set_path(path)
        assert plan.path() == path
    if form is not None:
        plan.set_form(form)
        assert plan.form() == form
    Ld, td = dev(L), dev(t2)
    R = torch.zeros_like(td)
    ws = plan.workspace()
    lad.ladder_apply(plan, Ld, td, R, ws)
    E = lad.ladder_energy(plan, td, R)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    out = R.cpu().numpy()
    del ws, R
    plan.close()
    return out, E


@pytest.mark.parametrize("path", ["fp64", "fp64_fused", "emu_plain", "emu_split"])
def test_c2_whole_R_against_the_oracle(c2, path):
    s, L, t2, ref, E_ref = c2
    if path.startswith("fp64"):
        R, E = _run(s, L, t2, lad.LADDER_FP64,
                    path=lad.LADDER_PATH_FUSED if path == "fp64_fused" else lad.LADDER_PATH_ERI)
        tol, diag = 1e-12, None
    else:
        R, E = _run(s, L, t2, lad.LADDER_EMU_BF16, form=0 if path == "emu_plain" else 1)
        tol, diag = 1e-10, 1e-10
    assert rel_fro(R, ref) <= tol
    # no element far off either: the largest element error against the largest element
    assert np.max(np.abs(R - ref)) <= 10 * tol * np.max(np.abs(ref))
    assert abs(E - E_ref) <= 1e-8
    assert_pair_symmetry(R, diag_tol=diag)
