"""ladder_energy_noalloc: the energy entry point for callers that cannot allocate.

Callers running under CUDA graph capture, or inside frameworks that forbid
any allocator but their own, cannot let the library call cudaMalloc.  This
entry point keeps its reduction scratch in a fixed array inside the library.
The test calls it through the C ABI and checks it against ladder_energy (the
plan-based entry point) and against the CPU oracle's E_L, on two calls in a
row, within the tolerance the energy tests use.  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL_E = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def _case(no, nv, nchol, seed):
    L, t2, _, _ = make_inputs(no, nv, nchol, seed)
    td = torch.from_numpy(t2).cuda()
    # Any R works for the energy; use a random one so both entry points see the same data.
    R = torch.from_numpy(np.random.default_rng(seed).standard_normal(t2.shape)).cuda()
    plan = lad.ladder_plan(no, nv, nchol)
    return plan, td, R, oracle.energy(t2, R.cpu().numpy())


def _noalloc_c_abi(td, R):
    E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    no, _, nv, _ = td.shape
    rc = lad.lib().ladder_energy_noalloc(int(no), int(nv), ctypes.c_void_p(td.data_ptr()),
                                        ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == lad.LADDER_OK, lad.ladder_strerror(rc)
    torch.cuda.synchronize()
    return float(E.item())


def test_noalloc_energy_matches_plan_energy_two_calls_in_a_row():
    s = CONFIGS["c1"]
    cases = [_case(s.no, s.nv, s.nchol, s.seed), _case(7, 45, 30, 77)]
    for plan, td, R, E_oracle in cases + cases[::-1]:
        E_ref = lad.ladder_energy(plan, td, R)
        E1 = _noalloc_c_abi(td, R)
        E2 = _noalloc_c_abi(td, R)
        assert abs(E1 - E_ref) <= TOL_E * abs(E_ref)
        assert abs(E1 - E_oracle) <= TOL_E * abs(E_oracle)
        assert E1 == E2


def test_noalloc_energy_rejects_shapes_beyond_its_scratch():
    td = torch.zeros(8, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    # no = 300, nv = 2000: ceil(9e4 * 63^2 / 64) partials >> 16384; rejected before any launch.
    rc = lad.lib().ladder_energy_noalloc(300, 2000, ctypes.c_void_p(td.data_ptr()), ctypes.c_void_p(td.data_ptr()),
                                        ctypes.c_void_p(E.data_ptr()), None)
    assert rc == lad.LADDER_ERR_ARG
    assert lad.lib().ladder_energy_noalloc(0, 10, None, None, None, None) == lad.LADDER_ERR_ARG
