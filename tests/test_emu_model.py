"""CPU checks of the emulation scheme's model (tests/emu_model.py) against the oracle.

The model restates the digit-slice scheme of the emulated-FP64 path in exact
integer arithmetic; these tests pin it to the FP64 oracle on small shapes, so
that the GPU comparisons against the model rest on a checked scheme.
"""
import numpy as np

import oracle
from conftest import rel_fro
from emu_model import emulated_ladder
from ladder_inputs import make_inputs, make_integer_inputs


def _errors(L, t2, **kw):
    ref = oracle.ladder(L, t2)
    R = emulated_ladder(L, t2, **kw)
    E = oracle.energy(t2, ref)
    return rel_fro(R, ref), abs(oracle.energy(t2, R) - E), abs(E)


def test_scheme_meets_the_stated_tolerances():
    L, t2, _, _ = make_inputs(5, 19, 72, 1235)
    dr, de, _ = _errors(L, t2, S=6)
    assert dr <= 1e-10
    assert de <= 1e-8


def test_integer_grid_is_exact():
    # Integer inputs small enough that no digit is dropped: every level sum is exact.
    L, t2 = make_integer_inputs(3, 9, 12, seed=2)
    assert np.array_equal(emulated_ladder(L, t2, S=6), oracle.ladder(L, t2))


def test_self_product_entries_remove_the_energy_bias():
    # Without the FP64 squared norms on V_ab,ba and V_aa,cc the dropped squares bias those
    # entries low and the energy error is coherent: about the size of the relative R error.
    L, t2, _, _ = make_inputs(8, 24, 100, 3)
    dr0, de0, E = _errors(L, t2, S=6, exact_self=False)
    dr1, de1, _ = _errors(L, t2, S=6, exact_self=True)
    assert de0 / E > 2e-12
    assert de1 / E < 5e-13
    assert dr1 <= dr0 * 1.01


def test_more_slices_reduce_the_error():
    # Each slice adds 7 bits up to S = 6; beyond that the fixed-point units of the
    # recombination (2^-49 in the ERI, 2^-42 in the ladder) set a floor near 1e-12.
    L, t2, _, _ = make_inputs(4, 15, 40, 9)
    errs = [_errors(L, t2, S=S)[0] for S in (5, 6, 7)]
    assert errs[0] > 50 * errs[1]
    assert errs[1] > 5 * errs[2]
