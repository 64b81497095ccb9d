"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: numpy's einsum of
the definition, exact integer arithmetic, closed forms, symmetries that the
mathematics fixes, linearity, and an independent trace formula for E_L.
The sizes are tiny so that pure-Python and einsum evaluations stay cheap.
"""
import math

import numpy as np
import pytest

import oracle
from ladder_inputs import make_inputs, make_integer_inputs, decay_factors, CONFIGS
from conftest import rel_fro


def _general(no, nv, nchol, seed):
    """Non-symmetric operands: catches index transpositions a symmetric L or t would hide."""
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((nchol, nv, nv))
    t2 = rng.standard_normal((no, no, nv, nv))
    return L, t2


@pytest.mark.parametrize("no,nv,nchol,seed", [(2, 4, 3, 1), (3, 5, 7, 2), (2, 7, 9, 3), (1, 1, 1, 4)])
def test_definition_matches_einsum(no, nv, nchol, seed):
    # Eq. vfunction-chol: R[i,j,a,b] = sum_{P,c,d} L[P,a,c] L[P,b,d] t2[i,j,c,d]
    L, t2 = _general(no, nv, nchol, seed)
    ref = np.einsum("pac,pbd,ijcd->ijab", L, L, t2, optimize=False)
    got = oracle.ladder(L, t2)
    assert rel_fro(got, ref) <= 1e-14


def test_definition_matches_einsum_c1_shape():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    ref = np.einsum("pac,pbd,ijcd->ijab", L, L, t2, optimize=True)
    got = oracle.ladder(L, t2)
    assert rel_fro(got, ref) <= 1e-13


def _exact_python(Li, ti):
    """Brute force with Python integers (exact)."""
    nchol, nv, _ = Li.shape
    no = ti.shape[0]
    L = [[[int(Li[p, a, c]) for c in range(nv)] for a in range(nv)] for p in range(nchol)]
    t = [[[[int(ti[i, j, c, d]) for d in range(nv)] for c in range(nv)] for j in range(no)] for i in range(no)]
    R = np.zeros((no, no, nv, nv))
    for a in range(nv):
        for b in range(nv):
            V = [[sum(L[p][a][c] * L[p][b][d] for p in range(nchol)) for d in range(nv)] for c in range(nv)]
            for i in range(no):
                for j in range(no):
                    R[i, j, a, b] = float(sum(V[c][d] * t[i][j][c][d] for c in range(nv) for d in range(nv)))
    return R


@pytest.mark.parametrize("sym", [True, False])
def test_integer_inputs_exact(sym):
    L, t2 = make_integer_inputs(3, 5, 6, seed=11, symmetric_L=sym, symmetric_t2=sym)
    got = oracle.ladder(L, t2)
    ref = _exact_python(L, t2)
    assert np.array_equal(got, ref)


def test_single_cholesky_vector_closed_form():
    # X = 1: R_ij = L0 T_ij L0^T for any (not necessarily symmetric) L0.
    L, t2 = _general(3, 6, 1, 5)
    ref = np.einsum("ac,ijcd,bd->ijab", L[0], t2, L[0])
    for i in range(3):
        for j in range(3):
            np.testing.assert_allclose(L[0] @ t2[i, j] @ L[0].T, ref[i, j], rtol=1e-13, atol=1e-13)
    assert rel_fro(oracle.ladder(L, t2), ref) <= 1e-14


def test_one_hot_amplitudes():
    # t_{i0 j0}^{c0 d0} = t_{j0 i0}^{d0 c0} = 1, else 0  =>  R_{i0 j0}^{ab} = (a c0|b d0).
    no, nv, nchol = 3, 5, 4
    L, _, _, _ = make_inputs(no, nv, nchol, seed=7)
    i0, j0, c0, d0 = 0, 2, 1, 3
    t2 = np.zeros((no, no, nv, nv))
    t2[i0, j0, c0, d0] = 1.0
    t2[j0, i0, d0, c0] = 1.0
    R = oracle.ladder(L, t2)
    for a in range(nv):
        for b in range(nv):
            v1 = math.fsum(L[p, a, c0] * L[p, b, d0] for p in range(nchol))
            v2 = math.fsum(L[p, a, d0] * L[p, b, c0] for p in range(nchol))
            assert R[i0, j0, a, b] == pytest.approx(v1, rel=1e-14, abs=1e-15)
            assert R[j0, i0, a, b] == pytest.approx(v2, rel=1e-14, abs=1e-15)
    mask = np.ones((no, no), dtype=bool)
    mask[i0, j0] = mask[j0, i0] = False
    assert np.all(R[mask] == 0.0)


def test_stored_eri_route_and_gram_structure():
    no, nv, nchol = 2, 6, 5
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=8)
    V = oracle.eri(L)
    np.testing.assert_allclose(V, np.einsum("pac,pbd->abcd", L, L), rtol=1e-14, atol=1e-14)
    # (ac|bd) as a matrix over (ac) x (bd) is a Gram matrix: symmetric positive semi-definite.
    G = V.transpose(0, 2, 1, 3).reshape(nv * nv, nv * nv)
    assert np.array_equal(G, G.T)
    w = np.linalg.eigvalsh(G)
    assert w.min() >= -1e-12 * w.max()
    assert np.linalg.matrix_rank(G, tol=1e-10 * w.max()) <= nchol
    assert rel_fro(oracle.ladder_stored(V, t2), oracle.ladder(L, t2)) <= 1e-15


def test_eri_eightfold_symmetry_for_symmetric_L():
    L, _, _, _ = make_inputs(1, 6, 5, seed=9)
    V = oracle.eri(L)  # V[a,b,c,d] = (ac|bd)
    np.testing.assert_allclose(V, V.transpose(2, 1, 0, 3), rtol=0, atol=1e-14)  # (ca|bd)
    np.testing.assert_allclose(V, V.transpose(0, 3, 2, 1), rtol=0, atol=1e-14)  # (ac|db)
    np.testing.assert_allclose(V, V.transpose(1, 0, 3, 2), rtol=0, atol=1e-14)  # (bd|ac)


def test_pair_symmetry_requires_symmetric_amplitudes():
    # R_ij^ab = R_ji^ba follows from t_ij^cd = t_ji^dc and (bd|ac) = (ac|bd) alone.
    no, nv, nchol = 3, 6, 5
    rng = np.random.default_rng(10)
    L = rng.standard_normal((nchol, nv, nv))  # deliberately not symmetric in (a, c)
    _, t2, _, _ = make_inputs(no, nv, nchol, seed=10)
    R = oracle.ladder(L, t2)
    assert rel_fro(R.transpose(1, 0, 3, 2), R) <= 1e-14
    _, t2n, _, _ = make_inputs(no, nv, nchol, seed=10, symmetric_t2=False)
    Rn = oracle.ladder(L, t2n)
    assert rel_fro(Rn.transpose(1, 0, 3, 2), Rn) > 1e-2


def test_linearity_and_power_of_two_scaling():
    no, nv, nchol = 2, 5, 4
    L, t1, _, _ = make_inputs(no, nv, nchol, seed=12)
    _, t2b, _, _ = make_inputs(no, nv, nchol, seed=13)
    al, be = 0.37, -1.25
    lhs = oracle.ladder(L, al * t1 + be * t2b)
    rhs = al * oracle.ladder(L, t1) + be * oracle.ladder(L, t2b)
    assert rel_fro(lhs, rhs) <= 1e-13
    # Scaling by powers of two commutes with every rounding: exact.
    assert np.array_equal(oracle.ladder(2.0 * L, t1), 4.0 * oracle.ladder(L, t1))
    assert np.array_equal(oracle.ladder(L, -t1), -oracle.ladder(L, t1))


def test_accumulates_into_R():
    no, nv, nchol = 2, 5, 4
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=14)
    R0 = np.random.default_rng(15).standard_normal((no, no, nv, nv))
    inc = oracle.ladder(L, t2)
    got = oracle.ladder(L, t2, R0)
    np.testing.assert_allclose(got - R0, inc, rtol=1e-12, atol=1e-15)


def test_pairs_mode_is_bitwise_the_full_mode():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R = oracle.ladder(L, t2)
    a = [0, 3, 18, 7, 7]
    b = [0, 11, 2, 7, 18]
    out = oracle.ladder_pairs(L, t2, a, b)
    for k in range(len(a)):
        assert np.array_equal(out[k], R[:, :, a[k], b[k]])


def test_energy_definition_and_trace_formula():
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R = oracle.ladder(L, t2)
    E = oracle.energy(t2, R)
    # Direct definition with exactly rounded summation.
    U = 2.0 * t2 - t2.transpose(0, 1, 3, 2)
    E_fsum = math.fsum((U * R).ravel())
    assert E == pytest.approx(E_fsum, rel=1e-14, abs=1e-16)
    # Independent of R: E = sum_P sum_ij tr(U_ij^T L_P T_ij L_P^T).
    E_tr = 0.0
    for p in range(s.nchol):
        Lp = L[p]
        for i in range(s.no):
            for j in range(s.no):
                E_tr += float(np.sum(U[i, j] * (Lp @ t2[i, j] @ Lp.T)))
    assert E == pytest.approx(E_tr, rel=1e-11)


def test_energy_of_random_R():
    rng = np.random.default_rng(16)
    t2 = rng.standard_normal((3, 3, 4, 4))
    R = rng.standard_normal((3, 3, 4, 4))
    E = oracle.energy(t2, R)
    ref = math.fsum(((2.0 * t2 - t2.transpose(0, 1, 3, 2)) * R).ravel())
    assert E == pytest.approx(ref, rel=1e-15, abs=1e-15)


def test_factorised_path_agrees_at_c1():
    # Independent algorithm: R_ij = sum_P L_P T_ij L_P^T (numpy BLAS), Eq. vfunction-chol
    # evaluated through the x o^2 v^2 intermediate instead of the v^4 one.
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R = np.zeros_like(t2)
    for p in range(s.nchol):
        R += np.einsum("ac,ijcd,bd->ijab", L[p], t2, L[p], optimize=True)
    assert rel_fro(oracle.ladder(L, t2), R) <= 1e-13


def test_generators():
    L, t2, eo, ev = make_inputs(3, 7, 10, seed=1)
    assert np.array_equal(L, L.transpose(0, 2, 1))
    assert np.array_equal(t2, t2.transpose(1, 0, 3, 2))
    L2, t22, _, _ = make_inputs(3, 7, 10, seed=1)
    assert np.array_equal(L, L2) and np.array_equal(t2, t22)
    f = decay_factors(100)
    for p in (0, 1, 24, 99):
        assert abs(f[p] - math.exp(-p / 24.0)) <= 2.0 * math.ulp(f[p])
    assert eo.min() >= -1.5 and eo.max() <= -0.3 and ev.min() >= 0.2 and ev.max() <= 3.0
    Li, ti = make_integer_inputs(2, 4, 3, seed=2)
    assert np.array_equal(Li, Li.transpose(0, 2, 1)) and np.array_equal(ti, ti.transpose(1, 0, 3, 2))
    assert np.all(Li == np.round(Li)) and np.all(np.abs(ti) <= 3)
