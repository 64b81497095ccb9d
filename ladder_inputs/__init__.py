"""Seeded synthetic inputs for the closed-shell particle-particle ladder.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It draws random numbers and shapes them like the operands
of the ladder term; it contains none of the ladder arithmetic itself.

Operands (all float64, C-contiguous):

* ``L[P, a, c]`` -- Cholesky vectors of the virtual-virtual ERI block
  (``<ab|cd> ~ sum_P L^P_ac L^P_bd``, Sec. "Acceleration of CC calculations",
  Eq. cholesky).  Symmetric in (a, c) because the orbitals are real, with
  entries N(0,1) * exp(-P/24), P zero-based.
* ``t2[i, j, a, b]`` -- doubles amplitudes with ``t_ij^ab = t_ji^ba``, drawn
  N(0, 0.01) (0.01 is the standard deviation) and divided by the orbital
  energy denominator ``2 + e_a + e_b - e_i - e_j`` with
  ``e_occ ~ U(-1.5, -0.3)`` and ``e_vir ~ U(0.2, 3.0)``.

Draw order from ``numpy.random.default_rng(seed)`` (PCG64): e_occ, e_vir,
the Gaussian field G for L, the Gaussian field X for t2.  L mirrors the upper
triangle of G (keeps N(0,1) marginals); t2 symmetrises X as
``(X + X.transpose(1,0,3,2)) / 2`` before dividing by the denominator.  The
denominator is formed as ``(2 + (e_a + e_b)) - (e_i + e_j)`` so that it is
exactly symmetric under the (ij, ab) swap in floating point, which keeps t2
exactly symmetric.  The decay factors exp(-P/24) are computed with Python's
``decimal`` module and rounded once, so they are bit-identical on every
platform.
"""
from __future__ import annotations

import decimal
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CONFIGS",
    "LadderShape",
    "decay_factors",
    "make_inputs",
    "make_integer_inputs",
    "batched_shapes",
    "make_batched_inputs",
]


@dataclass(frozen=True)
class LadderShape:
    no: int
    nv: int
    nchol: int
    seed: int
    name: str = ""


# The workloads: a water/cc-pVDZ-sized case, a case whose packed ERI fits in
# one batch, and a case whose full ERI block exceeds HBM.  Seeds 1234 + k.
CONFIGS = {
    "c1": LadderShape(no=5, nv=19, nchol=72, seed=1235, name="c1"),
    "c2": LadderShape(no=10, nv=200, nchol=630, seed=1236, name="c2"),
    "c3": LadderShape(no=20, nv=400, nchol=1260, seed=1237, name="c3"),
}

BATCHED_SEED = 1239
BATCHED_COUNT = 24


def decay_factors(nchol: int) -> np.ndarray:
    """exp(-P/24) for P = 0..nchol-1, correctly rounded to float64."""
    ctx = decimal.Context(prec=50)
    out = np.empty(nchol, dtype=np.float64)
    for p in range(nchol):
        out[p] = float(ctx.exp(ctx.divide(decimal.Decimal(-p), decimal.Decimal(24))))
    return out


def make_inputs(no: int, nv: int, nchol: int, seed: int, symmetric_t2: bool = True):
    """Return (L, t2, eps_occ, eps_vir) drawn as described in the module docstring.

    ``symmetric_t2=False`` skips the (ij, ab) symmetrisation of the Gaussian
    field; it exists only to show what happens when that precondition is
    violated.
    """
    rng = np.random.default_rng(seed)
    eps_occ = rng.uniform(-1.5, -0.3, size=no)
    eps_vir = rng.uniform(0.2, 3.0, size=nv)
    g = rng.standard_normal(size=(nchol, nv, nv))
    x = rng.normal(0.0, 0.01, size=(no, no, nv, nv))

    iu = np.triu_indices(nv)
    L = np.empty_like(g)
    for p in range(nchol):
        up = np.zeros((nv, nv))
        up[iu] = g[p][iu]
        sym = up + np.triu(up, 1).T
        L[p] = sym
    L *= decay_factors(nchol)[:, None, None]

    if symmetric_t2:
        s = (x + x.transpose(1, 0, 3, 2)) / 2.0
    else:
        s = x
    eab = eps_vir[:, None] + eps_vir[None, :]          # e_a + e_b (exactly symmetric)
    eij = eps_occ[:, None] + eps_occ[None, :]          # e_i + e_j (exactly symmetric)
    denom = (2.0 + eab)[None, None, :, :] - eij[:, :, None, None]
    t2 = s / denom
    return (np.ascontiguousarray(L), np.ascontiguousarray(t2), eps_occ, eps_vir)


def make_device_inputs(no: int, nv: int, nchol: int, seed: int, device="cuda"):
    """(L, t2) as torch float64 tensors drawn on the GPU with the same distributions and
    symmetries as ``make_inputs`` (torch's generator, so not the same numbers): for timing runs
    at shapes whose host-side generation would take minutes.  Not used for parity.  L is drawn
    in chunks of Cholesky vectors and t2 symmetrised pair by pair in place, so the device holds
    little more than L and t2 themselves while they are drawn."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)
    eps_occ = torch.empty(no, **f64).uniform_(-1.5, -0.3, generator=gen)
    eps_vir = torch.empty(nv, **f64).uniform_(0.2, 3.0, generator=gen)
    decay = torch.tensor(decay_factors(nchol), **f64)
    L = torch.empty((nchol, nv, nv), **f64)
    chunk = max(1, (1 << 27) // max(1, nv * nv))      # ~1 GB of draws at a time
    for p0 in range(0, nchol, chunk):
        p1 = min(nchol, p0 + chunk)
        g = torch.randn((p1 - p0, nv, nv), generator=gen, **f64)
        L[p0:p1] = torch.triu(g) + torch.triu(g, 1).transpose(1, 2)
        L[p0:p1] *= decay[p0:p1, None, None]
        del g
    t2 = torch.empty((no, no, nv, nv), **f64)
    for i in range(no):
        t2[i].normal_(0.0, 0.01, generator=gen)
    for i in range(no):                                # (X + X.transpose(1,0,3,2)) / 2, pair by pair
        for j in range(i, no):
            s = (t2[i, j] + t2[j, i].transpose(0, 1)) / 2.0
            t2[i, j] = s
            t2[j, i] = s.transpose(0, 1)
    eab = eps_vir[:, None] + eps_vir[None, :]
    eij = eps_occ[:, None] + eps_occ[None, :]
    for i in range(no):
        t2[i] /= (2.0 + eab)[None, :, :] - eij[i, :, None, None]
    return L, t2


def make_integer_inputs(no: int, nv: int, nchol: int, seed: int, lo: int = -3, hi: int = 3,
                        symmetric_L: bool = True, symmetric_t2: bool = True):
    """Integer-valued operands (entries in [lo, hi]) for exact-arithmetic checks."""
    rng = np.random.default_rng(seed)
    g = rng.integers(lo, hi + 1, size=(nchol, nv, nv)).astype(np.float64)
    x = rng.integers(lo, hi + 1, size=(no, no, nv, nv)).astype(np.float64)
    if symmetric_L:
        iu = np.triu_indices(nv)
        L = np.empty_like(g)
        for p in range(nchol):
            up = np.zeros((nv, nv))
            up[iu] = g[p][iu]
            L[p] = up + np.triu(up, 1).T
    else:
        L = g
    if symmetric_t2:
        # Copy the (i<=j)-half onto its (j,i,b,a) mirror so that t stays integer.
        t2 = x.copy()
        for i in range(no):
            for j in range(no):
                if j < i:
                    t2[i, j] = x[j, i].T
                elif j == i:
                    m = x[i, i]
                    iu = np.triu_indices(nv)
                    up = np.zeros((nv, nv))
                    up[iu] = m[iu]
                    t2[i, i] = up + np.triu(up, 1).T
    else:
        t2 = x
    return np.ascontiguousarray(L), np.ascontiguousarray(t2)


def batched_shapes(seed: int = BATCHED_SEED, count: int = BATCHED_COUNT):
    """Shapes of the uneven batch: no ~ U{5..30}, nv ~ U{60..320}, nchol = 3(no+nv)."""
    rng = np.random.default_rng(seed)
    no = rng.integers(5, 31, size=count)
    nv = rng.integers(60, 321, size=count)
    return [LadderShape(no=int(o), nv=int(v), nchol=int(3 * (o + v)),
                        seed=seed * 1000 + k, name=f"b{k}")
            for k, (o, v) in enumerate(zip(no, nv))]


def make_batched_inputs(shapes):
    """Per-instance (L, t2) for a list of LadderShape, each from its own seed."""
    out = []
    for s in shapes:
        L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
        out.append((L, t2))
    return out
