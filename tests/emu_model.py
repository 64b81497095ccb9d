"""Exact-arithmetic CPU model of the emulated-FP64 ladder (test infrastructure).

It restates, in numpy integer arithmetic, the digit-slice scheme that the
CUDA kernels implement, so that tests can (1) check the scheme's error on
small shapes against the FP64 oracle, and (2) pin properties the GPU must
reproduce (integer grids are exact).  It is not the oracle: the oracle is
the plain FP64 definition in ``oracle/``.

Scheme (FP64 emulated by BF16 digit slices, Ozaki-style splitting):

* Row groups of G consecutive rows share one exponent e with
  max|x| < 2^(e-1), so u = x 2^-e lies in (-1/2, 1/2).  The rows of L^T are
  (a, c) with c padded to vp = nv rounded up to 16 (zero pad rows), so the
  groups are 64 consecutive padded rows, as in the kernels.
* N = round_half_even(x 2^(7S - e)) (|N| <= 2^(7S-1)) is written in
  balanced base 128: N = sum_s d_s 128^(S-s), |d_s| <= 64.  Slice plane s
  holds d_s 2^(-7s) (exact in BF16: 7 significant bits).
* A product sum over K of two sliced operands keeps the pairs s + t <= S + 1.
  Levels l = s + t = 2..5 are exact integers while K * (l-1) * 64^2 <= 2^24
  (chunks of K <= 1024): each has its own FP32 accumulator; the levels >= 6
  share a fifth (inexact, weight <= 2^-28 of the leading level).
* ERI (K = nchol): the level sums form I = acc2 2^35 + acc3 2^28 + acc4 2^21
  + acc5 2^14 + round(A6 2^49), V = 2^(e_ac + e_bd - 49) I, where the row
  (a, c) of L^T is taken as (min(a, c), max(a, c)) (the same vector: L^P is
  symmetric; the kernels multiply only those rows).  V is re-sliced
  per pair row (a, b) with the exponent f_ab of the Cauchy-Schwarz bound
  |(ac|bd)| <= max_c ||L_ac|| max_d ||L_bd||.
* Entries where a row of L^T meets itself, V_ab,ba = ||L_ab||^2 and
  V_aa,cc = ||L_ac||^2, are taken from the FP64 squared norms instead: the
  level cut drops the squares d_s d_s there, an error of one sign that would
  add up coherently in E_L.
* Ladder (K = nv^2, chunks of 1024): per chunk J = acc2 2^28 + acc3 2^21
  + acc4 2^14 + acc5 2^7 + round(A6 2^42), summed exactly over chunks in
  int64; R_ij^ab = 2^(f_ab + g_ij - 42) sum J.
"""
from __future__ import annotations

import math

import numpy as np

DIGIT_BITS = 7
GROUP = 64
CHUNK = 1024


def group_exponents(x2d: np.ndarray, group: int = GROUP) -> np.ndarray:
    """e per group of `group` rows: smallest e with max|x| < 2^(e-1) (0 for an all-zero group)."""
    rows = x2d.shape[0]
    ng = (rows + group - 1) // group
    e = np.zeros(ng, dtype=np.int64)
    for g in range(ng):
        m = float(np.max(np.abs(x2d[g * group:(g + 1) * group]))) if x2d.size else 0.0
        if m > 0.0:
            e[g] = math.frexp(m)[1] + 1
    return e


def to_digits(x2d: np.ndarray, S: int, group: int = GROUP):
    """(digits [S, rows, K] int64, row exponent [rows] int64)."""
    e = group_exponents(x2d, group)
    erow = np.repeat(e, group)[: x2d.shape[0]]
    scaled = np.ldexp(x2d, (DIGIT_BITS * S - erow)[:, None])
    N = np.rint(scaled).astype(np.int64)
    d = np.zeros((S,) + x2d.shape, dtype=np.int64)
    for s in range(S - 1, 0, -1):
        low = ((N + 64) & 127) - 64
        d[s] = low
        N = (N - low) >> 7
    d[0] = N
    return d, erow


def from_digits(d: np.ndarray, erow: np.ndarray) -> np.ndarray:
    S = d.shape[0]
    v = np.zeros(d.shape[1:])
    for s in range(S):
        v += np.ldexp(d[s].astype(np.float64), (erow - DIGIT_BITS * (s + 1))[:, None])
    return v


def level_sums(dA: np.ndarray, dB: np.ndarray):
    """Exact integer level sums acc2..acc5 and the weighted tail A6 (float64) of
    sum_k A[m,k] B[n,k] over slice pairs s + t <= S + 1 (s, t 1-based)."""
    S = dA.shape[0]
    z = np.zeros((dA.shape[1], dB.shape[1]), dtype=np.int64)
    acc = {2: z.copy(), 3: z.copy(), 4: z.copy(), 5: z.copy()}
    a6 = np.zeros(z.shape)
    for s in range(1, S + 1):
        for t in range(1, S + 2 - s):
            prod = dA[s - 1] @ dB[t - 1].T
            lvl = s + t
            if lvl <= 5:
                acc[lvl] = acc[lvl] + prod
            else:
                a6 = a6 + np.ldexp(prod.astype(np.float64), -DIGIT_BITS * lvl)
    return acc[2], acc[3], acc[4], acc[5], a6


def _round_shift(I: np.ndarray, sh: np.ndarray) -> np.ndarray:
    """round(I / 2^sh), halves up; sh <= 0 shifts left."""
    out = np.empty_like(I)
    pos = sh > 0
    shp = np.where(pos, sh, 1)
    out[pos] = ((I + (np.int64(1) << (shp - 1))) >> shp)[pos]
    out[~pos] = (I << np.where(pos, 0, -sh))[~pos]
    return out


def pair_exponent_bound(L: np.ndarray) -> np.ndarray:
    """f[a, b] with max_c||L_ac|| max_d||L_bd|| (1 + 2^-20) < 2^(f-1)."""
    nchol, nv, _ = L.shape
    norms = np.sqrt(np.sum(L * L, axis=0))           # [a, c] = ||L[:, a, c]||
    na = norms.max(axis=1)
    f = np.zeros((nv, nv), dtype=np.int64)
    for a in range(nv):
        for b in range(nv):
            B = na[a] * na[b] * (1.0 + 2.0 ** -20)
            f[a, b] = math.frexp(B)[1] + 1 if B > 0 else 0
    return f


def emulated_ladder(L: np.ndarray, t2: np.ndarray, S: int = 6, group: int = GROUP, chunk: int = CHUNK,
                    exact_self: bool = True):
    """R = ladder(L, t2) through the emulation scheme (all pairs, no a <= b packing).

    exact_self=False keeps the truncated level sums on the self-product entries too
    (the uncorrected scheme, for comparison)."""
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    vp = (nv + 15) // 16 * 16                                     # the kernels' padded layout
    Ltp = np.zeros((nv, vp, nchol))
    Ltp[:, :nv, :] = L.transpose(1, 2, 0)                        # rows (a, c padded), K = P
    dLp, eLp = to_digits(Ltp.reshape(nv * vp, nchol), S, group)
    valid = (np.arange(nv)[:, None] * vp + np.arange(nv)[None, :]).ravel()
    dL, eL = dLp[:, valid, :], eLp[valid]
    I = np.zeros((nv * nv, nv * nv), dtype=np.int64)
    for k0 in range(0, nchol, chunk):
        sl = slice(k0, min(nchol, k0 + chunk))
        a2, a3, a4, a5, a6 = level_sums(dL[:, :, sl], dL[:, :, sl])   # [(ac), (bd)]
        I += (a2 << 35) + (a3 << 28) + (a4 << 21) + (a5 << 14) + np.rint(np.ldexp(a6, 49)).astype(np.int64)
    f = pair_exponent_bound(L)
    # rows (a, c), cols (b, d) -> V[(a, b), (c, d)].  L^P is symmetric, so the rows (a, c) and
    # (c, a) of L^T hold the same vector; the kernels multiply only the rows with a <= c, and
    # V_ab,cd comes from the row (min(a, c), max(a, c)) with that row's digits and exponent.
    ar = np.arange(nv)
    lo = np.minimum(ar[:, None], ar[None, :])
    hi = np.maximum(ar[:, None], ar[None, :])
    Ir = I.reshape(nv, nv, nv, nv)                               # [a, c, b, d]
    I4 = Ir[lo, hi].transpose(0, 2, 1, 3)                        # [a, b, c, d]
    e2 = eL.reshape(nv, nv)
    e4 = e2[lo, hi]                                              # e of the row used for (a, c)
    eb = e2                                                      # e of the column row (b, d)
    sh = f[:, :, None, None] - e4[:, None, :, None] - eb[None, :, None, :] + 49 - DIGIT_BITS * S
    Np = _round_shift(I4, sh).reshape(nv * nv, nv * nv)          # rows (a, b), K = (c, d)
    if exact_self:
        sq = np.sum(L * L, axis=0)                               # [a, c] = ||L[:, a, c]||^2
        a_, b_ = np.meshgrid(np.arange(nv), np.arange(nv), indexing="ij")
        Np[a_ * nv + b_, b_ * nv + a_] = np.rint(np.ldexp(sq[a_, b_], DIGIT_BITS * S - f[a_, b_])).astype(np.int64)
        Np[a_ * nv + a_, b_ * nv + b_] = np.rint(np.ldexp(sq[a_, b_], DIGIT_BITS * S - f[a_, a_])).astype(np.int64)
    assert np.all(np.abs(Np) <= (1 << (DIGIT_BITS * S - 1)))
    dV = np.zeros((S,) + Np.shape, dtype=np.int64)
    M = Np.copy()
    for s in range(S - 1, 0, -1):
        low = ((M + 64) & 127) - 64
        dV[s] = low
        M = (M - low) >> 7
    dV[0] = M
    T = t2.reshape(no * no, nv * nv)
    dT, eT = to_digits(T, S, group)
    K = nv * nv
    J = np.zeros((nv * nv, no * no), dtype=np.int64)
    for k0 in range(0, K, chunk):
        sl = slice(k0, min(K, k0 + chunk))
        b2, b3, b4, b5, b6 = level_sums(dV[:, :, sl], dT[:, :, sl])
        J += (b2 << 28) + (b3 << 21) + (b4 << 14) + (b5 << 7) + np.rint(np.ldexp(b6, 42)).astype(np.int64)
    fab = f.reshape(nv * nv)
    Rp = np.ldexp(J.astype(np.float64), fab[:, None] + eT[None, :] - 42)   # [(a, b), (i, j)]
    return Rp.T.reshape(no, no, nv, nv)
