// Emulated-FP64 path: both contractions of the ladder run on the tcgen05
// tensor cores as BF16 digit-slice products with FP32 accumulation in TMEM,
// recombined exactly in integer arithmetic; FP64 is used only to scale the
// final integer sums into R.
//
// Digit slices (FP64 emulation by splitting, the approach the introduction
// cites for Blackwell; this file fixes the variant): rows of an operand are
// grouped (64 rows per group) and share one power-of-two exponent e with
// max|x| < 2^(e-1).  N = rint(x 2^(7S-e)) is written in balanced base 128,
// N = sum_s d_s 128^(S-s) with |d_s| <= 64, and slice plane s holds the BF16
// value d_s 2^(-7s) (7 significant bits: exact).  A product sum over K keeps
// the slice pairs with s + t <= S + 1.  Every product d_s d_t fits in 12 bits,
// so each level sum l = s + t (l - 1 pairs) is an exact FP32 integer times
// 2^(-7l) while K (l - 1) 2^12 <= 2^24.  Levels 2..5 therefore get one exact
// TMEM accumulator each over chunks of K <= 1024; the levels >= 6 (weight
// <= 2^-28 of the leading level) share a fifth accumulator whose FP32
// rounding (the tensor core truncates while aligning) stays below 2^-40.
// Exactness of the leading levels does not depend on how the hardware rounds.
//
// ERI (C-split step 0, 'xac,xbd->acbd'): rows (a,c) and columns (b,d) of the
// Gram matrix of L^T, K = nchol in chunks of 1024.  Per chunk the epilogue adds
// I = acc2 2^35 + acc3 2^28 + acc4 2^21 + acc5 2^14 + rn(A6 2^49) into int64
// registers; V = 2^(e_ac + e_bd - 49) I.  V is re-sliced for the ladder with
// one exponent per (a,b) row taken from the Cauchy-Schwarz bound
// |(ac|bd)| <= max_c ||L_ac|| max_d ||L_bd|| (the ERI is a Gram matrix), so no
// pass over a whole V row is needed before slicing.  The O(nv) entries per pair row
// where a row of L^T meets itself (V_ab,ba and V_aa,cc) are rewritten from FP64 squared
// norms: the level cut drops squares there, a one-signed error (eri_self_kernel).
//
// Ladder (C-split step 1, 'acbd,ecfd->efab'): rows (a,b), columns (i,j),
// K = (c,d) = nv^2 in chunks of 1024.  Per chunk J = acc2 2^28 + acc3 2^21 +
// acc4 2^14 + acc5 2^7 + rn(A6 2^42); chunk sums are added in int64 (exact, so
// the order of the split-K atomics does not matter and the result is
// deterministic).  R_ij^ab += 2^(f_ab + g_ij - 42) sum J and the mirror
// R_ji^ba gets the same value.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "ladder_internal.h"
#include "tc_common.cuh"

namespace ladder {
namespace {

using namespace tc;

constexpr int kG = kExpGroupRows;  // rows per exponent group
constexpr int kEpiWarps = 12;      // ladder epilogue warps (3 per TMEM lane quadrant)
constexpr int kEpiPerQuad = kEpiWarps / 4;
constexpr int kLadRuns = 6 / kEpiPerQuad;   // 16-column chunks per epilogue warp
constexpr int kThreadsTC = 32 * (2 + kEpiWarps);
constexpr int kEriEpiWarps = 12;   // ERI epilogue warps (3 per TMEM lane quadrant)
constexpr int kThreadsEri = 32 * (2 + kEriEpiWarps);
constexpr int kEriRuns = kEmuTileN / (kEriEpiWarps / 4) / 8;  // runs of 8 columns per epilogue warp
static_assert(kEriRuns % 2 == 0, "runs are stored in sector pairs");
constexpr int kNumAcc = 5;         // exact levels 2, 3, 4, 5 and the shared levels >= 6
constexpr int kTmemCols = 512;     // 5 accumulators x 96 columns, rounded up to a power of two
constexpr int kAccStride = kEmuTileN;  // TMEM columns between accumulators
constexpr int kSmemBudget = 210 * 1024;

__host__ __device__ constexpr int bk_for(int S) { return S <= 6 ? 32 : 16; }
// ERI stage width (K columns per pipeline stage) and the most stages it keeps in flight.
constexpr int kEriBK = 32;
constexpr int kEriMaxStages = 4;
__host__ __device__ constexpr int eri_bk_for(int S) { return S <= 6 ? kEriBK : 16; }
// One stage: S planes of a 128-row tile (A) and S planes of a <= 96-row tile (B), BK columns.
__host__ __device__ constexpr int stage_bytes(int S) { return S * (kEmuTile + kEmuTileN) * bk_for(S) * 2; }
// ERI stage on a CTA pair: 128 rows of A and half (48 rows) of the 96-row B tile per CTA.
__host__ __device__ constexpr int eri_stage_bytes(int S) { return S * (kEmuTile + kEmuTileN / 2) * eri_bk_for(S) * 2; }
__host__ __device__ constexpr int eri_stages_for(int S) {
    return kSmemBudget / eri_stage_bytes(S) < kEriMaxStages ? kSmemBudget / eri_stage_bytes(S) : kEriMaxStages;
}
__host__ __device__ constexpr int eri_smem_bytes_for(int S) { return eri_stages_for(S) * eri_stage_bytes(S) + 1024; }
// Ladder on CTA pairs: the same per-CTA stage shape with the ladder's stage width.
__host__ __device__ constexpr int pair_stage_bytes(int S) { return S * (kEmuTile + kEmuTileN / 2) * bk_for(S) * 2; }
__host__ __device__ constexpr int pair_stages_for(int S) {
    return kSmemBudget / pair_stage_bytes(S) < 4 ? kSmemBudget / pair_stage_bytes(S) : 4;
}
__host__ __device__ constexpr int pair_smem_bytes_for(int S) { return pair_stages_for(S) * pair_stage_bytes(S) + 1024; }
__host__ __device__ constexpr int stages_for(int S) {
    return kSmemBudget / stage_bytes(S) < 4 ? kSmemBudget / stage_bytes(S) : 4;
}
__host__ __device__ constexpr int smem_bytes_for(int S) { return stages_for(S) * stage_bytes(S) + 1024; }

// ------------------------------------------------------------------ digits
// Balanced base-128 digits of N (|N| <= 2^(7S-1)) as BF16 plane values d_s 2^(-7s).
__device__ __forceinline__ float small_int_to_float(int v) {
    // exact for |v| < 2^22: 1.5 * 2^23 + v has an ulp of 1
    return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }  // 2^k, |k| < 127

template <int S>
__device__ __forceinline__ void digits_of(long long N, __nv_bfloat16 (&out)[S]) {
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
        const int low = (int)(((N + 64) & 127)) - 64;
        N = (N - low) >> 7;
        out[s] = __float2bfloat16_rn(small_int_to_float(low) * pow2f(-7 * (s + 1)));
    }
    out[0] = __float2bfloat16_rn(small_int_to_float((int)N) * pow2f(-7));
}

// round(I / 2^sh) with halves rounded up (sh <= 0 multiplies); values beyond
// +-lim cannot occur for a valid exponent bound and are clamped and flagged.
__device__ __forceinline__ long long rescale(long long I, int sh, long long lim, unsigned* status) {
    long long N;
    bool bad = false;
    if (sh > 62) {
        N = 0;
    } else if (sh > 0) {
        N = (I + (1LL << (sh - 1))) >> sh;
    } else {
        const int k = -sh;
        const unsigned long long mag = I < 0 ? (unsigned long long)(-I) : (unsigned long long)I;
        if (k >= 62 || (mag >> (62 - k)) != 0) {
            bad = I != 0;
            N = I < 0 ? -lim : (I > 0 ? lim : 0);
        } else {
            N = I << k;
        }
    }
    if (N > lim || N < -lim) {
        bad = true;
        N = N > 0 ? lim : -lim;
    }
    if (bad) atomicOr(status, kStatusNumeric);
    return N;
}

// round-half-even(x * 2^k) from the IEEE bits of x, with integer arithmetic only (the FP64
// conversion units are slow on this GPU).  Requires |x 2^k| < 2^62.
__device__ __forceinline__ long long scaled_rint(double x, int k) {
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (e ? (1LL << 52) : 0LL);
    const int ee = (e ? e : 1) - 1075 + k;  // |x| = m 2^(e - 1075)
    long long r;
    if (m == 0) {
        r = 0;
    } else if (ee >= 0) {
        r = m << (ee < 10 ? ee : 10);
    } else if (ee < -54) {
        r = 0;
    } else {
        const int sh = -ee;
        const long long q = m >> sh, rem = m & ((1LL << sh) - 1), half = 1LL << (sh - 1);
        r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
    return bits < 0 ? -r : r;
}

__device__ __forceinline__ int exponent_above(double m) {
    // smallest e with m < 2^(e-1); 0 for m == 0
    if (!(m > 0.0)) return 0;
    int E;
    frexp(m, &E);
    return E + 1;
}

// Balanced digits through a biased integer: with B = 64 (1 + 128 + ... + 128^(S-2)),
// N + B = sum_{s>=1} (d_s + 64) 128^(S-1-s) + d_0 128^(S-1) holds the digits d_s + 64 in
// [0, 127] as plain 7-bit fields, so each lower digit is a shift, a mask and one FFMA that
// turns the field u into the float (u - 64) 2^(-7(s+1)) (exponent-bias trick: the float with
// bits 0x4B400000 | u equals 1.5 2^23 + u).  d_0 is the arithmetic top of N + B.
template <int S>
__host__ __device__ constexpr long long digit_bias() {
    long long b = 0;
    for (int s = 1; s < S; ++s) b = b * 128 + 64;
    return b;
}

// Re-slices one run of 8 int64 values I (unit 2^(-sh) of the plane grid) into S planes of
// paired BF16 digits: N = round(I 2^-sh) (halves up), then the digits of N.  The fast path
// covers 1 <= sh <= 63 - 7S, where I + 2^(sh-1) + B 2^sh cannot overflow (|I| < 2^(sh+7S-1));
// other shifts take the general rescale.  A top digit beyond +-64 (an exponent bound that
// does not hold) is flagged.
template <int S>
__device__ __forceinline__ void slice_run(const long long (&I)[8], int sh, __nv_bfloat162 (&out)[S][4],
                                          unsigned* status) {
    constexpr long long B = digit_bias<S>();
    long long Nb[8];
    if (sh >= 1 && sh <= 63 - 7 * S) {
        const long long add = (1LL << (sh - 1)) + (B << sh);
#pragma unroll
        for (int k = 0; k < 8; ++k) Nb[k] = (I[k] + add) >> sh;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) Nb[k] = rescale(I[k], sh, 1LL << (7 * S - 1), status) + B;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        float f0[S], f1[S];
#pragma unroll
        for (int s = 1; s < S; ++s) {
            const int sft = 7 * (S - 1 - s);
            const float sc = pow2f(-7 * (s + 1)), off = -12582976.0f * sc;  // (1.5 2^23 + 64) 2^(-7(s+1))
            const uint32_t u0 = (uint32_t)((unsigned long long)Nb[k] >> sft) & 127u;
            const uint32_t u1 = (uint32_t)((unsigned long long)Nb[k + 1] >> sft) & 127u;
            f0[s] = fmaf(__uint_as_float(0x4B400000u | u0), sc, off);
            f1[s] = fmaf(__uint_as_float(0x4B400000u | u1), sc, off);
        }
        const int t0 = (int)(Nb[k] >> (7 * (S - 1))), t1 = (int)(Nb[k + 1] >> (7 * (S - 1)));
        bad |= (unsigned)(t0 + 64) > 128u || (unsigned)(t1 + 64) > 128u;
        f0[0] = fmaf(__int_as_float(0x4B400000 + t0), 0x1p-7f, -12582912.0f * 0x1p-7f);
        f1[0] = fmaf(__int_as_float(0x4B400000 + t1), 0x1p-7f, -12582912.0f * 0x1p-7f);
#pragma unroll
        for (int s = 0; s < S; ++s) out[s][k >> 1] = __floats2bfloat162_rn(f0[s], f1[s]);
    }
    if (bad) atomicOr(status, kStatusNumeric);
}

// N = round(I 2^-sh) (halves up) of one run of 8 int64 values, kept as integers (the V of the
// symmetric/antisymmetric form, which is combined before it is sliced), with the range check of
// slice_run.
template <int S>
__device__ __forceinline__ void round_run(const long long (&I)[8], int sh, long long (&N)[8], unsigned* status) {
    constexpr long long B = digit_bias<S>();
    if (sh >= 1 && sh <= 63 - 7 * S) {
        const long long add = 1LL << (sh - 1);
#pragma unroll
        for (int k = 0; k < 8; ++k) N[k] = (I[k] + add) >> sh;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) N[k] = rescale(I[k], sh, 1LL << (7 * S - 1), status);
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) bad |= (unsigned)((int)((N[k] + B) >> (7 * (S - 1))) + 64) > 128u;
    if (bad) atomicOr(status, kStatusNumeric);
}

// One 32-byte streaming store (a whole L2 sector), 32-byte aligned address.
__device__ __forceinline__ void st_cs_32B(void* ptr, const uint4& lo, const uint4& hi) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(ptr), "r"(lo.x), "r"(lo.y), "r"(lo.z),
                 "r"(lo.w), "r"(hi.x), "r"(hi.y), "r"(hi.z), "r"(hi.w)
                 : "memory");
}

// ------------------------------------------------------------------ prep kernels
// One block of 64 threads per group of 64 L^T rows r = (a,c): the group's exponent and,
// per row, ||L[:, a, c]||^2 (kept for the self-product entries of the ERI) and ||L[:, a, c]||
// folded into max_c by an atomic max on the IEEE bits.
// Rows are padded: r = a*vp + c, c < vp, the pad rows (c >= nv) are zero.
__global__ void __launch_bounds__(64) lt_rowstats_kernel(const double* __restrict__ L, int nchol, int nv, int vp,
                                                         int* __restrict__ lt_exp,
                                                         unsigned long long* __restrict__ lnorm_bits,
                                                         double* __restrict__ lsq) {
    const long long nv2 = (long long)nv * nv, rows = (long long)nv * vp;
    const long long r = (long long)blockIdx.x * kG + threadIdx.x;
    const int a = (int)(r / vp), c = (int)(r % vp);
    const bool valid = r < rows && c < nv;
    double m = 0.0, ss = 0.0;
    if (valid)
        for (int P = 0; P < nchol; ++P) {
            const double x = __ldg(L + (size_t)P * nv2 + (size_t)a * nv + c);
            m = fmax(m, fabs(x));
            ss = fma(x, x, ss);
        }
    __shared__ double red[2];
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) lt_exp[blockIdx.x] = exponent_above(fmax(red[0], red[1]));
    if (valid) {
        lsq[(size_t)a * nv + c] = ss;
        atomicMax(lnorm_bits + a, (unsigned long long)__double_as_longlong(sqrt(ss)));
    }
}

// f[a][b]: smallest f with max_c||L_ac|| max_d||L_bd|| (1 + 2^-20) < 2^(f-1).
__global__ void f_table_kernel(const unsigned long long* __restrict__ lnorm_bits, int nv, int* __restrict__ f) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)nv * nv) return;
    const double na = __longlong_as_double((long long)lnorm_bits[k / nv]);
    const double nb = __longlong_as_double((long long)lnorm_bits[k % nv]);
    f[k] = exponent_above(na * nb * (1.0 + 0x1p-20));
}

// L^T slices of the Cholesky vectors [pbase, pbase + nchol): tile of 64 P x 64 rows through shared
// memory; writes planes[s][r][P - pbase] (row stride xpad).
template <int S>
__global__ void __launch_bounds__(256) lt_slice_kernel(const double* __restrict__ L, int pbase, int nchol, int nv,
                                                       int vp, int xpad, const int* __restrict__ lt_exp,
                                                       __nv_bfloat16* __restrict__ planes,
                                                       unsigned* __restrict__ norm2, int nblk, unsigned* status) {
    __shared__ double tile[64][65];
    const long long nv2 = (long long)nv * nv, rows = (long long)nv * vp;
    const int P0 = blockIdx.x * 64;
    const long long r0 = (long long)blockIdx.y * 64;
    for (int i = threadIdx.x; i < 64 * 64; i += 256) {
        const int p = i >> 6, rr = i & 63;
        const long long r = r0 + rr;
        const int c = (int)(r % vp);
        tile[p][rr] = (P0 + p < nchol && r < rows && c < nv)
                          ? __ldg(L + (size_t)(pbase + P0 + p) * nv2 + (size_t)(r / vp) * nv + c)
                          : 0.0;
    }
    __syncthreads();
    const int rr = threadIdx.x >> 2, pseg = (threadIdx.x & 3) * 16;
    const long long r = r0 + rr;
    const int e = r < rows ? lt_exp[r0 / kG] : 0;
    const size_t plane = (size_t)rows * xpad;
    const int P0t = P0 + pseg;
    __align__(16) __nv_bfloat16 out[S][16];
    unsigned sq[S];
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) sq[s2] = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        __nv_bfloat16 d[S];
        digits_of<S>(scaled_rint(tile[pseg + k][rr], 7 * S - e), d);
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
            out[s2][k] = d[s2];
            const int di = __float2int_rn(__bfloat162float(d[s2]) * pow2f(7 * (s2 + 1)));   // the digit
            sq[s2] += (unsigned)(di * di);
        }
    }
    // Squared digit norms of this row over the block's 64 P (the four threads of a row are
    // adjacent lanes), added into the row's 1024-wide block of K: the exact-chunk bound.
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
        sq[s2] += __shfl_xor_sync(0xffffffffu, sq[s2], 1);
        sq[s2] += __shfl_xor_sync(0xffffffffu, sq[s2], 2);
    }
    if (r >= rows) return;
    if ((threadIdx.x & 3) == 0) {
        const int blk = P0 / kEmuChunkK;
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2)
            if (sq[s2] != 0) atomicAdd(norm2 + ((size_t)s2 * rows + r) * nblk + blk, sq[s2]);
    }
    if (P0t >= nchol) return;
    if (P0t + 16 <= xpad) {
        // 16 consecutive P of one row: two 16-byte stores per plane (xpad % 8 == 0, P0t % 16 == 0)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
            if (!LADDER_IN_BOUNDS((size_t)r * xpad + P0t + 16 <= plane, status)) continue;
            uint4* dst = reinterpret_cast<uint4*>(planes + s2 * plane + (size_t)r * xpad + P0t);
            dst[0] = reinterpret_cast<const uint4*>(out[s2])[0];
            dst[1] = reinterpret_cast<const uint4*>(out[s2])[1];
        }
    } else {
        for (int k = 0; k < 16 && P0t + k < xpad; ++k)
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2)
                if (LADDER_IN_BOUNDS((size_t)r * xpad + P0t + k < plane, status))
                    planes[s2 * plane + (size_t)r * xpad + P0t + k] = out[s2][k];
    }
}

// Exact chunk length of the ERI (K = nchol) from the digit norms.  A level-l accumulator sums, over
// the chunk, the products d_s d_t (s + t = l - 2, 0-based planes) of a row and a column of L^T; by
// Cauchy-Schwarz every partial sum of it is at most sum_{s+t} |d_s| |d_t| <= sum_{s+t} M_s M_t,
// where M_s is the largest 2-norm over rows of plane s's digits in one chunk-aligned window of K.
// Chunks of 1024 meet the limits (l - 1) 2^22 of levels 2..5 for any digits (|d| <= 64); a window
// of c blocks of 1024 (c = 2, 3, 4) is taken when its norms meet the same limits, so that every level
// sum stays an exact FP32 integer and the 32-bit pairings of the epilogue cannot overflow.
// cand[(c-2) S + s] = max over rows and aligned windows of c blocks of the squared norm of plane s.
constexpr int kEriMaxChunkBlocks = 4;

__global__ void __launch_bounds__(256) eri_chunk_norms_kernel(const unsigned* __restrict__ norm2, long long rows,
                                                              int S, int nblk, unsigned* __restrict__ cand) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int s2 = 0; s2 < S; ++s2) {
        unsigned best[kEriMaxChunkBlocks - 1] = {0, 0, 0};
        if (r < rows) {
            const unsigned* row = norm2 + ((size_t)s2 * rows + r) * nblk;
            for (int c = 2; c <= kEriMaxChunkBlocks; ++c)
                for (int w0 = 0; w0 < nblk; w0 += c) {
                    unsigned sum = 0;
                    for (int b = w0; b < w0 + c && b < nblk; ++b) sum += row[b];
                    best[c - 2] = max(best[c - 2], sum);
                }
        }
        for (int c = 0; c < kEriMaxChunkBlocks - 1; ++c) {
            unsigned v = best[c];
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0 && v != 0) atomicMax(cand + c * S + s2, v);
        }
    }
}

// One thread: the largest window (in blocks of 1024, at most max_blocks) that meets the limits,
// as K blocks of the ERI's stage width per chunk.
__global__ void eri_chunk_select_kernel(const unsigned* __restrict__ cand, int S, int max_blocks, int bk,
                                        int* __restrict__ kb_per_chunk) {
    int chosen = 1;
    for (int c = min(max_blocks, kEriMaxChunkBlocks); c >= 2 && chosen == 1; --c) {
        bool ok = true;
        for (int j = 0; j < 4 && ok; ++j) {   // accumulator j: level j + 2, planes s + t = j
            double bound = 0.0;
            for (int s2 = 0; s2 <= j && s2 < S; ++s2) {
                const int t = j - s2;
                if (t >= S) continue;
                bound += sqrt((double)cand[(c - 2) * S + s2]) * sqrt((double)cand[(c - 2) * S + t]);
            }
            ok = bound * (1.0 + 1e-9) + 1.0 <= (double)(j + 1) * 4194304.0;   // (l - 1) 2^22
        }
        if (ok) chosen = c;
    }
    *kb_per_chunk = chosen * kEmuChunkK / bk;
}

// max |T| per group of 64 T rows, via atomic max on the IEEE bits (T viewed [no^2][nv^2]).
__global__ void __launch_bounds__(256) t_rowmax_kernel(const double* __restrict__ t2, long long K, int rows,
                                                       unsigned long long* __restrict__ gmax) {
    const int row = blockIdx.y;
    const long long k0 = (long long)blockIdx.x * 8192;
    double m = 0.0;
    for (long long k = k0 + threadIdx.x; k < K && k < k0 + 8192; k += 256)
        m = fmax(m, fabs(__ldg(t2 + (size_t)row * K + k)));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(gmax + row / kG, (unsigned long long)__double_as_longlong(m));
}

__global__ void exp_from_max_kernel(const unsigned long long* __restrict__ gmax, int n, int* __restrict__ e) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) e[g] = exponent_above(__longlong_as_double((long long)gmax[g]));
}

// T slices: 8 consecutive k of one row per thread; planes[s][row][k] (row stride kpad).
// K index k = c*vp + d of a row; zero for the pad columns d >= nv.
template <int S>
__global__ void __launch_bounds__(256) t_slice_kernel(const double* __restrict__ t2, int nv, int vp, int rows,
                                                      int kpad, const int* __restrict__ t_exp,
                                                      __nv_bfloat16* __restrict__ planes, unsigned* status) {
    const long long per_row = kpad / 8;
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= per_row * rows) return;
    const int row = (int)(u / per_row);
    const long long k0 = (u % per_row) * 8;
    const int c = (int)(k0 / vp), d0 = (int)(k0 % vp);  // vp % 8 == 0: the 8 columns share c
    const int e = t_exp[row / kG];
    const size_t plane = (size_t)rows * kpad;
    const double* src = t2 + ((size_t)row * nv + c) * nv;
    __align__(16) __nv_bfloat16 out[S][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int dd = d0 + j;
        const double x = dd < nv ? __ldg(src + dd) : 0.0;
        __nv_bfloat16 dg[S];
        digits_of<S>(scaled_rint(x, 7 * S - e), dg);
#pragma unroll
        for (int s = 0; s < S; ++s) out[s][j] = dg[s];
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (LADDER_IN_BOUNDS((size_t)row * kpad + k0 + 8 <= plane, status))
            *reinterpret_cast<uint4*>(planes + s * plane + (size_t)row * kpad + k0) = *reinterpret_cast<uint4*>(out[s]);
}

// ------------------------------------------------------------------ symmetric/antisymmetric form
// With t_ij^cd = t_ji^dc the ladder splits into a part symmetric and a part antisymmetric in
// (i,j), each over c <= d only:
//   X_ij^ab = sum_{c<=d} V'_ab,cd T'_ij,cd   (i <= j),  V' = V_cd + V_dc (c < d), V_cc (c = d),
//                                                        T' = (T_ij,cd + T_ji,cd) / 2 (c < d), T_ij,cc
//   Y_ij^ab = sum_{c<d}  V''_ab,cd T''_ij,cd  (i < j),  V'' = V_cd - V_dc, T'' = (T_ij,cd - T_ji,cd) / 2
//   R_ij^ab = X + Y,  R_ji^ab = X - Y,
// half the multiply-adds of the plain ladder.  The rows (i <= j) are packed row-major,
// r(i,j) = i no - i(i-1)/2 + (j - i), and (i < j) the same without the diagonal; K' and K''
// are packed in word pairs of slots (pm_base), so that V' and V'' go out in 4-byte stores.

// (i, j) of packed row r of the upper triangle of an n x n grid (diag: with the diagonal).
__device__ __forceinline__ void tri_unpack(int r, int n, bool diag, int* i, int* j) {
    int a = 0, len = diag ? n : n - 1;
    while (r >= len && len > 0) {
        r -= len;
        ++a;
        --len;
    }
    *i = a;
    *j = a + r + (diag ? 0 : 1);
}

// One block per packed row of T' (r < np) or T'' (r >= np): max |value| into its 64-row group.
__global__ void __launch_bounds__(256) tpm_rowmax_kernel(const double* __restrict__ t2, int no, int nv, int np,
                                                         unsigned long long* __restrict__ gmax_p,
                                                         unsigned long long* __restrict__ gmax_m) {
    __shared__ int si, sj;
    const bool plus = (int)blockIdx.x < np;
    const int r = plus ? (int)blockIdx.x : (int)blockIdx.x - np;
    if (threadIdx.x == 0) tri_unpack(r, no, plus, &si, &sj);
    __syncthreads();
    const int i = si, j = sj;
    const long long nv2 = (long long)nv * nv;
    const double* tij = t2 + ((size_t)i * no + j) * nv2;
    const double* tji = t2 + ((size_t)j * no + i) * nv2;
    double m = 0.0;
    for (long long f = threadIdx.x; f < nv2; f += blockDim.x) {
        const int c = (int)(f / nv), d = (int)(f % nv);
        if (c > d || (!plus && c == d)) continue;
        const double a = __ldg(tij + f), b = __ldg(tji + f);
        const double v = plus ? (c == d ? a : 0.5 * (a + b)) : 0.5 * (a - b);
        m = fmax(m, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax((plus ? gmax_p : gmax_m) + r / kG, (unsigned long long)__double_as_longlong(m));
}

// T' and T'' digit planes: one block per packed row (i,j).
template <int S>
__global__ void __launch_bounds__(128) tpm_slice_kernel(const double* __restrict__ t2, int no, int nv, int np,
                                                        long long kp_pad, long long km_pad, int nm,
                                                        const int* __restrict__ e_p, const int* __restrict__ e_m,
                                                        __nv_bfloat16* __restrict__ tp, __nv_bfloat16* __restrict__ tm,
                                                        unsigned* status) {
    __shared__ int si, sj;
    const bool plus = (int)blockIdx.x < np;
    const int r = plus ? (int)blockIdx.x : (int)blockIdx.x - np;
    if (threadIdx.x == 0) tri_unpack(r, no, plus, &si, &sj);
    __syncthreads();
    const int i = si, j = sj;
    const long long nv2 = (long long)nv * nv;
    const double* tij = t2 + ((size_t)i * no + j) * nv2;
    const double* tji = t2 + ((size_t)j * no + i) * nv2;
    const int e = plus ? e_p[r / kG] : e_m[r / kG];
    const long long kpad = plus ? kp_pad : km_pad;
    const size_t plane = (size_t)(plus ? np : nm) * kpad;
    __nv_bfloat16* out = (plus ? tp : tm) + (size_t)r * kpad;
    const int dend = 2 * ((nv - 1) / 2) + 1;   // last slot of every row's last word
    // Rows c in turn, threads over its slots (coalesced reads of t_ij and t_ji, coalesced stores).
    for (int c = 0; c < (plus ? nv : nv - 1); ++c) {
        const long long k0 = pm_base(c, nv, plus);
        const int dlo = plus ? c : c + 1;
        for (int d = (dlo & ~1) + (int)threadIdx.x; d <= dend; d += blockDim.x) {   // whole words
            double v = 0.0;   // the slots outside the row get zero
            if (d >= dlo && d < nv) {
                const double a = __ldg(tij + (size_t)c * nv + d), b = __ldg(tji + (size_t)c * nv + d);
                v = plus ? (c == d ? a : 0.5 * (a + b)) : 0.5 * (a - b);
            }
            __nv_bfloat16 dg[S];
            digits_of<S>(scaled_rint(v, 7 * S - e), dg);
            const long long k = k0 + d;
            if (!LADDER_IN_BOUNDS((size_t)r * kpad + k < plane, status)) continue;
#pragma unroll
            for (int s = 0; s < S; ++s) out[s * plane + k] = dg[s];
        }
    }
}

struct CombineArgs {
    int nv, vp, npairs, ntile;        // ntile = 32-wide tiles per (c or d) axis
    size_t pplane, mplane;            // element strides between planes of V', V''
    long long kpad, kp_pad, km_pad;   // row strides of V (int64), V', V''
    const long long* vi;
    __nv_bfloat16* vp_out;
    __nv_bfloat16* vm_out;
    unsigned* status;
};

// Bits [SFT, SFT + W) of two unsigned values, the first in the low and the second in the high
// 16-bit half.  A field inside one 16-bit window of the same 32-bit word of both values takes
// one byte permute and a shift; otherwise each value is shifted first.
template <int SFT, int W>
__device__ __forceinline__ uint32_t field_pair(unsigned long long b0, unsigned long long b1) {
    constexpr uint32_t mask = ((1u << W) - 1u) * 0x00010001u;
    constexpr int k = SFT / 8, r = SFT - 8 * k;
    uint32_t v;
    if constexpr (k <= 2) {
        v = __byte_perm((uint32_t)b0, (uint32_t)b1, k | (k + 1) << 4 | (k + 4) << 8 | (k + 5) << 12) >> r;
    } else if constexpr (k >= 4 && k <= 6) {
        v = __byte_perm((uint32_t)(b0 >> 32), (uint32_t)(b1 >> 32), (k - 4) | (k - 3) << 4 | k << 8 | (k + 1) << 12) >> r;
    } else {
        v = __byte_perm((uint32_t)(b0 >> SFT), (uint32_t)(b1 >> SFT), 0x5410);
    }
    return v & mask;
}

__device__ __forceinline__ uint32_t bf16x2_fma(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// BF16 pairs (x, x) of 2^e and of -192 2^e = -1.5 2^(e+7).
__host__ __device__ constexpr uint32_t bf16_pair_pow2(int e) { return (uint32_t)((e + 127) << 7) * 0x00010001u; }
__host__ __device__ constexpr uint32_t bf16_pair_m192(int e) {
    return (uint32_t)(0x8000 | ((e + 134) << 7) | 0x40) * 0x00010001u;
}

// Digit planes of two slots as BF16 pairs: word s holds digit s of N0 in its low half and of N1
// in its high half (the slot order in memory); the digits of digits_of.  With the bias
// B + 64 128^(S-1), every digit, the top one included, is a plain field u of the biased value
// (d_s = u - 64; u <= 127 below the top, <= 128 at the top).  The BF16 with bits 0x4300 | u is
// 128 + u exactly, so one BF16x2 FMA per plane, (128 + u) 2^-k - 192 2^-k, gives the digit
// values d 2^-k of both slots exactly (k = 7(s+1)).
template <int S>
__device__ __forceinline__ void digit_words(long long N0, long long N1, uint32_t (&w)[S]) {
    constexpr long long Bt = digit_bias<S>() + (64LL << (7 * (S - 1)));
    const unsigned long long b0 = (unsigned long long)(N0 + Bt), b1 = (unsigned long long)(N1 + Bt);
    constexpr uint32_t m128 = 0x43004300u;
    w[0] = bf16x2_fma(field_pair<7 * (S - 1), 8>(b0, b1) | m128, bf16_pair_pow2(-7), bf16_pair_m192(-7));
#pragma unroll
    for (int s = 1; s < S; ++s) {
        uint32_t f;
        switch (S - 1 - s) {   // field position, a compile-time constant after unrolling
            case 0: f = field_pair<0, 7>(b0, b1); break;
            case 1: f = field_pair<7, 7>(b0, b1); break;
            case 2: f = field_pair<14, 7>(b0, b1); break;
            case 3: f = field_pair<21, 7>(b0, b1); break;
            case 4: f = field_pair<28, 7>(b0, b1); break;
            case 5: f = field_pair<35, 7>(b0, b1); break;
            default: f = field_pair<42, 7>(b0, b1); break;
        }
        w[s] = bf16x2_fma(f | m128, bf16_pair_pow2(-7 * (s + 1)), bf16_pair_m192(-7 * (s + 1)));
    }
}

// V' and V'' of every pair row of a block from its int64 V (N on the grid of exponent f_ab), on
// the grid of exponent f_ab + 1: N' = round((N_cd + N_dc) / 2) (c < d) or round(N_cc / 2),
// N'' = round((N_cd - N_dc) / 2), halves rounded up, so |N'|, |N''| <= 2^(7S-1) and the digits
// stay within +-64.  One block per (pair row, 32x32 tile of (c,d) with c-tile <= d-tile), in
// row-major tile order so that the blocks writing neighbouring segments of a V' row run at the
// same time (their partial sectors meet in L2); the tile and its transpose pass through shared
// memory so that every global access is a row segment, and each thread writes whole words
// (slots d, d + 1) of the packed V' and V''.  128 threads: with 17 KB of shared memory per
// block, twelve blocks per SM keep their loads in flight together.
constexpr int kCombineThreads = 128;

template <int S>
__global__ void __launch_bounds__(kCombineThreads) vpm_combine_kernel(CombineArgs p) {
    __shared__ long long ta[32][33], tb[32][33];   // ta[c][d] = N(c,d), tb[d][c] = N(d,c)
    __shared__ long long base_p[32], base_m[32];  // pm_base of the tile's rows c
    const long long ntp = (long long)p.ntile * (p.ntile + 1) / 2;
    const long long blk = blockIdx.x;
    const int row = (int)(blk / ntp);
    int tc, td;
    tri_unpack((int)(blk % ntp), p.ntile, true, &tc, &td);
    const int c0 = tc * 32, d0 = td * 32;
    // 16-byte streaming loads of two columns (vp % 8 == 0: a pair never straddles vp; the pad
    // columns nv <= d < vp are read but not used).
    for (int t = threadIdx.x; t < 2 * 32 * 16; t += kCombineThreads) {
        const int q = t & 15, u = (t >> 4) & 31, which = t >> 9;
        const int rr = (which == 0 ? c0 : d0) + u, col0 = (which == 0 ? d0 : c0) + 2 * q;
        long long (*dst)[33] = which == 0 ? ta : tb;
        longlong2 x = make_longlong2(0, 0);
        if (rr < p.nv && col0 < p.vp)
            x = __ldcs(reinterpret_cast<const longlong2*>(p.vi + (size_t)row * p.kpad + (size_t)rr * p.vp + col0));
        dst[u][2 * q] = x.x;
        dst[u][2 * q + 1] = x.y;
    }
    if (threadIdx.x < 32) {
        base_p[threadIdx.x] = pm_base(c0 + threadIdx.x, p.nv, true);
        base_m[threadIdx.x] = pm_base(c0 + threadIdx.x, p.nv, false);
    }
    __syncthreads();
    uint32_t* const outp = reinterpret_cast<uint32_t*>(p.vp_out + (size_t)row * p.kp_pad);
    uint32_t* const outm = reinterpret_cast<uint32_t*>(p.vm_out + (size_t)row * p.km_pad);
    const size_t pw = p.pplane / 2, mw = p.mplane / 2;   // plane strides in words
    // Items (c row u, word of slots d = d0 + 2k, d + 1): a warp covers 16 words of two rows.
    for (int t = threadIdx.x; t < 32 * 16; t += kCombineThreads) {
        const int u = t >> 4, k = t & 15;
        const int c = c0 + u, d = d0 + 2 * k;
        if (c >= p.nv || d >= p.nv) continue;
        const bool in1 = d + 1 < p.nv;
        const long long a0 = ta[u][2 * k], a1 = ta[u][2 * k + 1], b0 = tb[2 * k][u], b1 = tb[2 * k + 1][u];
        uint32_t w[S];
        if (d + 1 >= c) {   // a word of row c of V'
            const long long n0 = d < c ? 0 : ((d > c ? a0 + b0 : a0) + 1) >> 1;
            const long long n1 = in1 ? ((d + 1 > c ? a1 + b1 : a1) + 1) >> 1 : 0;
            digit_words<S>(n0, n1, w);
            const long long wi = (base_p[u] + d) >> 1;
            if (LADDER_IN_BOUNDS(((size_t)row * p.kp_pad >> 1) + wi < pw, p.status))
#pragma unroll
                for (int s = 0; s < S; ++s) outp[s * pw + wi] = w[s];
        }
        if (d >= c && c < p.nv - 1) {   // a word of row c of V''
            const long long n0 = d > c ? (a0 - b0 + 1) >> 1 : 0;
            const long long n1 = in1 ? (a1 - b1 + 1) >> 1 : 0;
            digit_words<S>(n0, n1, w);
            const long long wi = (base_m[u] + d) >> 1;
            if (LADDER_IN_BOUNDS(((size_t)row * p.km_pad >> 1) + wi < mw, p.status))
#pragma unroll
                for (int s = 0; s < S; ++s) outm[s * mw + wi] = w[s];
        }
    }
}

// R from X (rows i <= j) and Y (rows i < j) of one block pair: R_ij^ab += X + Y, R_ji^ab += X - Y,
// and the mirrors R_ji^ba = R_ij^ab, R_ij^ba = R_ji^ab for a < b.  Grid: x over pairs, y over rows.
__global__ void __launch_bounds__(256) finalize_pm_kernel(const unsigned long long* __restrict__ rpx,
                                                          const unsigned long long* __restrict__ rpy, int npairs,
                                                          int no, int nv, int np, int nm,
                                                          const int2* __restrict__ pairs,
                                                          const int* __restrict__ f_tab,
                                                          const int* __restrict__ e_p, const int* __restrict__ e_m,
                                                          double* __restrict__ R, unsigned* status) {
    __shared__ int si, sj;
    const size_t total = (size_t)no * no * nv * nv;
    (void)total;
    for (int r = blockIdx.y; r < np; r += gridDim.y) {
        __syncthreads();
        if (threadIdx.x == 0) tri_unpack(r, no, true, &si, &sj);
        __syncthreads();
        const int i = si, j = sj;
        const int r2 = r - (i + 1);   // (i, j) among the rows with i < j
        for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < npairs; m += gridDim.x * blockDim.x) {
            const int2 ab = pairs[m];
            const int f = f_tab[ab.x * nv + ab.y] + 1;
            const double X = ldexp((double)(long long)rpx[(size_t)m * np + r], f + e_p[r / kG] - 42);
            const double Y = i < j ? ldexp((double)(long long)rpy[(size_t)m * nm + r2], f + e_m[r2 / kG] - 42) : 0.0;
            const size_t ij_ab = (((size_t)i * no + j) * nv + ab.x) * nv + ab.y;
            const size_t ji_ab = (((size_t)j * no + i) * nv + ab.x) * nv + ab.y;
            const size_t ji_ba = (((size_t)j * no + i) * nv + ab.y) * nv + ab.x;
            const size_t ij_ba = (((size_t)i * no + j) * nv + ab.y) * nv + ab.x;
            if (LADDER_IN_BOUNDS(ij_ab < total, status)) R[ij_ab] += X + Y;
            if (i < j && LADDER_IN_BOUNDS(ji_ab < total, status)) R[ji_ab] += X - Y;
            if (ab.x < ab.y) {
                if (LADDER_IN_BOUNDS(ji_ba < total, status)) R[ji_ba] += X + Y;
                if (i < j && LADDER_IN_BOUNDS(ij_ba < total, status)) R[ij_ba] += X - Y;
            }
        }
    }
}

// ------------------------------------------------------------------ shared tcgen05 pieces
struct Ring {
    int stage = 0;
    uint32_t phase = 0;
    __device__ __forceinline__ void next(int stages) {
        if (++stage == stages) {
            stage = 0;
            phase ^= 1u;
        }
    }
};

// Issue the S(S+1)/2 slice-pair MMAs of one stage (BK / 16 K-steps) into the 5 accumulators.
// The shared-memory descriptors are built once per stage; each MMA only adds the plane
// and K-step offset (in 16-byte units) to the start-address field.
// a_group_bytes: distance of the 8-row core groups of A (0: dense planes).
template <int S, bool PAIR = false, int BK = bk_for(S)>
__device__ __forceinline__ void issue_pairs(uint32_t tmem, uint32_t sA, uint32_t sB, uint32_t a_plane_bytes,
                                            uint32_t b_plane_bytes, uint32_t idesc, bool (&first)[kNumAcc],
                                            uint32_t a_group_bytes = 0) {
    const uint64_t da = smem_desc_kmajor(sA, BK * 2, a_group_bytes), db = smem_desc_kmajor(sB, BK * 2);
    const uint32_t ap = a_plane_bytes >> 4, bp = b_plane_bytes >> 4;
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int t = 0; t + s < S; ++t) {
                const int j = (s + t + 2 < 6 ? s + t + 2 : 6) - 2;
                const uint64_t ad = da + (uint64_t)(s * ap + kk * 2);
                const uint64_t bd = db + (uint64_t)(t * bp + kk * 2);
                if (PAIR)
                    mma_bf16_pair(tmem + j * kAccStride, ad, bd, idesc, first[j] ? 0u : 1u);
                else
                    mma_bf16(tmem + j * kAccStride, ad, bd, idesc, first[j] ? 0u : 1u);
                first[j] = false;
            }
        }
    }
}

// Accumulator j holds level j+2 (exact, value = integer * 2^(-7(j+2))) for j < 4 and the levels
// >= 6 (rounded) for j = 4.  The exact levels are integers of magnitude <= K (l-1) 2^12 <= 2^24
// (K <= 1024), so the pairs acc2 2^7 + acc3 and acc4 2^7 + acc5 stay below 2^30 and
// 3 2^29 + 2^24 < 2^31: they are formed in 32-bit arithmetic and only the two pair sums and the
// rounded tail are widened, in the fixed-point unit 2^(-7 U).
__device__ __forceinline__ int acc_int(uint32_t bits, int lvl) {
    return __float2int_rn(__uint_as_float(bits) * pow2f(7 * lvl));
}
template <int U>
__device__ __forceinline__ long long acc_head(uint32_t b2, uint32_t b3) {
    return (long long)(acc_int(b2, 2) * 128 + acc_int(b3, 3)) << (7 * (U - 3));
}
// round-half-even(f 2^k) for |f 2^k| < 2^40 with 32-bit conversions only (a 64-bit conversion
// runs on this GPU's slow FP64 pipe): t = f 2^(k-16) splits exactly into its integer part q and
// fraction r, and f 2^k = q 2^16 + r 2^16 with q 2^16 even, so rounding r 2^16 rounds the sum.
__device__ __forceinline__ long long f32_scaled_rint(float f, int k) {
    const float t = f * pow2f(k - 16);
    const int q = __float2int_rz(t);
    const float r = t - (float)q;
    return ((long long)q << 16) + __float2int_rn(r * 65536.0f);
}
template <int U>
__device__ __forceinline__ long long acc_tail(int i4, uint32_t b5, uint32_t b6) {
    return ((long long)(i4 * 128 + acc_int(b5, 5)) << (7 * (U - 5))) + f32_scaled_rint(__uint_as_float(b6), 7 * U);
}

// Work of one ERI launch: up to kMaxItems items (an instance's block pair each), every one with
// its own L^T tensor maps and tables, and one list of tiles over all of them, so a single
// persistent launch covers several instances.
constexpr int kMaxItems = 32;

// Rows of L^T per ERI tile: 256 rows as 32 chunks of 8 consecutive rows (one TMA box each).
constexpr int kEriChunkRows = 8;
constexpr int kEriTileChunks = 2 * kEmuTile / kEriChunkRows;

struct EriItem {
    int nv, vp, nchol, a0, na, b0, nb, kpad;
    size_t plane_stride;  // elements between V planes
    const int2* chunks;   // (first L^T row, rows) of every chunk, kEriTileChunks per row tile
    const int* row_start;
    const int* lt_exp;
    const int* f_tab;
    __nv_bfloat16* vplanes;
    long long* vint;      // non-null: V as int64 N (row stride kpad) instead of digit planes
    const int* kbc;       // K blocks (of the stage width) per exact chunk, chosen on the device
    int acc_mode;         // int64 V over batches of Cholesky vectors: 3 one batch (round), 0 first
                          // (store the raw sums), 1 middle (add), 2 last (add, then round)
};

struct EriBatch {
    CUtensorMap ta[kMaxItems];  // L^T slices, 8-row boxes (A chunks)
    CUtensorMap tb[kMaxItems];  // L^T slices, 48-row boxes (B)
    EriItem item[kMaxItems];
    const int4* entries;        // (row tile, column tile, item, 0)
    int nentries, nitems;
    unsigned* status;
    unsigned long long wait_ns; // limit of every bounded mbarrier wait (ns of the global timer)
};

// ------------------------------------------------------------------ ERI kernel
// L^P is symmetric, so the rows (x,y) = x vp + y and (y,x) of L^T hold the same vector and the
// Gram matrix only needs the rows with x <= y: (xy|bd) is V_xb at column y vp + d (x in the
// block's a range, b >= x) and V_yb at column x vp + d (y in the a range, x < y, b >= y).
// A CTA pair computes one 256-row x 96-column (b,d) tile with 2-SM MMAs (cta_group::2,
// M = 256); the tile's rows are 32 chunks of 8 consecutive L^T rows taken from the row
// segments the block needs.  CTA r holds chunks [16r, 16r+16) (A) and B rows [48r, 48r+48)
// of every stage and the accumulators of its 128 rows.  In shared memory a stage's A part is
// [chunk][plane][8 rows][BK]: one 3-D TMA box per chunk, and every plane is a K-major operand
// whose 8-row groups lie S*8*BK*2 bytes apart.  Both CTAs' TMA loads complete on the leader's
// (rank 0) full barrier; the leader issues the MMAs and its commits release the stage and
// publish the accumulators in both CTAs; the epilogue warps of both CTAs release the
// accumulators to the leader.  K = nchol runs in exact chunks (kbc stages each).  CTA pair c runs
// the entries c, c + pairs, ...: at any time the pairs work on neighbouring entries, which share
// the band's row tiles and a few column tiles in L2.
template <int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreadsEri, 1)
    eri_emu_kernel(const __grid_constant__ EriBatch B) {
    constexpr int BK = eri_bk_for(S), STAGES = eri_stages_for(S);
    constexpr int CPC = kEmuTile / kEriChunkRows;                       // chunks per CTA
    constexpr uint32_t AGROUP = kEriChunkRows * BK * 2;                 // 8 rows of one plane
    constexpr uint32_t ACHUNK = S * AGROUP, BPLANE = (kEmuTileN / 2) * BK * 2;
    constexpr uint32_t ABYTES = CPC * ACHUNK;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[STAGES], empty[STAGES], acc_full, acc_empty, done;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);   // leader: its producer's arrive + both CTAs' bytes
            mbar_init(&empty[i], 1);  // the leader's multicast commit
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 2 * kEriEpiWarps);
        mbar_init(&done, 1);
        fence_barrier_init();
        for (int i = 0; i < B.nitems; ++i) {
            tma_prefetch_desc(&B.ta[i]);
            tma_prefetch_desc(&B.tb[i]);
        }
    }
    if (warp == 1) tmem_alloc_pair(&tmem_base, kTmemCols);
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    bool failed = false;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer (both CTAs).  The row tiles of a band are re-read by every
        // column tile of the band: they are kept in L2 (evict-last) ahead of the B columns, which
        // pass through, and of the V planes, which are written once and streamed.
        Ring ring;
        bool ok = true;
        const uint64_t keep = policy_evict_last();
        for (int e = cluster; e < B.nentries && ok; e += nclusters) {
            const int4 en = B.entries[e];
            const EriItem& p = B.item[en.z];
            const int nkb = (p.nchol + BK - 1) / BK;
            int arow[CPC];
            const int2* ch = p.chunks + (size_t)en.x * kEriTileChunks + CPC * (int)rank;
#pragma unroll
            for (int c = 0; c < CPC; ++c) arow[c] = ch[c].x;
            const int brow = p.b0 * p.vp + en.y * kEmuTileN + (kEmuTileN / 2) * (int)rank;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                if (!(ok = mbar_wait(&empty[ring.stage], ring.phase ^ 1u, B.status, kStatusTimeout, B.wait_ns))) break;
                unsigned char* st = smem + ring.stage * eri_stage_bytes(S);
                if (rank == 0) mbar_arrive_expect_tx(&full[ring.stage], 2 * eri_stage_bytes(S));
                const uint32_t fb = mapa_rank(smem_u32(&full[ring.stage]), 0);
#pragma unroll
                for (int c = 0; c < CPC; ++c)
                    tma_load_3d_2sm_hint(st + c * ACHUNK, &B.ta[en.z], fb, kb * BK, arow[c], 0, keep);
                tma_load_3d_2sm(st + ABYTES, &B.tb[en.z], fb, kb * BK, brow, 0);
                ring.next(STAGES);
            }
        }
        failed = !ok;
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // ---------------- MMA issuer (leader CTA only)
        Ring ring;
        const uint32_t idesc = idesc_bf16_f32(2 * kEmuTile, kEmuTileN);
        bool ok = true;
        int it = 0;
        for (int e = cluster; e < B.nentries && ok; e += nclusters) {
            const EriItem& p = B.item[B.entries[e].z];
            const int nkb = (p.nchol + BK - 1) / BK;
            const int kb_per_chunk = *p.kbc;
            const int nch = (nkb + kb_per_chunk - 1) / kb_per_chunk;
            for (int ch = 0; ch < nch && ok; ++ch, ++it) {
                if (!(ok = mbar_wait(&acc_empty, (uint32_t)(it & 1) ^ 1u, B.status, kStatusTimeout, B.wait_ns))) break;
                tc_fence_after();
                bool first[kNumAcc] = {true, true, true, true, true};
                const int kb1 = min((ch + 1) * kb_per_chunk, nkb);
                for (int kb = ch * kb_per_chunk; kb < kb1 && ok; ++kb) {
                    if (!(ok = mbar_wait(&full[ring.stage], ring.phase, B.status, kStatusTimeout, B.wait_ns))) break;
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + ring.stage * eri_stage_bytes(S));
                    issue_pairs<S, true, BK>(tmem, st, st + ABYTES, AGROUP, BPLANE, idesc, first, ACHUNK);
                    mma_commit_pair_mc(&empty[ring.stage], (uint16_t)0x3);
                    ring.next(STAGES);
                }
                if (ok) mma_commit_pair_mc(&acc_full, (uint16_t)0x3);
            }
        }
        mma_commit_pair_mc(&done, (uint16_t)0x3);
        failed = !ok;
    } else if (warp >= 2) {
        // ---------------- epilogue: exact int64 recombination, then re-slicing into the V planes.
        // Warp: TMEM lane quadrant q (this CTA's tile rows 32q..32q+31) and kEriRuns runs of 8
        // columns.  Several warps per quadrant keep enough independent work in flight to re-slice
        // a tile while the MMAs of the next one run.
        const int q = warp & 3, h = (warp - 2) >> 2;
        const uint32_t acc_empty_leader = mapa_rank(smem_u32(&acc_empty), 0);
        long long run[kEriRuns][8];
        int it = 0;
        bool ok = true;
        // With vp >= 48 the warp's 48 columns touch at most two b and two exponent groups, so
        // the exponent tables of a tile come down to ten loads per thread, issued before the
        // accumulators are waited for so that their latency hides behind the MMAs.
        for (int e = cluster; e < B.nentries && ok; e += nclusters) {
            const int4 en = B.entries[e];
            const EriItem& p = B.item[en.z];
            const int Ncols = p.nb * p.vp;
            const bool few_tables = p.vp >= 8 * kEriRuns;
            const int nkb = (p.nchol + BK - 1) / BK;
            const int kb_per_chunk = *p.kbc;
            const int nch = (nkb + kb_per_chunk - 1) / kb_per_chunk;
            const int qt = en.y;
            // this thread's tile row: chunk (first L^T row, rows) and the row (x, y) in it
            const int r_tile = kEmuTile * (int)rank + 32 * q + lane;
            const int2 chk = p.chunks[(size_t)en.x * kEriTileChunks + r_tile / kEriChunkRows];
            const int row = chk.x + r_tile % kEriChunkRows;
            const int x = row / p.vp, y = row - x * p.vp;
            const bool row_ok = r_tile % kEriChunkRows < chk.y;
            const bool direct = row_ok && x >= p.a0 && x < p.a0 + p.na;             // V_xb, column y
            const bool mirror = row_ok && y > x && y >= p.a0 && y < p.a0 + p.na;    // V_yb, column x
            const int col0 = qt * kEmuTileN + 8 * kEriRuns * h;            // first column of the warp
            const int colz = min(col0 + 8 * (kEriRuns - 1), Ncols - 1);   // last valid run start
            const int bq0 = col0 / p.vp, gq0 = (p.b0 * p.vp + col0) / kG;
            int e_row = 0, rs_d = 0, rs_m = 0, fd0 = 0, fd1 = 0, fm0 = 0, fm1 = 0, x0 = 0, x1 = 0;
            if (row_ok) {
                e_row = p.lt_exp[row / kG];
                if (direct) rs_d = p.row_start[x - p.a0];
                if (mirror) rs_m = p.row_start[y - p.a0];
                if (few_tables && col0 < Ncols) {
                    if (direct) {
                        fd0 = p.f_tab[x * p.nv + p.b0 + bq0];
                        fd1 = p.f_tab[x * p.nv + p.b0 + colz / p.vp];
                    }
                    if (mirror) {
                        fm0 = p.f_tab[y * p.nv + p.b0 + bq0];
                        fm1 = p.f_tab[y * p.nv + p.b0 + colz / p.vp];
                    }
                    x0 = p.lt_exp[gq0];
                    x1 = p.lt_exp[(p.b0 * p.vp + colz) / kG];
                }
            }
#pragma unroll
            for (int g = 0; g < kEriRuns; ++g)
#pragma unroll
                for (int k = 0; k < 8; ++k) run[g][k] = 0;
            for (int ch = 0; ch < nch; ++ch, ++it) {
                if (!(ok = mbar_wait(&acc_full, (uint32_t)(it & 1), B.status, kStatusTimeout, B.wait_ns))) break;
                tc_fence_after();
#pragma unroll
                for (int g = 0; g < kEriRuns; ++g) {   // accumulators 0-1, then 2-4: fewer live registers
                    const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + 8 * (kEriRuns * h + g);
                    uint32_t v[3][8];
                    tmem_ld8(base, v[0]);
                    tmem_ld8(base + kAccStride, v[1]);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 8; ++k) run[g][k] += acc_head<7>(v[0][k], v[1][k]);
#pragma unroll
                    for (int j = 0; j < 3; ++j) tmem_ld8(base + (2 + j) * kAccStride, v[j]);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 8; ++k) run[g][k] += acc_tail<7>(acc_int(v[0][k], 4), v[1][k], v[2][k]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(acc_empty_leader);
            }
            if (!ok) break;
            // With vp % 16 == 0 each run of 8 columns lies in one b and starts at d % 8 == 0, and the
            // runs 2k, 2k+1 (same b) fill one 32-byte sector, which goes out as one store per plane
            // (pad columns come out zero): half-written sectors would come back from DRAM.
            // Run pairs outermost, so that a pair's registers die once both targets have it.
#pragma unroll
            for (int gp = 0; gp < kEriRuns / 2; ++gp)
            for (int tg = 0; tg < 2; ++tg) {   // target 0: V_xb at column y; 1: V_yb at column x
            if (!(tg == 0 ? direct : mirror)) continue;
            const int a = tg == 0 ? x : y, c = tg == 0 ? y : x;
            const int rs = tg == 0 ? rs_d : rs_m, f0 = tg == 0 ? fd0 : fm0, f1 = tg == 0 ? fd1 : fm1;
            uint4 prev[S];
#pragma unroll
            for (int g = 2 * gp; g < 2 * gp + 2; ++g) {
                const int col = col0 + 8 * g;
                const int bq = col / p.vp, b = p.b0 + bq, d = col - bq * p.vp;
                if (col >= Ncols || a > b) continue;
                int f_ab, e_bd;
                if (few_tables) {
                    f_ab = bq == bq0 ? f0 : f1;
                    e_bd = (p.b0 * p.vp + col) / kG == gq0 ? x0 : x1;
                } else {
                    f_ab = p.f_tab[a * p.nv + b];
                    e_bd = p.lt_exp[(p.b0 * p.vp + col) / kG];
                }
                const int sh = f_ab - e_row - e_bd + 49 - 7 * S;
                const size_t off = (size_t)(rs + (b - max(a, p.b0))) * p.kpad + (size_t)c * p.vp + d;
                if (p.vint != nullptr) {   // 64 bytes: two whole sectors
                    __align__(16) long long N[8];
                    // this target's exact sum: the product, plus (Cholesky batches) the sums the
                    // earlier batches left in this V element (the other target has its own)
                    long long I[8];
#pragma unroll
                    for (int k2 = 0; k2 < 8; ++k2) I[k2] = run[g][k2];
                    if ((p.acc_mode == 1 || p.acc_mode == 2) && off + 8 <= p.plane_stride) {
                        const longlong2* src = reinterpret_cast<const longlong2*>(p.vint + off);
#pragma unroll
                        for (int k2 = 0; k2 < 4; ++k2) {
                            const longlong2 v2 = __ldcs(src + k2);
                            I[2 * k2] += v2.x;
                            I[2 * k2 + 1] += v2.y;
                        }
                    }
                    if (p.acc_mode >= 2) {
                        round_run<S>(I, sh, N, B.status);
                    } else {
#pragma unroll
                        for (int k2 = 0; k2 < 8; ++k2) N[k2] = I[k2];
                    }
                    const uint4* w4 = reinterpret_cast<const uint4*>(N);
                    if (LADDER_IN_BOUNDS(off + 8 <= p.plane_stride, B.status)) {
                        st_cs_32B(p.vint + off, w4[0], w4[1]);
                        st_cs_32B(p.vint + off + 4, w4[2], w4[3]);
                    }
                    continue;
                }
                __align__(16) __nv_bfloat162 out[S][4];
                slice_run<S>(run[g], sh, out, B.status);
                // streaming stores: V is read back only by the ladder
                if ((g & 1) == 0) {  // runs 2k, 2k+1: same b, both valid or both skipped
#pragma unroll
                    for (int s2 = 0; s2 < S; ++s2) prev[s2] = *reinterpret_cast<const uint4*>(out[s2]);
                } else {
#pragma unroll
                    for (int s2 = 0; s2 < S; ++s2)
                        if (LADDER_IN_BOUNDS(off >= 8 && off + 8 <= p.plane_stride, B.status))
                            st_cs_32B(p.vplanes + s2 * p.plane_stride + off - 8, prev[s2],
                                      *reinterpret_cast<const uint4*>(out[s2]));
                }
            }
            }
        }
        failed = !ok;
    }
    // Every CTA waits for the leader's last commit (all MMAs that read its shared memory are done).
    if (threadIdx.x == 64) mbar_wait(&done, 0, B.status, kStatusTimeout, B.wait_ns);
    if (failed) grace_delay(2000000);  // an aborted pipeline: let copies already in flight land
    tc_fence_before();
    cluster_sync();  // no CTA leaves while its peer may still write into it or signal it
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, kTmemCols);
    }
}

// ------------------------------------------------------------------ self-product entries
// In the Gram matrix V = L^T L^T^T two rows meet themselves where (a,c) and (b,d) name the
// same values of the symmetric L: (c,d) = (b,a) in every pair row (a,b), V_ab,ba = ||L_ab||^2,
// and (c,c) in the a = b rows, V_aa,cc = ||L_ac||^2.  There the slice products that the level
// cut drops include the squares d_s d_s, which are never negative, so the cut biases exactly
// these entries low, and E_L sums that bias coherently over all (i,j,a,b).  After the ERI of a
// block this kernel rewrites them from the FP64 squared norms: one thread per pair row for
// (b,a) (a < b), and one per (a, c) for the diagonal rows of the block.
struct SelfArgs {
    int nv, vp, kpad, a0, a1, b0, b1, npairs;
    size_t plane_stride;
    const int2* pairs;      // pair (a, b) of each V row of the block
    const int* row_start;   // first V row of each a of the block
    const int* f_tab;
    const double* lsq;      // ||L[:, a, c]||^2 [nv][nv]
    __nv_bfloat16* vplanes;
    long long* vint;        // non-null: V held as int64 N
    unsigned* status;
};

template <int S>
__global__ void __launch_bounds__(256) eri_self_kernel(SelfArgs p) {
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int a, b, c, d;
    long long row;
    if (u < p.npairs) {
        const int2 ab = p.pairs[u];
        a = ab.x;
        b = ab.y;
        if (a == b) return;  // the diagonal rows are handled below, (b,a) = (a,a) included
        c = b;
        d = a;
        row = u;
    } else {
        const int lo = max(p.a0, p.b0), hi = min(p.a1, p.b1);
        const long long v = u - p.npairs;
        if (hi <= lo || v >= (long long)(hi - lo) * p.nv) return;
        a = lo + (int)(v / p.nv);
        b = a;
        c = (int)(v % p.nv);
        d = c;
        row = p.row_start[a - p.a0];  // the first row of a is (a, max(a, b0)) = (a, a)
    }
    long long N = scaled_rint(p.lsq[(size_t)a * p.nv + c], 7 * S - p.f_tab[a * p.nv + b]);
    const long long lim = 1LL << (7 * S - 1);
    if (N > lim) {  // cannot happen under the Cauchy-Schwarz exponent bound
        atomicOr(p.status, kStatusNumeric);
        N = lim;
    }
    const size_t off = (size_t)row * p.kpad + (size_t)c * p.vp + d;
    if (!LADDER_IN_BOUNDS(off < p.plane_stride, p.status)) return;
    if (p.vint != nullptr) {
        p.vint[off] = N;
        return;
    }
    __nv_bfloat16 dg[S];
    digits_of<S>(N, dg);
#pragma unroll
    for (int s = 0; s < S; ++s) p.vplanes[s * p.plane_stride + off] = dg[s];
}

// ------------------------------------------------------------------ ladder kernel
// Work of one ladder launch: up to kMaxItems items (an instance's block pair each), each with
// its T and V tensor maps and its int64 accumulator; their work units are numbered one after
// the other, so one persistent launch covers several instances.
struct LadItem {
    int M, N, n_mt, n_nt, n_ch, kb_per_chunk, nkb;
    int swap;                // 0: rows m = pairs, columns n = (i,j); 1: rows m = (i,j), columns n = pairs
    int no2;
    int gm;                  // row tiles per group of the tile order (see tile_coords)
    long long ubeg, units;   // first unit of this item in the launch, and its unit count
    long long tbeg, ntiles;  // first tile of this item in the launch, and its tile count
    unsigned long long* rp;  // int64 fixed-point accumulator [npairs][no2]
};

struct LadBatch {
    CUtensorMap ta[kMaxItems];  // A: T slices of the item's instance
    CUtensorMap tb[kMaxItems];  // B: V planes of the item
    LadItem item[kMaxItems];
    long long units;            // all items' units
    long long tiles;            // all items' tiles
    int nitems, BN;
    unsigned* status;
    unsigned long long wait_ns; // limit of every bounded mbarrier wait (ns of the global timer)
};

// Item of a unit, for units visited in increasing order.
struct ItemCursor {
    int k = 0;
    __device__ __forceinline__ int seek(const LadBatch& B, long long u) {
        while (k + 1 < B.nitems && u >= B.item[k + 1].ubeg) ++k;
        return k;
    }
};

// (row tile, column tile) of tile `tile` of an item.  Tiles run in groups of gm row tiles: within
// a group, down the gm row tiles of a column tile, then to the next column tile, so that the tiles
// one wave of workers takes at the same time share gm row tiles' A chunks and P / gm column tiles'
// B chunks in L2.
__device__ __forceinline__ void tile_coords(const LadItem& p, long long tile, int& mt, int& nt) {
    if (p.gm <= 1) {
        nt = (int)(tile % p.n_nt);
        mt = (int)(tile / p.n_nt);
        return;
    }
    const long long per = (long long)p.gm * p.n_nt;
    const long long g = tile / per;
    const int first = (int)(g * p.gm);
    const int rows = min(p.gm, p.n_mt - first);
    const long long local = tile - g * per;
    mt = first + (int)(local % rows);
    nt = (int)(local / rows);
}

// The units one worker (a CTA, or a CTA pair) of P runs, in increasing order: first whole tiles,
// tile w, w + P, w + 2P, ... up to the last full wave of P tiles, every K chunk of a tile in turn,
// so that the P workers of a wave move through K together and share each chunk of their operands
// in L2; then an even share of the units of the tiles left over (stream-K), which keeps the load
// balanced.  `last` marks the last unit of the worker's stream-K share (its sums are flushed).
struct UnitSeq {
    long long t = 0, full = 0, P = 1, tail_u = 0, tail_end = 0;
    int k = 0, ch = 0;
    bool in_tail = false;
    __device__ __forceinline__ void init(const LadBatch& B, long long w, long long workers) {
        P = workers;
        full = B.tiles / P * P;
        t = w;
        in_tail = t >= full;
        long long tu0 = B.units;   // first unit of tile `full`
        for (int i = 0; i < B.nitems; ++i)
            if (full < B.item[i].tbeg + B.item[i].ntiles) {
                tu0 = B.item[i].ubeg + (full - B.item[i].tbeg) * B.item[i].n_ch;
                break;
            }
        const long long n = B.units - tu0;
        tail_u = tu0 + n * w / P;
        tail_end = tu0 + n * (w + 1) / P;
    }
    __device__ __forceinline__ bool next(const LadBatch& B, long long& u, bool& last) {
        if (!in_tail) {
            while (t >= B.item[k].tbeg + B.item[k].ntiles) ++k;
            const LadItem& it = B.item[k];
            u = it.ubeg + (t - it.tbeg) * it.n_ch + ch;
            last = false;
            if (++ch == it.n_ch) {
                ch = 0;
                t += P;
                in_tail = t >= full;
            }
            return true;
        }
        if (tail_u >= tail_end) return false;
        u = tail_u++;
        last = tail_u == tail_end;
        return true;
    }
};

// True when unit u + 1 belongs to another (item, row tile, column tile) than unit u of item k.
__device__ __forceinline__ bool tile_ends(const LadBatch& B, int k, long long u) {
    const LadItem& it = B.item[k];
    if (u + 1 >= it.ubeg + it.units) return true;
    return (u + 1 - it.ubeg) / it.n_ch != (u - it.ubeg) / it.n_ch;
}

// Work unit = (row tile, column tile, K chunk), chunk fastest; each CTA takes a
// contiguous range of units (stream-K) and flushes its int64 sums with atomics
// whenever its (row tile, column tile) changes.
template <int S>
__global__ void __launch_bounds__(kThreadsTC, 1) ladder_emu_kernel(const __grid_constant__ LadBatch B) {
    constexpr int BK = bk_for(S), STAGES = stages_for(S);
    constexpr uint32_t APLANE = kEmuTile * BK * 2;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[STAGES], empty[STAGES], acc_full, acc_empty, done;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t BPLANE = (uint32_t)B.BN * BK * 2;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, kEpiWarps);
        mbar_init(&done, 1);
        fence_barrier_init();
        for (int i = 0; i < B.nitems; ++i) {
            tma_prefetch_desc(&B.ta[i]);
            tma_prefetch_desc(&B.tb[i]);
        }
    }
    if (warp == 1) tmem_alloc(&tmem_base, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // T slices (A) are re-read for every pair tile and stay in L2; the V planes (B) stream.
        Ring ring;
        int issued[STAGES] = {};
        const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
        bool ok = true;
        const uint32_t bytes = (uint32_t)S * (kEmuTile + B.BN) * BK * 2;
        ItemCursor cur;
        UnitSeq seq;
        seq.init(B, blockIdx.x, gridDim.x);
        long long u;
        bool last_u;
        while (ok && seq.next(B, u, last_u)) {
            const int ik = cur.seek(B, u);
            const LadItem& p = B.item[ik];
            const long long ul = u - p.ubeg;
            const int ch = (int)(ul % p.n_ch);
            const long long tile = ul / p.n_ch;
            int mt, nt;
                tile_coords(p, tile, mt, nt);
            const int kb1 = min((ch + 1) * p.kb_per_chunk, p.nkb);
            for (int kb = ch * p.kb_per_chunk; kb < kb1 && ok; ++kb) {
                if (!(ok = mbar_wait(&empty[ring.stage], ring.phase ^ 1u, B.status, kStatusTimeout, B.wait_ns))) break;
                unsigned char* st = smem + ring.stage * stage_bytes(S);
                mbar_arrive_expect_tx(&full[ring.stage], bytes);
                tma_load_3d_hint(st, &B.ta[ik], &full[ring.stage], kb * BK, mt * kEmuTile, 0, keep);
                tma_load_3d_hint(st + S * APLANE, &B.tb[ik], &full[ring.stage], kb * BK, nt * B.BN, 0, stream);
                ++issued[ring.stage];
                ring.next(STAGES);
            }
        }
        for (int i = 0; i < STAGES; ++i)
            if (issued[i]) mbar_wait(&full[i], (uint32_t)((issued[i] - 1) & 1), B.status, kStatusTimeout, B.wait_ns);
    } else if (warp == 1 && lane == 0) {
        Ring ring;
        const uint32_t idesc = idesc_bf16_f32(kEmuTile, B.BN);
        bool ok = true;
        int it = 0;
        ItemCursor cur;
        UnitSeq seq;
        seq.init(B, blockIdx.x, gridDim.x);
        long long u;
        bool last_u;
        for (; ok && seq.next(B, u, last_u); ++it) {
            const LadItem& p = B.item[cur.seek(B, u)];
            const int ch = (int)((u - p.ubeg) % p.n_ch);
            if (!(ok = mbar_wait(&acc_empty, (uint32_t)(it & 1) ^ 1u, B.status, kStatusTimeout, B.wait_ns))) break;
            tc_fence_after();
            bool first[kNumAcc] = {true, true, true, true, true};
            const int kb1 = min((ch + 1) * p.kb_per_chunk, p.nkb);
            for (int kb = ch * p.kb_per_chunk; kb < kb1 && ok; ++kb) {
                if (!(ok = mbar_wait(&full[ring.stage], ring.phase, B.status, kStatusTimeout, B.wait_ns))) break;
                tc_fence_after();
                const uint32_t st = smem_u32(smem + ring.stage * stage_bytes(S));
                issue_pairs<S>(tmem, st, st + S * APLANE, APLANE, BPLANE, idesc, first);
                mma_commit(&empty[ring.stage]);
                ring.next(STAGES);
            }
            if (ok) mma_commit(&acc_full);
        }
        mma_commit(&done);
        mbar_wait(&done, 0, B.status, kStatusTimeout, B.wait_ns);
    } else if (warp >= 2) {
        // Each warp: TMEM lane quadrant q, column chunks ci = h, h+2, h+4 (16 columns each).
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int nchunks = B.BN / 16;
        long long run[kLadRuns][16];
#pragma unroll
        for (int i = 0; i < kLadRuns; ++i)
#pragma unroll
            for (int k = 0; k < 16; ++k) run[i][k] = 0;
        int it = 0;
        ItemCursor cur;
        UnitSeq seq;
        seq.init(B, blockIdx.x, gridDim.x);
        long long u;
        bool last_u;
        for (; seq.next(B, u, last_u); ++it) {
            if (!mbar_wait(&acc_full, (uint32_t)(it & 1), B.status, kStatusTimeout, B.wait_ns)) break;
            tc_fence_after();
#pragma unroll
            for (int i = 0; i < kLadRuns; ++i) {
                const int ci = h + kEpiPerQuad * i;
                if (ci < nchunks) {
                    const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + 16 * ci;
                    uint32_t v[3][16];
                    tmem_ld16(base, v[0]);
                    tmem_ld16(base + kAccStride, v[1]);
                    tmem_ld16(base + 2 * kAccStride, v[2]);
                    tmem_ld_wait();
                    int i4[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        run[i][k] += acc_head<6>(v[0][k], v[1][k]);
                        i4[k] = acc_int(v[2][k], 4);
                    }
                    tmem_ld16(base + 3 * kAccStride, v[0]);
                    tmem_ld16(base + 4 * kAccStride, v[1]);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 16; ++k) run[i][k] += acc_tail<6>(i4[k], v[0][k], v[1][k]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty);
            // Flush at the end of an (item, row tile, column tile) run or of this CTA's range.
            const int ik = cur.seek(B, u);
            const LadItem& p = B.item[ik];
            const long long tile = (u - p.ubeg) / p.n_ch;
            if (last_u || tile_ends(B, ik, u)) {
                int mt, nt;
                tile_coords(p, tile, mt, nt);
                const int m = mt * kEmuTile + 32 * q + lane;
#pragma unroll
                for (int i = 0; i < kLadRuns; ++i) {
                    const int ci = h + kEpiPerQuad * i;
                    if (ci < nchunks) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            const int n = nt * B.BN + 16 * ci + k;
                            if (m < p.M && n < p.N && run[i][k] != 0) {
                                const size_t idx = p.swap ? (size_t)n * p.no2 + m : (size_t)m * p.no2 + n;
                                if (LADDER_IN_BOUNDS(idx < (size_t)(p.swap ? p.N : p.M) * p.no2, B.status))
                                    atomicAdd(p.rp + idx, (unsigned long long)run[i][k]);
                            }
                            run[i][k] = 0;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Ladder on CTA pairs, for o^2 > 128: rows = (i,j) in 256-row tiles (128 per CTA), columns =
// 96 pairs (48 per CTA), 2-SM MMAs; V streams from HBM ceil(o^2 / 256) times.  Work units are
// (row tile, column tile, K chunk) with the chunk fastest; cluster c takes a contiguous range of
// units and each CTA flushes its int64 sums with atomics whenever the tile changes.
template <int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreadsTC, 1)
    ladder_pair_kernel(const __grid_constant__ LadBatch B) {
    constexpr int BK = bk_for(S), STAGES = pair_stages_for(S);
    constexpr uint32_t APLANE = kEmuTile * BK * 2, BPLANE = (kEmuTileN / 2) * BK * 2;
    constexpr uint32_t ABYTES = S * APLANE;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[STAGES], empty[STAGES], acc_full, acc_empty, done;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const long long cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 2 * kEpiWarps);
        mbar_init(&done, 1);
        fence_barrier_init();
        for (int i = 0; i < B.nitems; ++i) {
            tma_prefetch_desc(&B.ta[i]);
            tma_prefetch_desc(&B.tb[i]);
        }
    }
    if (warp == 1) tmem_alloc_pair(&tmem_base, kTmemCols);
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    bool failed = false;

    if (warp == 0 && lane == 0) {
        // T slices (A) are re-read for every pair tile and stay in L2; the V planes (B) stream.
        Ring ring;
        bool ok = true;
        const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
        ItemCursor cur;
        UnitSeq seq;
        seq.init(B, cluster, nclusters);
        long long u;
        bool last_u;
        while (ok && seq.next(B, u, last_u)) {
            const int ik = cur.seek(B, u);
            const LadItem& p = B.item[ik];
            const long long ul = u - p.ubeg;
            const int ch = (int)(ul % p.n_ch);
            const long long tile = ul / p.n_ch;
            int mt, nt;
                tile_coords(p, tile, mt, nt);
            const int arow = mt * 2 * kEmuTile + kEmuTile * (int)rank;
            const int brow = nt * kEmuTileN + (kEmuTileN / 2) * (int)rank;
            const int kb1 = min((ch + 1) * p.kb_per_chunk, p.nkb);
            for (int kb = ch * p.kb_per_chunk; kb < kb1 && ok; ++kb) {
                if (!(ok = mbar_wait(&empty[ring.stage], ring.phase ^ 1u, B.status, kStatusTimeout, B.wait_ns))) break;
                unsigned char* st = smem + ring.stage * pair_stage_bytes(S);
                if (rank == 0) mbar_arrive_expect_tx(&full[ring.stage], 2 * pair_stage_bytes(S));
                const uint32_t fb = mapa_rank(smem_u32(&full[ring.stage]), 0);
                tma_load_3d_2sm_hint(st, &B.ta[ik], fb, kb * BK, arow, 0, keep);
                tma_load_3d_2sm_hint(st + ABYTES, &B.tb[ik], fb, kb * BK, brow, 0, stream);
                ring.next(STAGES);
            }
        }
        failed = !ok;
    } else if (warp == 1 && lane == 0 && rank == 0) {
        Ring ring;
        const uint32_t idesc = idesc_bf16_f32(2 * kEmuTile, kEmuTileN);
        bool ok = true;
        int it = 0;
        ItemCursor cur;
        UnitSeq seq;
        seq.init(B, cluster, nclusters);
        long long u;
        bool last_u;
        for (; ok && seq.next(B, u, last_u); ++it) {
            const LadItem& p = B.item[cur.seek(B, u)];
            const int ch = (int)((u - p.ubeg) % p.n_ch);
            if (!(ok = mbar_wait(&acc_empty, (uint32_t)(it & 1) ^ 1u, B.status, kStatusTimeout, B.wait_ns))) break;
            tc_fence_after();
            bool first[kNumAcc] = {true, true, true, true, true};
            const int kb1 = min((ch + 1) * p.kb_per_chunk, p.nkb);
            for (int kb = ch * p.kb_per_chunk; kb < kb1 && ok; ++kb) {
                if (!(ok = mbar_wait(&full[ring.stage], ring.phase, B.status, kStatusTimeout, B.wait_ns))) break;
                tc_fence_after();
                const uint32_t st = smem_u32(smem + ring.stage * pair_stage_bytes(S));
                issue_pairs<S, true>(tmem, st, st + ABYTES, APLANE, BPLANE, idesc, first);
                mma_commit_pair_mc(&empty[ring.stage], (uint16_t)0x3);
                ring.next(STAGES);
            }
            if (ok) mma_commit_pair_mc(&acc_full, (uint16_t)0x3);
        }
        mma_commit_pair_mc(&done, (uint16_t)0x3);
        failed = !ok;
    } else if (warp >= 2) {
        const int q = warp & 3, h = (warp - 2) >> 2;
        const uint32_t acc_empty_leader = mapa_rank(smem_u32(&acc_empty), 0);
        long long run[kLadRuns][16];
#pragma unroll
        for (int i = 0; i < kLadRuns; ++i)
#pragma unroll
            for (int k = 0; k < 16; ++k) run[i][k] = 0;
        int it = 0;
        bool ok = true;
        ItemCursor cur;
        UnitSeq seq;
        seq.init(B, cluster, nclusters);
        long long u;
        bool last_u;
        for (; seq.next(B, u, last_u); ++it) {
            if (!(ok = mbar_wait(&acc_full, (uint32_t)(it & 1), B.status, kStatusTimeout, B.wait_ns))) break;
            tc_fence_after();
#pragma unroll
            for (int cc = 0; cc < kLadRuns; ++cc) {
                const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + 16 * (h + kEpiPerQuad * cc);
                uint32_t v[3][16];
                tmem_ld16(base, v[0]);
                tmem_ld16(base + kAccStride, v[1]);
                tmem_ld16(base + 2 * kAccStride, v[2]);
                tmem_ld_wait();
                int i4[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    run[cc][k] += acc_head<6>(v[0][k], v[1][k]);
                    i4[k] = acc_int(v[2][k], 4);
                }
                tmem_ld16(base + 3 * kAccStride, v[0]);
                tmem_ld16(base + 4 * kAccStride, v[1]);
                tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < 16; ++k) run[cc][k] += acc_tail<6>(i4[k], v[0][k], v[1][k]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(acc_empty_leader);
            const int ik = cur.seek(B, u);
            const LadItem& p = B.item[ik];
            const long long tile = (u - p.ubeg) / p.n_ch;
            if (last_u || tile_ends(B, ik, u)) {
                int mt, nt;
                tile_coords(p, tile, mt, nt);
                const int m = mt * 2 * kEmuTile + kEmuTile * (int)rank + 32 * q + lane;  // (i,j)
#pragma unroll
                for (int cc = 0; cc < kLadRuns; ++cc)
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int n = nt * kEmuTileN + 16 * (h + kEpiPerQuad * cc) + k;       // pair
                        if (m < p.M && n < p.N && run[cc][k] != 0 &&
                            LADDER_IN_BOUNDS((size_t)n * p.no2 + m < (size_t)p.N * p.no2, B.status))
                            atomicAdd(p.rp + (size_t)n * p.no2 + m, (unsigned long long)run[cc][k]);
                        run[cc][k] = 0;
                    }
            }
        }
        failed = !ok;
    }
    if (threadIdx.x == 64) mbar_wait(&done, 0, B.status, kStatusTimeout, B.wait_ns);
    if (failed) grace_delay(2000000);
    tc_fence_before();
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, kTmemCols);
    }
}

// R[i,j,a,b] += 2^(f_ab + g_ij - 42) J[(a,b), (i,j)] and the mirror R[j,i,b,a] for a < b.
__global__ void finalize_kernel(const unsigned long long* __restrict__ rp, int npairs, int no, int nv,
                                const int2* __restrict__ pairs, const int* __restrict__ f_tab,
                                const int* __restrict__ t_exp, double* __restrict__ R, unsigned* status) {
    const int no2 = no * no;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)npairs * no2) return;
    const int m = (int)(k / no2), n = (int)(k % no2);
    const int2 ab = pairs[m];
    const long long J = (long long)rp[k];
    const double v = ldexp((double)J, f_tab[ab.x * nv + ab.y] + t_exp[n / kG] - 42);
    const int i = n / no, j = n % no;
    const size_t x = (((size_t)i * no + j) * nv + ab.x) * nv + ab.y, y = (((size_t)j * no + i) * nv + ab.y) * nv + ab.x;
    if (LADDER_IN_BOUNDS(x < (size_t)no2 * nv * nv, status)) R[x] += v;
    if (ab.x < ab.y && LADDER_IN_BOUNDS(y < (size_t)no2 * nv * nv, status)) R[y] += v;
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// 3-D BF16 map over planes[z][y][x]: x = K (extent `inner`, row stride `row_bytes`),
// y = rows, z = planes (stride `plane_bytes`).  Box {bk, box_rows, planes}; OOB reads give 0.
bool make_tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t planes, uint64_t row_bytes,
               uint64_t plane_bytes, uint32_t bk, uint32_t box_rows, uint32_t box_planes = 0) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {inner, rows, planes};
    cuuint64_t strides[2] = {row_bytes, plane_bytes};
    cuuint32_t box[3] = {bk, box_rows, box_planes ? box_planes : (cuuint32_t)planes};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapSwizzle sw = bk * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : bk * 2 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                 : CU_TENSOR_MAP_SWIZZLE_32B;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}


// Padded (c, d) layout of the emulated path: vp = nv rounded up to 16 (emu_vp), K = nv * vp.
inline int padded_vp(int nv) { return emu_vp(nv); }

// Cholesky vectors sliced at a time: all of them, or the plan's batch.
inline int lt_batch(const ladder_plan_s& p) { return p.pb > 0 && p.pb < p.nchol ? p.pb : p.nchol; }

// L^T digit planes of the Cholesky vectors [pbase, pbase + count), their digit norms and the ERI's
// exact chunk for them (three kernels, memsets of the norm accumulators).
template <int S>
cudaError_t slice_lt(const ladder_plan_s& p, const double* L, void* ws, int pbase, int count, cudaStream_t s) {
    const int vp = padded_vp(p.nv);
    const long long rows = (long long)p.nv * vp;
    const int xpad = (int)align_up((size_t)lt_batch(p), 8);
    const int nblk = (xpad + kEmuChunkK - 1) / kEmuChunkK;
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, p.ws.lt_norm2), 0, (size_t)S * rows * nblk * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(at<char>(ws, p.ws.eri_cand), 0, (size_t)S * 3 * 4, s)) != cudaSuccess) return e;
    lt_slice_kernel<S><<<dim3((count + 63) / 64, (unsigned)((rows + 63) / 64)), 256, 0, s>>>(
        L, pbase, count, p.nv, vp, xpad, at<int>(ws, p.ws.lt_exp), at<__nv_bfloat16>(ws, p.ws.lt_slices),
        at<unsigned>(ws, p.ws.lt_norm2), nblk, p.d_status);
    eri_chunk_norms_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(at<unsigned>(ws, p.ws.lt_norm2), rows, S,
                                                                         nblk, at<unsigned>(ws, p.ws.eri_cand));
    eri_chunk_select_kernel<<<1, 1, 0, s>>>(at<unsigned>(ws, p.ws.eri_cand), S, p.eri_chunk_max, eri_bk_for(S),
                                            at<int>(ws, p.ws.eri_kbc));
    return cudaGetLastError();
}

template <int S>
cudaError_t prep_impl(const ladder_plan_s& p, const double* L, const double* t2, void* ws, cudaStream_t s) {
    const long long nv2 = (long long)p.nv * p.nv;
    const int vp = padded_vp(p.nv);
    const long long rows = (long long)p.nv * vp;
    const int no2 = p.no * p.no;
    const int kpad = (int)rows;
    const int ngt = (no2 + kG - 1) / kG;
    // kernels: L^T statistics, pair exponents, L^T slices, chunk norms and choice (here unless the
    // Cholesky vectors are sliced batch by batch with the blocks), then the T side (row maxima,
    // exponents, slices; the split form has two exponent passes when rows i < j exist)
    const bool batched_p = lt_batch(p) < p.nchol;
    const int t_kernels = p.form == 0 ? 3 : (p.no > 1 ? 4 : 3);
    LaunchTimer tm(p, s, LADDER_KERNEL_PREP, (batched_p ? 2 : 5) + t_kernels);
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, p.ws.lnorm), 0, (size_t)p.nv * 8, s)) != cudaSuccess) return e;
    if (p.form == 0 && (e = cudaMemsetAsync(at<char>(ws, p.ws.t_gmax), 0, (size_t)ngt * 8, s)) != cudaSuccess)
        return e;
    lt_rowstats_kernel<<<(unsigned)((rows + kG - 1) / kG), kG, 0, s>>>(L, p.nchol, p.nv, vp, at<int>(ws, p.ws.lt_exp),
                                                                        at<unsigned long long>(ws, p.ws.lnorm),
                                                                        at<double>(ws, p.ws.lsq));
    f_table_kernel<<<(unsigned)((nv2 + 255) / 256), 256, 0, s>>>(at<unsigned long long>(ws, p.ws.lnorm), p.nv,
                                                                   at<int>(ws, p.ws.v_exp));
    if (!batched_p && (e = slice_lt<S>(p, L, ws, 0, p.nchol, s)) != cudaSuccess) return e;
    if (p.form == 0) {
        t_rowmax_kernel<<<dim3((unsigned)((nv2 + 8191) / 8192), no2), 256, 0, s>>>(
            t2, nv2, no2, at<unsigned long long>(ws, p.ws.t_gmax));
        exp_from_max_kernel<<<(ngt + 255) / 256, 256, 0, s>>>(at<unsigned long long>(ws, p.ws.t_gmax), ngt,
                                                               at<int>(ws, p.ws.t_exp));
        const long long units = (long long)(kpad / 8) * no2;
        t_slice_kernel<S><<<(unsigned)((units + 255) / 256), 256, 0, s>>>(
            t2, p.nv, vp, no2, kpad, at<int>(ws, p.ws.t_exp), at<__nv_bfloat16>(ws, p.ws.t_slices), p.d_status);
        return cudaGetLastError();
    }
    // symmetric/antisymmetric form: T' (rows i <= j, c <= d) and T'' (rows i < j, c < d)
    const PmDims d = pm_dims(p.no, p.nv);
    const int ngp = (d.np + kG - 1) / kG, ngm = (d.nm + kG - 1) / kG;
    if ((e = cudaMemsetAsync(at<char>(ws, p.ws.tp_gmax), 0, (size_t)ngp * 8, s)) != cudaSuccess) return e;
    if (ngm > 0 && (e = cudaMemsetAsync(at<char>(ws, p.ws.tm_gmax), 0, (size_t)ngm * 8, s)) != cudaSuccess) return e;
    tpm_rowmax_kernel<<<(unsigned)(d.np + d.nm), 256, 0, s>>>(t2, p.no, p.nv, d.np,
                                                                at<unsigned long long>(ws, p.ws.tp_gmax),
                                                                at<unsigned long long>(ws, p.ws.tm_gmax));
    exp_from_max_kernel<<<(ngp + 255) / 256, 256, 0, s>>>(at<unsigned long long>(ws, p.ws.tp_gmax), ngp,
                                                           at<int>(ws, p.ws.tp_exp));
    if (ngm > 0)
        exp_from_max_kernel<<<(ngm + 255) / 256, 256, 0, s>>>(at<unsigned long long>(ws, p.ws.tm_gmax), ngm,
                                                               at<int>(ws, p.ws.tm_exp));
    tpm_slice_kernel<S><<<(unsigned)(d.np + d.nm), 128, 0, s>>>(
        t2, p.no, p.nv, d.np, d.kp_pad, d.km_pad, d.nm, at<int>(ws, p.ws.tp_exp), at<int>(ws, p.ws.tm_exp),
        at<__nv_bfloat16>(ws, p.ws.tp_slices), at<__nv_bfloat16>(ws, p.ws.tm_slices), p.d_status);
    return cudaGetLastError();
}

// The ERI work item of one block pair of a plan whose workspace starts at ws: its tables and
// its two L^T tensor maps.
// count: Cholesky vectors in the L^T planes (the batch); acc_mode as in EriItem.
template <int S>
bool eri_item(const ladder_plan_s& p, const BlockPair& bp, void* ws, EriItem* it, CUtensorMap* ta, CUtensorMap* tb,
              int count = 0, int acc_mode = 3) {
    constexpr int EBK = eri_bk_for(S);
    const int vp = padded_vp(p.nv);
    if (vp % 16 != 0) return false;   // the epilogue stores whole 32-byte sectors
    if (count <= 0) count = p.nchol;
    const long long rows = (long long)p.nv * vp;
    const int xpad = (int)align_up((size_t)lt_batch(p), 8);
    if (!make_tmap(ta, at<char>(ws, p.ws.lt_slices), count, rows, S, (uint64_t)xpad * 2, (uint64_t)rows * xpad * 2,
                   EBK, kEriChunkRows) ||
        !make_tmap(tb, at<char>(ws, p.ws.lt_slices), count, rows, S, (uint64_t)xpad * 2, (uint64_t)rows * xpad * 2,
                   EBK, kEmuTileN / 2))
        return false;
    const int* row_start = reinterpret_cast<const int*>(p.d_tables) + bp.rows_off;
    const int2* chunks = reinterpret_cast<const int2*>(p.d_tables) + bp.chunks_off;
    *it = EriItem{p.nv, vp, count, bp.a0, bp.a1 - bp.a0, bp.b0, bp.b1 - bp.b0, (int)rows,
                  (size_t)p.max_pairs * (size_t)rows, chunks, row_start, at<int>(ws, p.ws.lt_exp), at<int>(ws, p.ws.v_exp),
                  at<__nv_bfloat16>(ws, p.ws.v_blk), p.form == 1 ? at<long long>(ws, p.ws.v_blk) : nullptr,
                  at<int>(ws, p.ws.eri_kbc), acc_mode};
    return true;
}

// One persistent ERI launch over every tile of the batch: no more CTA pairs than fit at once
// (a cluster that waited for a free slot would process its share of the tiles after all the
// others).
template <int S>
void launch_eri_batch(const EriBatch& eb, int max_clusters, cudaStream_t s) {
    const int clusters = std::max(1, std::min(eb.nentries, max_clusters));
    eri_emu_kernel<S><<<2 * clusters, kThreadsEri, eri_smem_bytes_for(S), s>>>(eb);
}

// The self-product entries of one block pair, after its ERI.
template <int S>
void launch_self(const ladder_plan_s& p, const BlockPair& bp, void* ws, cudaStream_t s) {
    const int vp = padded_vp(p.nv);
    const int kpad = p.nv * vp;
    const int2* table = reinterpret_cast<const int2*>(p.d_tables);
    const int* row_start = reinterpret_cast<const int*>(p.d_tables) + bp.rows_off;
    const int ndiag = std::max(0, std::min(bp.a1, bp.b1) - std::max(bp.a0, bp.b0));
    const long long nself = (long long)bp.npairs + (long long)ndiag * p.nv;
    SelfArgs sa{p.nv, vp, kpad, bp.a0, bp.a1, bp.b0, bp.b1, bp.npairs, (size_t)p.max_pairs * kpad,
                table + bp.pairs_off, row_start, at<int>(ws, p.ws.v_exp), at<double>(ws, p.ws.lsq),
                at<__nv_bfloat16>(ws, p.ws.v_blk), p.form == 1 ? at<long long>(ws, p.ws.v_blk) : nullptr,
                p.d_status};
    eri_self_kernel<S><<<(unsigned)((nself + 255) / 256), 256, 0, s>>>(sa);
}

// The ladder runs on CTA pairs (256-row (i,j) tiles) when o^2 > 128.
inline bool ladder_on_pairs(const ladder_plan_s& p) { return p.no * p.no > kEmuTile; }

// The ladder work item of one block pair of a plan whose workspace starts at ws; its units are
// numbered from ubeg in the launch.
// Column tile (pairs) of the ladder: 96 on CTA pairs (48 per CTA), the plan's width on one SM.
inline int ladder_bn(const ladder_plan_s& p, bool pair) { return pair ? kEmuTileN : p.lad_bn; }

template <int S>
bool ladder_item(const ladder_plan_s& p, const BlockPair& bp, void* ws, long long ubeg, LadItem* it, CUtensorMap* ta,
                 CUtensorMap* tb, long long tbeg = 0) {
    constexpr int BK = bk_for(S);
    const bool pair = ladder_on_pairs(p);
    const int bn = ladder_bn(p, pair);
    const int vp = padded_vp(p.nv);
    const int kpad = p.nv * vp, no2 = p.no * p.no;
    const size_t vplane = (size_t)p.max_pairs * kpad;
    if (!make_tmap(ta, at<char>(ws, p.ws.t_slices), kpad, no2, S, (uint64_t)kpad * 2, (uint64_t)no2 * kpad * 2, BK,
                   kEmuTile) ||
        !make_tmap(tb, at<char>(ws, p.ws.v_blk), kpad, bp.npairs, S, (uint64_t)kpad * 2, (uint64_t)vplane * 2, BK,
                   pair ? kEmuTileN / 2 : bn))
        return false;
    LadItem x{};
    x.swap = 1;
    x.no2 = no2;
    x.M = no2;
    x.N = bp.npairs;
    x.n_mt = (x.M + (pair ? 2 : 1) * kEmuTile - 1) / ((pair ? 2 : 1) * kEmuTile);
    x.n_nt = (x.N + bn - 1) / bn;
    x.nkb = (kpad + BK - 1) / BK;
    x.kb_per_chunk = kEmuChunkK / BK;
    x.n_ch = (x.nkb + x.kb_per_chunk - 1) / x.kb_per_chunk;
    x.units = (long long)x.n_mt * x.n_nt * x.n_ch;
    x.ubeg = ubeg;
    x.ntiles = (long long)x.n_mt * x.n_nt;
    x.tbeg = tbeg;
    x.gm = x.n_mt < 4 ? x.n_mt : 4;   // waves of P tiles: 4 row tiles x P/4 column tiles
    x.rp = at<unsigned long long>(ws, p.ws.rp_int);
    *it = x;
    return true;
}

// One persistent ladder launch over every unit of the batch (all items on CTA pairs, or all on
// single CTAs).
template <int S>
void launch_ladder_batch(const LadBatch& lb, bool on_pairs, int max_pair_clusters, int num_sms, cudaStream_t s) {
    if (on_pairs) {
        const long long clusters = std::max<long long>(1, std::min<long long>(lb.units, max_pair_clusters));
        ladder_pair_kernel<S><<<(unsigned)(2 * clusters), kThreadsTC, pair_smem_bytes_for(S), s>>>(lb);
    } else {
        ladder_emu_kernel<S><<<(unsigned)std::max<long long>(1, std::min<long long>(lb.units, num_sms)), kThreadsTC,
                               smem_bytes_for(S), s>>>(lb);
    }
}

// Ladder work item X (plus) or Y (minus) of the symmetric/antisymmetric form of one block pair.
template <int S>
bool ladder_item_pm(const ladder_plan_s& p, const BlockPair& bp, void* ws, long long ubeg, bool plus, LadItem* it,
                    CUtensorMap* ta, CUtensorMap* tb, long long tbeg = 0) {
    constexpr int BK = bk_for(S);
    const PmDims d = pm_dims(p.no, p.nv);
    const int rows = plus ? d.np : d.nm;
    const long long K = plus ? d.kp : d.km, kpad = plus ? d.kp_pad : d.km_pad;
    const bool pair = rows > kEmuTile;
    const int bn = ladder_bn(p, pair);
    if (!make_tmap(ta, at<char>(ws, plus ? p.ws.tp_slices : p.ws.tm_slices), K, rows, S, (uint64_t)kpad * 2,
                   (uint64_t)rows * kpad * 2, BK, kEmuTile) ||
        !make_tmap(tb, at<char>(ws, plus ? p.ws.vp_blk : p.ws.vm_blk), K, bp.npairs, S, (uint64_t)kpad * 2,
                   (uint64_t)p.max_pairs * kpad * 2, BK, pair ? kEmuTileN / 2 : bn))
        return false;
    LadItem x{};
    x.swap = 1;
    x.no2 = rows;
    x.M = rows;
    x.N = bp.npairs;
    x.n_mt = (rows + (pair ? 2 : 1) * kEmuTile - 1) / ((pair ? 2 : 1) * kEmuTile);
    x.n_nt = (x.N + bn - 1) / bn;
    x.nkb = (int)((K + BK - 1) / BK);
    x.kb_per_chunk = kEmuChunkK / BK;
    x.n_ch = (x.nkb + x.kb_per_chunk - 1) / x.kb_per_chunk;
    x.units = (long long)x.n_mt * x.n_nt * x.n_ch;
    x.ubeg = ubeg;
    x.ntiles = (long long)x.n_mt * x.n_nt;
    x.tbeg = tbeg;
    x.gm = x.n_mt < 4 ? x.n_mt : 4;   // waves of P tiles: 4 row tiles x P/4 column tiles
    x.rp = at<unsigned long long>(ws, plus ? p.ws.rpx : p.ws.rpy);
    *it = x;
    return true;
}

// Split form, shared by single plans and groups: zero the X and Y accumulators of a block pair.
// Y's accumulator starts at zero whenever there are rows i < j, also when K'' is empty (nv = 1):
// the finalisation reads it for those rows.
cudaError_t clear_pm_acc(const ladder_plan_s& p, const BlockPair& bp, void* ws, cudaStream_t s) {
    const PmDims d = pm_dims(p.no, p.nv);
    cudaError_t e = cudaMemsetAsync(at<char>(ws, p.ws.rpx), 0, (size_t)bp.npairs * d.np * 8, s);
    if (e == cudaSuccess && d.nm > 0) e = cudaMemsetAsync(at<char>(ws, p.ws.rpy), 0, (size_t)bp.npairs * d.nm * 8, s);
    return e;
}

// Split form: V' and V'' of a block pair from its int64 V.
template <int S>
void launch_combine(const ladder_plan_s& p, const BlockPair& bp, void* ws, cudaStream_t s) {
    const PmDims d = pm_dims(p.no, p.nv);
    const int vp = padded_vp(p.nv);
    CombineArgs ca{p.nv, vp, bp.npairs, (p.nv + 31) / 32, (size_t)p.max_pairs * d.kp_pad,
                   (size_t)p.max_pairs * d.km_pad, (long long)p.nv * vp, d.kp_pad, d.km_pad,
                   at<long long>(ws, p.ws.v_blk), at<__nv_bfloat16>(ws, p.ws.vp_blk),
                   at<__nv_bfloat16>(ws, p.ws.vm_blk), p.d_status};
    const long long units = (long long)bp.npairs * ca.ntile * (ca.ntile + 1) / 2;
    vpm_combine_kernel<S><<<(unsigned)units, kCombineThreads, 0, s>>>(ca);
}

// Split form: the X item (and the Y item, when there are rows i < j and K'' is not empty) of a
// block pair, each appended to the batch of its CTA shape (lb[0]: single CTAs, lb[1]: CTA pairs)
// after the units and tiles already there.  False when a batch is full.
template <int S>
bool add_pm_items(const ladder_plan_s& p, const BlockPair& bp, void* ws, LadBatch* lb) {
    const PmDims d = pm_dims(p.no, p.nv);
    const bool has_y = d.nm > 0 && d.km > 0;
    for (int part = 0; part < (has_y ? 2 : 1); ++part) {
        LadBatch& b = lb[(part == 0 ? d.np : d.nm) > kEmuTile ? 1 : 0];
        if (b.nitems >= kMaxItems) return false;
        LadItem* it = &b.item[b.nitems];
        if (!ladder_item_pm<S>(p, bp, ws, b.units, part == 0, it, &b.ta[b.nitems], &b.tb[b.nitems], b.tiles))
            return false;
        b.units += it->units;
        b.tiles += it->ntiles;
        ++b.nitems;
    }
    return true;
}

// Split form: R from the X and Y accumulators of a block pair.
void launch_finalize_pm(const ladder_plan_s& p, const BlockPair& bp, void* ws, double* R, cudaStream_t s) {
    const PmDims d = pm_dims(p.no, p.nv);
    const unsigned gx = (unsigned)std::min<long long>((bp.npairs + 255) / 256, 1024);
    const unsigned gy = (unsigned)std::min(d.np, 65535);
    finalize_pm_kernel<<<dim3(gx, gy), 256, 0, s>>>(
        at<unsigned long long>(ws, p.ws.rpx), at<unsigned long long>(ws, p.ws.rpy), bp.npairs, p.no, p.nv, d.np, d.nm,
        reinterpret_cast<const int2*>(p.d_tables) + bp.pairs_off, at<int>(ws, p.ws.v_exp), at<int>(ws, p.ws.tp_exp),
        at<int>(ws, p.ws.tm_exp), R, p.d_status);
}

// One block pair in the symmetric/antisymmetric form: ERI and self-product entries as in the
// plain form, V -> V', V'', the X and Y ladders (one launch each: at no=100 nv=700 nchol=4000 one
// launch for both took 5 % longer, at lower clocks under the power cap), and the four-way
// finalisation.
template <int S>
cudaError_t block_pm_impl(const ladder_plan_s& p, const BlockPair& bp, const double* L, double* R, void* ws,
                          cudaStream_t s) {
    cudaError_t e;
    if ((e = clear_pm_acc(p, bp, ws, s)) != cudaSuccess) return e;
    const int2* table = reinterpret_cast<const int2*>(p.d_tables);
    EriBatch eb{};
    eb.nitems = 1;
    eb.nentries = bp.ntiles;
    eb.entries = reinterpret_cast<const int4*>(table + bp.tiles_off);
    eb.status = p.d_status;
    eb.wait_ns = p.wait_ns;
    const int pb = lt_batch(p);
    if (pb >= p.nchol) {
        if (!eri_item<S>(p, bp, ws, &eb.item[0], &eb.ta[0], &eb.tb[0])) return cudaErrorInvalidValue;
        LaunchTimer tm(p, s, LADDER_KERNEL_ERI, 2);
        launch_eri_batch<S>(eb, p.eri_clusters > 0 ? p.eri_clusters : p.num_sms / 2, s);
        launch_self<S>(p, bp, ws, s);
    } else {
        // Cholesky vectors in batches: each batch's L^T planes are sliced into the workspace and its
        // ERI adds its exact int64 sums into V (same fixed-point unit for every batch: the exponents
        // are those of all the vectors); the last batch rounds V onto the pair's grid.
        for (int P0 = 0; P0 < p.nchol; P0 += pb) {
            const int count = std::min(pb, p.nchol - P0);
            const bool first = P0 == 0, last = P0 + pb >= p.nchol;
            {
                LaunchTimer tm(p, s, LADDER_KERNEL_PREP, 3);
                if ((e = slice_lt<S>(p, L, ws, P0, count, s)) != cudaSuccess) return e;
            }
            if (!eri_item<S>(p, bp, ws, &eb.item[0], &eb.ta[0], &eb.tb[0], count, first ? 0 : (last ? 2 : 1)))
                return cudaErrorInvalidValue;
            LaunchTimer tm(p, s, LADDER_KERNEL_ERI, last ? 2 : 1);
            launch_eri_batch<S>(eb, p.eri_clusters > 0 ? p.eri_clusters : p.num_sms / 2, s);
            if (last) launch_self<S>(p, bp, ws, s);
        }
    }
    {
        LaunchTimer tm(p, s, LADDER_KERNEL_COMBINE);
        launch_combine<S>(p, bp, ws, s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int fit = p.pair_clusters > 0 ? p.pair_clusters : p.num_sms / 2;
    {
        const PmDims dd = pm_dims(p.no, p.nv);
        const bool has_y = dd.nm > 0 && dd.km > 0;
        for (int part = 0; part < (has_y ? 2 : 1); ++part) {
            static thread_local LadBatch lb;
            lb = LadBatch{};
            lb.nitems = 1;
            lb.status = p.d_status;
            lb.wait_ns = p.wait_ns;
            if (!ladder_item_pm<S>(p, bp, ws, 0, part == 0, &lb.item[0], &lb.ta[0], &lb.tb[0]))
                return cudaErrorInvalidValue;
            lb.BN = ladder_bn(p, lb.item[0].M > kEmuTile);
            lb.units = lb.item[0].units;
            lb.tiles = lb.item[0].ntiles;
            LaunchTimer tm(p, s, LADDER_KERNEL_LADDER);
            launch_ladder_batch<S>(lb, lb.item[0].M > kEmuTile, fit, p.num_sms, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    {
        LaunchTimer tm(p, s, LADDER_KERNEL_FINISH);
        launch_finalize_pm(p, bp, ws, R, s);
    }
    return cudaGetLastError();
}

template <int S>
cudaError_t block_impl(const ladder_plan_s& p, const BlockPair& bp, const double* L, double* R, void* ws,
                       cudaStream_t s) {
    if (p.form == 1) return block_pm_impl<S>(p, bp, L, R, ws, s);
    if (lt_batch(p) < p.nchol) return cudaErrorInvalidValue;   // batches of vectors need the split form's int64 V
    const int no2 = p.no * p.no;
    cudaError_t e;
    // int64 ladder accumulator of this block pair starts at zero
    if ((e = cudaMemsetAsync(at<char>(ws, p.ws.rp_int), 0, (size_t)bp.npairs * no2 * 8, s)) != cudaSuccess) return e;

    const int2* table = reinterpret_cast<const int2*>(p.d_tables);
    EriBatch eb{};
    eb.nitems = 1;
    eb.nentries = bp.ntiles;
    eb.entries = reinterpret_cast<const int4*>(table + bp.tiles_off);
    eb.status = p.d_status;
    eb.wait_ns = p.wait_ns;
    if (!eri_item<S>(p, bp, ws, &eb.item[0], &eb.ta[0], &eb.tb[0])) return cudaErrorInvalidValue;
    {
        LaunchTimer tm(p, s, LADDER_KERNEL_ERI, 2);
        launch_eri_batch<S>(eb, p.eri_clusters > 0 ? p.eri_clusters : p.num_sms / 2, s);
        launch_self<S>(p, bp, ws, s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // Rows = (i,j), columns = 96 pairs, so the V planes stream from HBM once per row tile:
    // o^2 <= 128 in one 128-row tile (one SM per tile); larger o^2 in 256-row tiles on CTA pairs.
    LadBatch lb{};
    lb.nitems = 1;
    lb.BN = ladder_bn(p, ladder_on_pairs(p));
    lb.status = p.d_status;
    lb.wait_ns = p.wait_ns;
    if (!ladder_item<S>(p, bp, ws, 0, &lb.item[0], &lb.ta[0], &lb.tb[0])) return cudaErrorInvalidValue;
    lb.units = lb.item[0].units;
    lb.tiles = lb.item[0].ntiles;
    {
        LaunchTimer tm(p, s, LADDER_KERNEL_LADDER);
        launch_ladder_batch<S>(lb, ladder_on_pairs(p), p.pair_clusters > 0 ? p.pair_clusters : p.num_sms / 2,
                               p.num_sms, s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        LaunchTimer tm(p, s, LADDER_KERNEL_FINISH);
        const long long n = (long long)bp.npairs * no2;
        finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(at<unsigned long long>(ws, p.ws.rp_int),
                                                                    bp.npairs, p.no, p.nv, table + bp.pairs_off,
                                                                    at<int>(ws, p.ws.v_exp), at<int>(ws, p.ws.t_exp), R,
                                                                    p.d_status);
    }
    return cudaGetLastError();
}

// A group of instances, each planned as one block pair: every instance's operand preparation,
// then ONE persistent ERI launch over all their tiles, their self-product entries, ONE
// persistent ladder launch per ladder shape (single CTAs for o^2 <= 128, CTA pairs above) over
// all their units, and their finalisation.  The instances' workspaces start at ws[k].  The
// ERI tile list (z = position of the instance in the group) is built by the caller.
template <int S>
cudaError_t group_impl(const ladder_plan_s& parent, const ladder_plan_s* const* subs, int n, void* const* ws,
                       const double* const* L, const double* const* t2, double* const* R, const int4* entries,
                       int nentries, cudaStream_t s) {
    if (n < 1 || n > kMaxItems) return cudaErrorInvalidValue;
    cudaError_t e;
    for (int k = 0; k < n; ++k) {
        const ladder_plan_s& p = *subs[k];
        if (p.bps.size() != 1 || (p.form == 1 && lt_batch(p) < p.nchol)) return cudaErrorInvalidValue;
        if ((e = prep_impl<S>(p, L[k], t2[k], ws[k], s)) != cudaSuccess) return e;
        e = p.form == 1 ? clear_pm_acc(p, p.bps[0], ws[k], s)
                        : cudaMemsetAsync(at<char>(ws[k], p.ws.rp_int), 0, (size_t)p.bps[0].npairs * p.no * p.no * 8, s);
        if (e != cudaSuccess) return e;
    }
    static thread_local EriBatch eb;   // ~10 KB: kept off the stack
    eb = EriBatch{};
    eb.nitems = n;
    eb.nentries = nentries;
    eb.entries = entries;
    eb.status = parent.d_status;
    eb.wait_ns = parent.wait_ns;
    for (int k = 0; k < n; ++k)
        if (!eri_item<S>(*subs[k], subs[k]->bps[0], ws[k], &eb.item[k], &eb.ta[k], &eb.tb[k]))
            return cudaErrorInvalidValue;
    const int eri_fit = subs[0]->eri_clusters > 0 ? subs[0]->eri_clusters : subs[0]->num_sms / 2;
    const int pair_fit = subs[0]->pair_clusters > 0 ? subs[0]->pair_clusters : subs[0]->num_sms / 2;
    {
        LaunchTimer tm(parent, s, LADDER_KERNEL_ERI, 1 + n);
        launch_eri_batch<S>(eb, eri_fit, s);
        for (int k = 0; k < n; ++k) launch_self<S>(*subs[k], subs[k]->bps[0], ws[k], s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int n_pm = 0;
    for (int k = 0; k < n; ++k) n_pm += subs[k]->form == 1;
    if (n_pm > 0) {   // instances in the split form: V', V'' from their int64 V
        LaunchTimer tm(parent, s, LADDER_KERNEL_COMBINE, n_pm);
        for (int k = 0; k < n; ++k)
            if (subs[k]->form == 1) launch_combine<S>(*subs[k], subs[k]->bps[0], ws[k], s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // One persistent ladder launch per CTA shape over the items of every instance of the group
    // (one item per plain instance, X and Y per split-form instance).
    static thread_local LadBatch lbs[2];
    lbs[0] = LadBatch{};
    lbs[1] = LadBatch{};
    for (int k = 0; k < n; ++k) {
        const ladder_plan_s& p = *subs[k];
        if (p.form == 1) {
            if (!add_pm_items<S>(p, p.bps[0], ws[k], lbs)) return cudaErrorInvalidValue;
            continue;
        }
        LadBatch& lb = lbs[ladder_on_pairs(p) ? 1 : 0];
        if (lb.nitems >= kMaxItems) return cudaErrorInvalidValue;
        LadItem* it = &lb.item[lb.nitems];
        if (!ladder_item<S>(p, p.bps[0], ws[k], lb.units, it, &lb.ta[lb.nitems], &lb.tb[lb.nitems], lb.tiles))
            return cudaErrorInvalidValue;
        lb.units += it->units;
        lb.tiles += it->ntiles;
        ++lb.nitems;
    }
    for (int shape = 0; shape < 2; ++shape) {   // 0: single CTAs, 1: CTA pairs
        LadBatch& lb = lbs[shape];
        if (lb.nitems == 0) continue;
        lb.BN = shape == 1 ? kEmuTileN : parent.lad_bn;   // every single-CTA item of the group uses it
        lb.status = parent.d_status;
        lb.wait_ns = parent.wait_ns;
        LaunchTimer tm(parent, s, LADDER_KERNEL_LADDER);
        launch_ladder_batch<S>(lb, shape == 1, pair_fit, subs[0]->num_sms, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        LaunchTimer tm(parent, s, LADDER_KERNEL_FINISH, n);
        for (int k = 0; k < n; ++k) {
            const ladder_plan_s& p = *subs[k];
            const BlockPair& bp = p.bps[0];
            if (p.form == 1) {
                launch_finalize_pm(p, bp, ws[k], R[k], s);
                continue;
            }
            const long long cnt = (long long)bp.npairs * p.no * p.no;
            finalize_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
                at<unsigned long long>(ws[k], p.ws.rp_int), bp.npairs, p.no, p.nv,
                reinterpret_cast<const int2*>(p.d_tables) + bp.pairs_off, at<int>(ws[k], p.ws.v_exp),
                at<int>(ws[k], p.ws.t_exp), R[k], parent.d_status);
        }
    }
    return cudaGetLastError();
}

}  // namespace

template <int S>
cudaError_t set_attributes() {
    cudaError_t e = cudaFuncSetAttribute(eri_emu_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         eri_smem_bytes_for(S));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ladder_emu_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes_for(S));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ladder_pair_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pair_smem_bytes_for(S));
    return e;
}

template <int S>
int max_clusters_impl(int kind) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kind == 0 ? kThreadsEri : kThreadsTC, 1, 1);
    cfg.dynamicSmemBytes = kind == 0 ? eri_smem_bytes_for(S) : pair_smem_bytes_for(S);
    int n = 0;
    const cudaError_t e = kind == 0 ? cudaOccupancyMaxActiveClusters(&n, (void*)eri_emu_kernel<S>, &cfg)
                                    : cudaOccupancyMaxActiveClusters(&n, (void*)ladder_pair_kernel<S>, &cfg);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

int emu_max_clusters(int nslices, int kind) {
    switch (nslices) {
        case 5: return max_clusters_impl<5>(kind);
        case 6: return max_clusters_impl<6>(kind);
        case 7: return max_clusters_impl<7>(kind);
        case 8: return max_clusters_impl<8>(kind);
        default: return 0;
    }
}

bool emu_supported(int no, int nv, int nchol, int nslices) {
    (void)no;
    (void)nv;
    (void)nchol;
    return nslices >= 5 && nslices <= 8;
}

cudaError_t emu_set_attributes(int nslices) {
    switch (nslices) {
        case 5: return set_attributes<5>();
        case 6: return set_attributes<6>();
        case 7: return set_attributes<7>();
        case 8: return set_attributes<8>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_emu_prep(const ladder_plan_s& p, const double* L, const double* t2, void* ws, cudaStream_t s) {
    switch (p.nslices) {
        case 5: return prep_impl<5>(p, L, t2, ws, s);
        case 6: return prep_impl<6>(p, L, t2, ws, s);
        case 7: return prep_impl<7>(p, L, t2, ws, s);
        case 8: return prep_impl<8>(p, L, t2, ws, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_emu_group(const ladder_plan_s& parent, const ladder_plan_s* const* subs, int n, void* const* ws,
                             const double* const* L, const double* const* t2, double* const* R, const int4* entries,
                             int nentries, cudaStream_t s) {
    switch (parent.nslices) {
        case 5: return group_impl<5>(parent, subs, n, ws, L, t2, R, entries, nentries, s);
        case 6: return group_impl<6>(parent, subs, n, ws, L, t2, R, entries, nentries, s);
        case 7: return group_impl<7>(parent, subs, n, ws, L, t2, R, entries, nentries, s);
        case 8: return group_impl<8>(parent, subs, n, ws, L, t2, R, entries, nentries, s);
        default: return cudaErrorInvalidValue;
    }
}

int emu_max_group() { return kMaxItems; }

int emu_eri_stage_k(int nslices) { return eri_bk_for(nslices); }

cudaError_t launch_emu_block(const ladder_plan_s& p, const BlockPair& bp, const double* L, double* R, void* ws,
                             cudaStream_t s) {
    switch (p.nslices) {
        case 5: return block_impl<5>(p, bp, L, R, ws, s);
        case 6: return block_impl<6>(p, bp, L, R, ws, s);
        case 7: return block_impl<7>(p, bp, L, R, ws, s);
        case 8: return block_impl<8>(p, bp, L, R, ws, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ladder
