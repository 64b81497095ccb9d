// Native FP64 path: Cholesky->ERI GEMM and ladder GEMM on FP64 DMMA
// (mma.sync m8n8k4 .f64), one (A, B) block pair at a time.
//
//   ERI   (C-split step0 'xac,xbd->acbd'):  V[(ab),(cd)] = sum_P L[P,a,c] L[P,b,d]
//   ladder (C-split step1 'acbd,ecfd->efab'): R[i,j,a,b] += sum_{cd} V[(ab),(cd)] t2[i,j,c,d]
//                                             and, for a < b, R[j,i,b,a] += the same value.
//
// The ERI is the Gram matrix of the rows (a,c) of L^T, so one GEMM tile covers
// rows r = (a - a0) nv + c and columns q = (b - b0) nv + d; in L both are
// contiguous offsets (a0 nv + r), (b0 nv + q) of the row L[P].  The epilogue
// scatters the tile into the packed V block (only a <= b is kept).  The ladder
// epilogue adds straight into R: every element of R belongs to exactly one
// (pair, ij) -- (i,j,a,b) for the pair (a,b), and its mirror (j,i,b,a) with
// b > a, which no pair owns directly -- so no atomics are needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ladder_internal.h"

namespace ladder {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;
constexpr int PADM = 66;  // smem row length (doubles); [k][m] layout
constexpr int THREADS = 128;

__device__ __forceinline__ void dmma_8x8x4(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// Operand whose row k (contraction index) is contiguous over m: elem(m,k) = base[k*ld + m].
struct KOuter {
    const double* base;
    size_t ld;
    int M, K;
    __device__ __forceinline__ void load(double (&r)[8], int m0, int k0) const {
        const int t = threadIdx.x;
        const int m = t & 63;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = (t >> 6) + 2 * i;
            const int gm = m0 + m, gk = k0 + k;
            r[i] = (gm < M && gk < K) ? __ldg(base + (size_t)gk * ld + gm) : 0.0;
        }
    }
    __device__ __forceinline__ void store(double (*s)[PADM], const double (&r)[8]) const {
        const int t = threadIdx.x;
        const int m = t & 63;
#pragma unroll
        for (int i = 0; i < 8; ++i) s[(t >> 6) + 2 * i][m] = r[i];
    }
};

// Operand whose row m is contiguous over k: elem(m,k) = base[m*ld + k].
struct KInner {
    const double* base;
    size_t ld;
    int M, K;
    __device__ __forceinline__ void load(double (&r)[8], int m0, int k0) const {
        const int t = threadIdx.x;
        const int k = t & 15;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = (t >> 4) + 8 * i;
            const int gm = m0 + m, gk = k0 + k;
            r[i] = (gm < M && gk < K) ? __ldg(base + (size_t)gm * ld + gk) : 0.0;
        }
    }
    __device__ __forceinline__ void store(double (*s)[PADM], const double (&r)[8]) const {
        const int t = threadIdx.x;
        const int k = t & 15;
#pragma unroll
        for (int i = 0; i < 8; ++i) s[k][(t >> 4) + 8 * i] = r[i];
    }
};

// acc[mi][ni][e]: row wm*32 + mi*8 + lane/4, col wn*32 + ni*8 + 2*(lane%4) + e.
template <class OpA, class OpB>
__device__ __forceinline__ void dgemm_tile(const OpA& A, const OpB& B, int m0, int n0, int K,
                                           double (&acc)[4][4][2]) {
    __shared__ double sA[2][TK][PADM];
    __shared__ double sB[2][TK][PADM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;

    double ra[8], rb[8];
    A.load(ra, m0, 0);
    B.load(rb, n0, 0);
    A.store(sA[0], ra);
    B.store(sB[0], rb);
    __syncthreads();
    const int nk = (K + TK - 1) / TK;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        const bool more = kt + 1 < nk;
        if (more) {
            A.load(ra, m0, (kt + 1) * TK);
            B.load(rb, n0, (kt + 1) * TK);
        }
#pragma unroll
        for (int kk = 0; kk < TK; kk += 4) {
            double af[4], bf[4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) af[mi] = sA[cur][kk + (lane & 3)][wm * 32 + mi * 8 + (lane >> 2)];
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) bf[ni] = sB[cur][kk + (lane & 3)][wn * 32 + ni * 8 + (lane >> 2)];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) dmma_8x8x4(acc[mi][ni], af[mi], bf[ni]);
        }
        if (more) {
            A.store(sA[cur ^ 1], ra);
            B.store(sB[cur ^ 1], rb);
        }
        __syncthreads();
    }
}

// ERI for one block pair: rows r in [0, na*nv) <-> (a0 + r/nv, r%nv), columns q
// in [0, nb*nv) <-> (b0 + q/nv, q%nv); writes V[row(a,b)][c*nv + d] for a <= b.
__global__ void __launch_bounds__(THREADS) eri_fp64_kernel(const double* __restrict__ L, int nv, int nchol,
                                                           int a0, int na, int b0, int nb,
                                                           const int* __restrict__ row_start,
                                                           double* __restrict__ V) {
    const int Mrows = na * nv, Ncols = nb * nv;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    // Skip tiles whose smallest a exceeds their largest b.
    const int a_min = a0 + m0 / nv;
    const int b_max = b0 + (min(n0 + TN, Ncols) - 1) / nv;
    if (a_min > b_max) return;
    const size_t nv2 = (size_t)nv * nv;
    KOuter A{L + (size_t)a0 * nv, nv2, Mrows, nchol};
    KOuter B{L + (size_t)b0 * nv, nv2, Ncols, nchol};
    double acc[4][4][2];
    dgemm_tile(A, B, m0, n0, nchol, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int r = m0 + wm * 32 + mi * 8 + (lane >> 2);
        if (r >= Mrows) continue;
        const int a = a0 + r / nv, c = r % nv;
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int q = n0 + wn * 32 + ni * 8 + 2 * (lane & 3) + e;
                if (q >= Ncols) continue;
                const int b = b0 + q / nv, d = q % nv;
                if (a > b) continue;
                const int row = row_start[a - a0] + (b - max(a, b0));
                V[(size_t)row * nv2 + (size_t)c * nv + d] = acc[mi][ni][e];
            }
    }
}

// Ladder for one block pair: Rp[m][n] = sum_k V[m][k] T[n][k], T = t2 viewed [no*no][nv*nv];
// then R[i,j,a,b] += Rp and (a < b) R[j,i,b,a] += Rp, with (a,b) = pairs[m], (i,j) = (n/no, n%no).
__global__ void __launch_bounds__(THREADS) ladder_fp64_kernel(const double* __restrict__ V,
                                                              const double* __restrict__ t2, int no,
                                                              int nv, int npairs,
                                                              const int2* __restrict__ pairs,
                                                              double* __restrict__ R) {
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const size_t nv2 = (size_t)nv * nv;
    const int N = no * no;
    KInner A{V, nv2, npairs, (int)nv2};
    KInner B{t2, nv2, N, (int)nv2};
    double acc[4][4][2];
    dgemm_tile(A, B, m0, n0, (int)nv2, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int m = m0 + wm * 32 + mi * 8 + (lane >> 2);
        if (m >= npairs) continue;
        const int2 ab = pairs[m];
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = n0 + wn * 32 + ni * 8 + 2 * (lane & 3) + e;
                if (n >= N) continue;
                const int i = n / no, j = n % no;
                const double v = acc[mi][ni][e];
                R[(((size_t)i * no + j) * nv + ab.x) * nv + ab.y] += v;
                if (ab.x < ab.y) R[(((size_t)j * no + i) * nv + ab.y) * nv + ab.x] += v;
            }
    }
}

// ---------------------------------------------------------------- factorised path
// R_ij = sum_P L_P T_ij L_P^T (Sec. "Acceleration of CC calculations": the evaluation order that
// contracts the amplitudes with one Cholesky factor at a time, x o^2 v^3 work per factor, instead
// of rebuilding (ac|bd)), over the amplitude pairs i <= j only (R_ji = R_ij^T, from
// t_ji^cd = t_ij^dc), in batches of Cholesky vectors P in [P0, P0 + pb):
//   W[ij][a][p][d] = sum_c L[P0+p, a, c] t2[i, j, c, d]        (fact_w_kernel)
//   R[i,j,a,b] += sum_{p,d} W[ij][a][p][d] L[P0+p, b, d]        (fact_r_kernel)
//   and R[j,i,b,a] += the same value for i < j.
// (i, j) of packed index u of the upper triangle (i <= j) of an n x n grid, row-major.
__device__ __forceinline__ void upper_pair(int u, int n, int& i, int& j) {
    int r = 0, start = 0;
    while (start + (n - r) <= u) {
        start += n - r;
        ++r;
    }
    i = r;
    j = r + (u - start);
}

// L rows b over the contraction index k = (p, d) of a batch of Cholesky vectors:
// elem(b, k) = L[P0 + k / nv][b][k % nv].
struct LPanel {
    const double* base;  // L + P0 * nv^2
    int nv, M, K;
    __device__ __forceinline__ void load(double (&r)[8], int m0, int k0) const {
        const int t = threadIdx.x;
        const int gk = k0 + (t & 15);
        const int p = gk / nv, d = gk - p * nv;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int gm = m0 + (t >> 4) + 8 * i;
            r[i] = (gm < M && gk < K) ? __ldg(base + ((size_t)p * nv + gm) * nv + d) : 0.0;
        }
    }
    __device__ __forceinline__ void store(double (*s)[PADM], const double (&r)[8]) const {
        const int t = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 8; ++i) s[t & 15][(t >> 4) + 8 * i] = r[i];
    }
};

// Grid: x over a tiles, y over d tiles, z over (p, ij) with ij fastest (z < pb * npij).
__global__ void __launch_bounds__(THREADS) fact_w_kernel(const double* __restrict__ L, const double* __restrict__ t2,
                                                         int no, int nv, int P0, int pb, int npij,
                                                         double* __restrict__ W) {
    const int z = blockIdx.z, u = z % npij, p = z / npij;
    int i, j;
    upper_pair(u, no, i, j);
    const size_t nv2 = (size_t)nv * nv;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    KInner A{L + (size_t)(P0 + p) * nv2, (size_t)nv, nv, nv};              // (a, c)
    KOuter B{t2 + ((size_t)i * no + j) * nv2, (size_t)nv, nv, nv};          // (d, c)
    double acc[4][4][2];
    dgemm_tile(A, B, m0, n0, nv, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    double* Wu = W + (size_t)u * nv * pb * nv;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int a = m0 + wm * 32 + mi * 8 + (lane >> 2);
        if (a >= nv) continue;
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int d = n0 + wn * 32 + ni * 8 + 2 * (lane & 3) + e;
                if (d < nv) Wu[((size_t)a * pb + p) * nv + d] = acc[mi][ni][e];
            }
    }
}

// Grid: x over a tiles, y over b tiles, z over ij (packed i <= j).
__global__ void __launch_bounds__(THREADS) fact_r_kernel(const double* __restrict__ L, const double* __restrict__ W,
                                                         int no, int nv, int P0, int pb, double* __restrict__ R) {
    const int u = blockIdx.z;
    int i, j;
    upper_pair(u, no, i, j);
    const size_t nv2 = (size_t)nv * nv;
    const int K = pb * nv;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    KInner A{W + (size_t)u * nv * K, (size_t)K, nv, K};                     // (a, (p, d))
    LPanel B{L + (size_t)P0 * nv2, nv, nv, K};                              // (b, (p, d))
    double acc[4][4][2];
    dgemm_tile(A, B, m0, n0, K, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    double* Rij = R + ((size_t)i * no + j) * nv2;
    double* Rji = R + ((size_t)j * no + i) * nv2;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int a = m0 + wm * 32 + mi * 8 + (lane >> 2);
        if (a >= nv) continue;
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int b = n0 + wn * 32 + ni * 8 + 2 * (lane & 3) + e;
                if (b >= nv) continue;
                const double v = acc[mi][ni][e];
                Rij[(size_t)a * nv + b] += v;
                if (i < j) Rji[(size_t)b * nv + a] += v;
            }
    }
}

// ---------------------------------------------------------------- fused path
// The two C-split steps of one batch (Sec. "An Asymmetric and Dynamic Splitting Protocol",
// Table 1: step 0 'xac,xbd->acbd', step 1 'acbd,ecfd->efab') kept on the chip: (ac|bd) never
// reaches HBM.  A CTA owns a tile of FA x FBT pairs (a, b) and all no^2 amplitude rows (i, j); it
// walks the (c, d) plane in FC x FD chunks.  For each chunk it builds
//   V[(a,c),(b,d)] = sum_P L[P,a,c] L[P,b,d]            (64 x 16 FBT DMMA GEMM, K = nchol)
// into shared memory and contracts it at once with the amplitudes,
//   acc[(i,j),(a,b)] += sum_{c,d in chunk} t2[i,j,c,d] V[(a,c),(b,d)],
// the accumulators staying in registers for the whole walk (warp w owns the 8-row (i,j) tiles
// w, w + 8, ..., so no^2 <= 64 MT).  The epilogue adds them into R[i,j,a,b] and, for a < b, into
// R[j,i,b,a]: the same ownership as the ladder epilogue above, so no atomics.  FP64 DMMA is the
// bound (about 3.5 flop per clock per SM on this GPU), so the simple staging below keeps it busy;
// what matters is issuing no DMMA without use: an 8 x 8 ERI sub-tile has one a and one b, so the
// sub-tiles of pairs a > b, of rows c >= nv or columns d >= nv (the ragged last chunk) and of a
// or b past the block are skipped, as are the ladder's K steps whose (c, d) lie past nv.
constexpr int FA = 4, FC = 16, FD = 16;
constexpr int FM = FA * FC;                 // ERI chunk rows (a,c): 64
constexpr int FK = 16;                      // Cholesky vectors per staging step
constexpr int FTHREADS = 256;

template <int FBT>
struct FusedShape {
    static constexpr int FN = FBT * FD;             // ERI chunk columns (b,d)
    static constexpr int WN = FN / 16;              // warps along the columns (16 each)
    static constexpr int WM = 8 / WN;               // warps along the rows
    static constexpr int MI = FM / WM / 8;          // 8-row sub-tiles per warp
    static constexpr int NPAIR = FA * FBT;          // pairs of the tile
    static constexpr int NT = NPAIR / 8;            // 8-pair ladder column tiles
    static constexpr int VLD = FN + 1;              // V chunk row length (doubles)
    static constexpr int BPT = FN * FK / FTHREADS;  // B staging values per thread
    static constexpr int STAGE = 2 * FK * (FM + FN);
    static constexpr int SMEM = STAGE > FM * VLD ? STAGE : FM * VLD;
    static_assert(WN * WM == 8 && MI >= 1 && NT >= 1 && BPT >= 1, "warp layout");
};

template <int MT, int FBT>
__global__ void __launch_bounds__(FTHREADS) ladder_fused_fp64_kernel(const double* __restrict__ L,
                                                                     const double* __restrict__ t2, int no, int nv,
                                                                     int nchol, int a0, int a1, int b0, int b1,
                                                                     double* __restrict__ R) {
    using Sh = FusedShape<FBT>;
    constexpr int FN = Sh::FN, MI = Sh::MI, NT = Sh::NT;
    // Staging buffers sA[2][FK][FM], sB[2][FK][FN] during a chunk's ERI; the V chunk Vs[FM][VLD]
    // during its ladder step (the two phases are separated by barriers).
    __shared__ __align__(16) double smem[Sh::SMEM];
    double(*sA)[FK][FM] = reinterpret_cast<double(*)[FK][FM]>(smem);
    double(*sB)[FK][FN] = reinterpret_cast<double(*)[FK][FN]>(smem + 2 * FK * FM);
    double(*Vs)[Sh::VLD] = reinterpret_cast<double(*)[Sh::VLD]>(smem);

    const int nta = (a1 - a0 + FA - 1) / FA;
    const int at = a0 + (int)(blockIdx.x % nta) * FA, bt = b0 + (int)(blockIdx.x / nta) * FBT;
    if (at > min(bt + FBT, b1) - 1) return;   // no pair a <= b in the tile
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp / Sh::WN, wn = warp % Sh::WN;   // ERI: warp rows of 8 MI, columns of 16
    const int no2 = no * no, mtiles = (no2 + 7) / 8;
    const size_t nv2 = (size_t)nv * nv;

    double acc[MT][NT][2];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = 0.0;

    // Staging map: A row m = t % 64 at the vectors t / 64 + 4i; B row n = t % FN at the vectors
    // t / FN + (256 / FN) i.
    const int am = threadIdx.x & 63, ak = threadIdx.x >> 6;
    const int bn = threadIdx.x % FN, bk = threadIdx.x / FN;
    const int arow = at + am / FC, brow = bt + bn / FD;
    // The warp's ERI sub-tiles: a of row sub-tile mi, b of its 16 columns.
    const int b_w = bt + wn;
    // Ladder column tile nt holds pairs nt*8 .. nt*8+7 (a_i = n / FBT, b_i = n % FBT): in use when
    // its smallest a is inside the block.
    bool nt_on[NT];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) nt_on[nt] = at + (nt * 8) / FBT < a1;

    for (int c0 = 0; c0 < nv; c0 += FC) {
        const int ac = c0 + am % FC;
        const bool a_ok = arow < a1 && ac < nv;
        const double* pa = L + (size_t)arow * nv + ac;
        // row sub-tile mi: a = at + (wm*8MI + 8mi) / 16, first c = c0 + (8mi) % 16 (wm*8MI is a
        // multiple of 16 whenever MI >= 2)
        bool m_on[MI];
        int a_of[MI];
#pragma unroll
        for (int mi = 0; mi < MI; ++mi) {
            const int r0 = wm * 8 * MI + mi * 8;
            a_of[mi] = at + r0 / FC;
            m_on[mi] = a_of[mi] < a1 && c0 + r0 % FC < nv;
        }
        for (int d0 = 0; d0 < nv; d0 += FD) {
            const int bd = d0 + bn % FD;
            const bool b_ok = brow < b1 && bd < nv;
            const double* pb = L + (size_t)brow * nv + bd;
            bool on[MI][2];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < 2; ++ni)
                    on[mi][ni] = m_on[mi] && b_w < b1 && d0 + ni * 8 < nv && a_of[mi] <= b_w;
            // ---- ERI chunk: e[mi][ni][.] = rows wm*8MI + mi*8 + lane/4, columns wn*16 + ni*8 + 2(lane%4) + .
            double e[MI][2][2];
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < 2; ++ni) e[mi][ni][0] = e[mi][ni][1] = 0.0;
            double ra[4], rb[Sh::BPT];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int P = ak + 4 * i;
                ra[i] = a_ok && P < nchol ? __ldg(pa + (size_t)P * nv2) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < Sh::BPT; ++i) {
                const int P = bk + (FTHREADS / FN) * i;
                rb[i] = b_ok && P < nchol ? __ldg(pb + (size_t)P * nv2) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) sA[0][ak + 4 * i][am] = ra[i];
#pragma unroll
            for (int i = 0; i < Sh::BPT; ++i) sB[0][bk + (FTHREADS / FN) * i][bn] = rb[i];
            __syncthreads();
            const int nk = (nchol + FK - 1) / FK;
            for (int kt = 0; kt < nk; ++kt) {
                const int cur = kt & 1;
                const bool more = kt + 1 < nk;
                if (more) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int P = (kt + 1) * FK + ak + 4 * i;
                        ra[i] = a_ok && P < nchol ? __ldg(pa + (size_t)P * nv2) : 0.0;
                    }
#pragma unroll
                    for (int i = 0; i < Sh::BPT; ++i) {
                        const int P = (kt + 1) * FK + bk + (FTHREADS / FN) * i;
                        rb[i] = b_ok && P < nchol ? __ldg(pb + (size_t)P * nv2) : 0.0;
                    }
                }
#pragma unroll
                for (int kk = 0; kk < FK; kk += 4) {
                    double af[MI], bf[2];
#pragma unroll
                    for (int mi = 0; mi < MI; ++mi)
                        af[mi] = sA[cur][kk + (lane & 3)][wm * 8 * MI + mi * 8 + (lane >> 2)];
#pragma unroll
                    for (int ni = 0; ni < 2; ++ni) bf[ni] = sB[cur][kk + (lane & 3)][wn * 16 + ni * 8 + (lane >> 2)];
#pragma unroll
                    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                        for (int ni = 0; ni < 2; ++ni)
                            if (on[mi][ni]) dmma_8x8x4(e[mi][ni], af[mi], bf[ni]);   // warp-uniform
                }
                if (more) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) sA[cur ^ 1][ak + 4 * i][am] = ra[i];
#pragma unroll
                    for (int i = 0; i < Sh::BPT; ++i) sB[cur ^ 1][bk + (FTHREADS / FN) * i][bn] = rb[i];
                }
                __syncthreads();
            }
            // The staging buffers are dead now: the V chunk takes their place (zero where skipped).
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < 2; ++ni)
#pragma unroll
                    for (int x = 0; x < 2; ++x)
                        Vs[wm * 8 * MI + mi * 8 + (lane >> 2)][wn * 16 + ni * 8 + 2 * (lane & 3) + x] = e[mi][ni][x];
            __syncthreads();
            // ---- ladder step over the chunk's K = (c, d), c = k / FD, d = k % FD.
            // B operand of pair n = (a_i, b_i) = (n / FBT, n % FBT): V[(a_i, c), (b_i, d)].
            int vr[NT], vc[NT];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int n = nt * 8 + (lane >> 2);
                vr[nt] = (n / FBT) * FC;
                vc[nt] = (n % FBT) * FD;
            }
            const int c_end = min(FC, nv - c0), d_end = min(FD, nv - d0);
            for (int c = 0; c < c_end; ++c) {
#pragma unroll
                for (int dd = 0; dd < FD; dd += 4) {
                    if (dd >= d_end) break;   // warp-uniform: the K steps past nv
                    const int d = dd + (lane & 3);
                    const bool cd_ok = d < d_end;
                    double v[NT];
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) v[nt] = Vs[vr[nt] + c][vc[nt] + d];
                    const double* tk = t2 + (size_t)(c0 + c) * nv + (d0 + d);
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        const int tile = warp + 8 * mt;
                        if (tile < mtiles) {   // warp-uniform
                            const int ij = tile * 8 + (lane >> 2);
                            const double tv = cd_ok && ij < no2 ? __ldg(tk + (size_t)ij * nv2) : 0.0;
#pragma unroll
                            for (int nt = 0; nt < NT; ++nt)
                                if (nt_on[nt]) dmma_8x8x4(acc[mt][nt], tv, v[nt]);
                        }
                    }
                }
            }
            __syncthreads();   // Vs is read by every warp before the next chunk stages into it
        }
    }
    // ---- epilogue: acc[mt][nt][x] is row (i,j) = (warp + 8 mt) * 8 + lane/4, pair n = nt*8 + 2(lane%4) + x.
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
        const int ij = (warp + 8 * mt) * 8 + (lane >> 2);
        if (warp + 8 * mt >= mtiles || ij >= no2) continue;
        const int i = ij / no, j = ij % no;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                const int n = nt * 8 + 2 * (lane & 3) + x;
                const int a = at + n / FBT, b = bt + n % FBT;
                if (a >= a1 || b >= b1 || a > b) continue;
                const double v = acc[mt][nt][x];
                R[(((size_t)i * no + j) * nv + a) * nv + b] += v;
                if (a < b) R[(((size_t)j * no + i) * nv + b) * nv + a] += v;
            }
    }
}

// Pair tiles of a block pair that hold a pair a <= b, for FA x fb tiles.
long long fused_tiles(const BlockPair& bp, int fb) {
    long long n = 0;
    for (int at = bp.a0; at < bp.a1; at += FA)
        for (int bt = bp.b0; bt < bp.b1; bt += fb)
            if (at <= std::min(bt + fb, bp.b1) - 1) ++n;
    return n;
}

template <int FBT>
cudaError_t launch_fused_fbt(const ladder_plan_s& p, const BlockPair& bp, const double* L, const double* t2,
                             double* R, cudaStream_t s) {
    const int mtiles = (p.no * p.no + 7) / 8, per_warp = (mtiles + 7) / 8;
    const long long nta = (bp.a1 - bp.a0 + FA - 1) / FA, ntb = (bp.b1 - bp.b0 + FBT - 1) / FBT;
    if (per_warp > 16 || nta * ntb > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)(nta * ntb);
#define LADDER_FUSED_LAUNCH(MT)                                                                           \
    ladder_fused_fp64_kernel<MT, FBT><<<grid, FTHREADS, 0, s>>>(L, t2, p.no, p.nv, p.nchol, bp.a0, bp.a1, \
                                                                bp.b0, bp.b1, R)
    if (per_warp <= 1) LADDER_FUSED_LAUNCH(1);
    else if (per_warp <= 2) LADDER_FUSED_LAUNCH(2);
    else if (per_warp <= 4) LADDER_FUSED_LAUNCH(4);
    else if (per_warp <= 8) LADDER_FUSED_LAUNCH(8);
    else LADDER_FUSED_LAUNCH(16);
#undef LADDER_FUSED_LAUNCH
    return cudaGetLastError();
}

}  // namespace

int fused_fp64_max_rows() { return 8 * 8 * 16; }

int fused_fp64_tile_b(const ladder_plan_s& p, const BlockPair& bp) {
    // The 4 x 2 tile (two CTAs per SM, half the work per CTA, so the SMs' shares of the tiles
    // come out more even) unless the 4 x 4 one (one CTA per SM: its accumulators take most of the
    // registers) fills the SMs' shares better by more than 2 % of the work.
    const double sms = std::max(1, p.num_sms);
    const long long t4 = fused_tiles(bp, 4), t2_ = fused_tiles(bp, 2);
    const double fill4 = t4 / (std::ceil(t4 / sms) * sms), fill2 = t2_ / (std::ceil(t2_ / sms) * sms);
    return fill4 > fill2 + 0.02 ? 4 : 2;
}

cudaError_t launch_fp64_fused(const ladder_plan_s& p, const BlockPair& bp, const double* L, const double* t2,
                              double* R, cudaStream_t s) {
    LaunchTimer t(p, s, LADDER_KERNEL_FUSED);
    return fused_fp64_tile_b(p, bp) == 2 ? launch_fused_fbt<2>(p, bp, L, t2, R, s)
                                         : launch_fused_fbt<4>(p, bp, L, t2, R, s);
}

cudaError_t launch_fp64_factorised(const ladder_plan_s& p, const double* L, const double* t2, double* R, void* ws,
                                   cudaStream_t s) {
    const int npij = p.no * (p.no + 1) / 2;
    double* W = reinterpret_cast<double*>(static_cast<char*>(ws) + p.ws.w_blk);
    const unsigned tiles = (unsigned)((p.nv + TM - 1) / TM);
    for (int P0 = 0; P0 < p.nchol; P0 += p.fact_pb) {
        const int pb = std::min(p.fact_pb, p.nchol - P0);
        {
            LaunchTimer t(p, s, LADDER_KERNEL_FACT_W);
            fact_w_kernel<<<dim3(tiles, tiles, (unsigned)(pb * npij)), THREADS, 0, s>>>(L, t2, p.no, p.nv, P0, pb,
                                                                                       npij, W);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        {
            LaunchTimer t(p, s, LADDER_KERNEL_FACT_R);
            fact_r_kernel<<<dim3(tiles, tiles, (unsigned)npij), THREADS, 0, s>>>(L, W, p.no, p.nv, P0, pb, R);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fp64_block(const ladder_plan_s& p, const BlockPair& bp, const double* L,
                              const double* t2, double* R, void* ws, cudaStream_t s) {
    const int na = bp.a1 - bp.a0, nb = bp.b1 - bp.b0;
    const int2* pairs = reinterpret_cast<const int2*>(p.d_tables) + bp.pairs_off;
    const int* row_start = reinterpret_cast<const int*>(reinterpret_cast<const int2*>(p.d_tables)) + bp.rows_off;
    double* V = reinterpret_cast<double*>(static_cast<char*>(ws) + p.ws.v_blk);
    dim3 g1((na * p.nv + TM - 1) / TM, (nb * p.nv + TN - 1) / TN);
    {
        LaunchTimer t(p, s, LADDER_KERNEL_ERI);
        eri_fp64_kernel<<<g1, THREADS, 0, s>>>(L, p.nv, p.nchol, bp.a0, na, bp.b0, nb, row_start, V);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2((bp.npairs + TM - 1) / TM, (p.no * p.no + TN - 1) / TN);
    {
        LaunchTimer t(p, s, LADDER_KERNEL_LADDER);
        ladder_fp64_kernel<<<g2, THREADS, 0, s>>>(V, t2, p.no, p.nv, bp.npairs, pairs, R);
    }
    return cudaGetLastError();
}

}  // namespace ladder
