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

}  // namespace

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
