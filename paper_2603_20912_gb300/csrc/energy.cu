// Ladder energy E_L = sum_{ijab} (2 t2[i,j,a,b] - t2[i,j,b,a]) R[i,j,a,b] in FP64.
//
// Two launches with a fixed reduction tree, so the value is bit-reproducible
// for a given (no, nv) and grid: every block accumulates a fixed, strided set
// of (i,j) slabs, reduces them in shared memory, and writes one partial; one
// block then sums the partials in index order.  Each (i,j) slab is an nv x nv
// matrix; the transposed read t2[i,j,b,a] goes through a shared-memory tile so
// that both reads are coalesced.
#include <cuda_runtime.h>

#include "ladder_internal.h"

namespace ladder {
namespace {

constexpr int ETHREADS = 256;
constexpr int ET = 32;  // transpose tile

__device__ __forceinline__ double block_sum(double v, double* red) {
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int w = ETHREADS / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// Work unit = one (i, j, a-tile, b-tile) 32x32 tile of the slab.
__global__ void __launch_bounds__(ETHREADS) energy_partial_kernel(const double* __restrict__ t2,
                                                                  const double* __restrict__ R, int no,
                                                                  int nv, double* __restrict__ partials) {
    __shared__ double tt[ET][ET + 1];
    __shared__ double red[ETHREADS];
    const int ntile = (nv + ET - 1) / ET;
    const long long units = (long long)no * no * ntile * ntile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    double acc = 0.0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int bt = (int)(u % ntile);
        const int at = (int)((u / ntile) % ntile);
        const long long ij = u / ((long long)ntile * ntile);
        const double* slab_t = t2 + (size_t)ij * nv * nv;
        const double* slab_r = R + (size_t)ij * nv * nv;
        // Load t2[ij][b][a] for b in the b-tile (rows), a in the a-tile (cols) -> tt[b][a].
        for (int r = ty; r < ET; r += 8) {
            const int b = bt * ET + r, a = at * ET + tx;
            tt[r][tx] = (b < nv && a < nv) ? slab_t[(size_t)b * nv + a] : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < ET; r += 8) {
            const int a = at * ET + r, b = bt * ET + tx;
            if (a < nv && b < nv) {
                const size_t o = (size_t)a * nv + b;
                acc += (2.0 * slab_t[o] - tt[tx][r]) * slab_r[o];
            }
        }
        __syncthreads();
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(ETHREADS) energy_final_kernel(const double* __restrict__ partials, int n,
                                                                double* __restrict__ E) {
    __shared__ double red[ETHREADS];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += ETHREADS) acc += partials[k];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) *E = s;
}

}  // namespace

cudaError_t launch_energy(const ladder_plan_s& p, const double* t2, const double* R, double* E_dev,
                          cudaStream_t s) {
    energy_partial_kernel<<<p.n_partials, ETHREADS, 0, s>>>(t2, R, p.no, p.nv, p.d_partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<1, ETHREADS, 0, s>>>(p.d_partials, p.n_partials, E_dev);
    return cudaGetLastError();
}

}  // namespace ladder
