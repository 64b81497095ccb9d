// ladder_energy_noalloc: the ladder energy for callers that cannot allocate
// device memory.
//
// Some callers of this library cannot call cudaMalloc at the point where they
// need E_L: code running while a CUDA stream is being captured into a graph
// (allocation is not a capturable operation), host frameworks that own every
// byte of device memory through their own pool and forbid other allocators,
// and real-time loops that must not take the allocator's locks.  For them
// this entry point needs no plan and no workspace: its reduction scratch is
// a file-scope __device__ array that every device loading the library holds
// until the process exits (kMaxPartials doubles = 128 KiB per device).
//
// Host code must not pass the array's name to a kernel: in host code that
// name is only a host-side shadow, so a kernel given it would fault or, where
// the GPU can reach host memory, silently use the wrong memory.  The device
// address is looked up with cudaGetSymbolAddress, with that device current, on
// the first call made on that device, and again whenever the driver context
// current on the calling thread is not the one the address was taken in (after
// cudaDeviceReset the module is loaded afresh and the array may sit elsewhere;
// a caller's own driver-API context holds its own copy of the array).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "ladder_internal.h"

namespace {

constexpr int kMaxPartials = LADDER_NOALLOC_MAX_PARTIALS;  // scratch capacity (doubles)
static_assert(kMaxPartials * sizeof(double) == 128 * 1024, "the header documents 128 KiB of scratch");
constexpr int kUnitsPerBlock = 64;         // 32x32 tiles reduced by one block (fixed: reproducible sums)
constexpr int kThreads = 256;
constexpr int kTile = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_scratch[kMaxPartials];

std::mutex g_setup_mutex;
struct ScratchAddr {
    CUcontext ctx = nullptr;   // driver context the address belongs to
    double* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

__device__ __forceinline__ double block_sum(double v, double* red) {
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// Block b reduces the contiguous units [b*kUnitsPerBlock, (b+1)*kUnitsPerBlock); a unit is one
// 32x32 (a, b) tile of one (i, j) slab.  It writes exactly one partial, so no scratch entry needs
// clearing between calls.
__global__ void __launch_bounds__(kThreads) energy_partial_fixed(const double* __restrict__ t2,
                                                                 const double* __restrict__ R, int no, int nv,
                                                                 long long units, double* __restrict__ partials) {
    __shared__ double tt[kTile][kTile + 1];
    __shared__ double red[kThreads];
    const int ntile = (nv + kTile - 1) / kTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc = 0.0;
    const long long u0 = (long long)blockIdx.x * kUnitsPerBlock;
    const long long u1 = u0 + kUnitsPerBlock < units ? u0 + kUnitsPerBlock : units;
    for (long long u = u0; u < u1; ++u) {
        const int bt = (int)(u % ntile);
        const int at = (int)((u / ntile) % ntile);
        const long long ij = u / ((long long)ntile * ntile);
        const double* st = t2 + (size_t)ij * nv * nv;
        const double* sr = R + (size_t)ij * nv * nv;
        for (int r = ty; r < kTile; r += kThreads / 32) {
            const int b = bt * kTile + r, a = at * kTile + tx;
            tt[r][tx] = (b < nv && a < nv) ? st[(size_t)b * nv + a] : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < kTile; r += kThreads / 32) {
            const int a = at * kTile + r, b = bt * kTile + tx;
            if (a < nv && b < nv) {
                const size_t o = (size_t)a * nv + b;
                acc += (2.0 * st[o] - tt[tx][r]) * sr[o];
            }
        }
        __syncthreads();
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) energy_final_fixed(const double* __restrict__ partials, int n,
                                                               double* __restrict__ E) {
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += kThreads) acc += partials[k];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) *E = s;
}

// The driver's cuCtxGetCurrent, reached through the runtime (no link-time libcuda dependency).
PFN_cuCtxGetCurrent_v4000 ctx_get_current() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
    });
    return fn;
}

// Device address of the scratch array on the current device, looked up once per device and
// driver context.  Before the runtime has bound a context to the thread, cuCtxGetCurrent gives
// none; the lookup itself binds the device's primary context, which is then recorded.
int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return LADDER_ERR_UNSUPPORTED;
    auto get_ctx = ctx_get_current();
    if (!get_ctx) return LADDER_ERR_CUDA;
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) return LADDER_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchAddr& e = g_scratch_addr[dev];
    if (e.addr == nullptr || ctx == nullptr || e.ctx != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || p == nullptr) return LADDER_ERR_CUDA;
        if (ctx == nullptr && (get_ctx(&ctx) != CUDA_SUCCESS || ctx == nullptr)) return LADDER_ERR_CUDA;
        e.addr = static_cast<double*>(p);
        e.ctx = ctx;
    }
    *out = e.addr;
    return LADDER_OK;
}

}  // namespace

extern "C" int ladder_energy_noalloc(int no, int nv, const double* t2, const double* R, double* E_dev,
                                     cudaStream_t stream) {
    if (no < 1 || nv < 1 || !t2 || !R || !E_dev) return LADDER_ERR_ARG;
    const long long ntile = (nv + kTile - 1) / kTile;
    const long long units = (long long)no * no * ntile * ntile;
    const long long nblocks = (units + kUnitsPerBlock - 1) / kUnitsPerBlock;
    if (nblocks > kMaxPartials) return LADDER_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LADDER_ERR_CUDA;
    double* partials = nullptr;
    const int rc = scratch_address(dev, &partials);
    if (rc != LADDER_OK) return rc;
    energy_partial_fixed<<<(unsigned)nblocks, kThreads, 0, stream>>>(t2, R, no, nv, units, partials);
    if (cudaGetLastError() != cudaSuccess) return LADDER_ERR_CUDA;
    energy_final_fixed<<<1, kThreads, 0, stream>>>(partials, (int)nblocks, E_dev);
    if (cudaGetLastError() != cudaSuccess) return LADDER_ERR_CUDA;
    return LADDER_OK;
}
