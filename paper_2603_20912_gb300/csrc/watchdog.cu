// ladder_watchdog_selftest: exercises the bounded wait that every tcgen05 kernel of the
// library uses for its mbarriers.  One thread initialises an mbarrier that nothing ever
// arrives on and waits on it with that same wait; the wait must give up after its time
// limit, record the timeout flag in a status word and let the kernel return, so the context
// stays usable.  Nothing faults, traps or loops without bound: the missing arrival only
// makes the wait run out.
#include <cuda_runtime.h>

#include "ladder_internal.h"
#include "tc_common.cuh"

namespace {

__global__ void watchdog_probe_kernel(unsigned* status, unsigned long long* waited_ns, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        ladder::tc::mbar_init(&bar, 1);
        ladder::tc::fence_barrier_init();
        const uint64_t t0 = ladder::tc::global_ns();
        ladder::tc::mbar_wait(&bar, 0, status, ladder::kStatusTimeout, limit_ns);
        *waited_ns = ladder::tc::global_ns() - t0;
    }
}

}  // namespace

extern "C" int ladder_watchdog_selftest(double limit_s, double* waited_ms, cudaStream_t stream) {
    if (!(limit_s >= 0.0) || limit_s > 60.0 || (limit_s > 0.0 && limit_s < 1e-3)) return LADDER_ERR_ARG;
    const unsigned long long limit_ns =
        limit_s == 0.0 ? ladder::kDefaultWaitNs : (unsigned long long)(limit_s * 1e9 + 0.5);
    unsigned* d_status = nullptr;
    unsigned long long* d_ns = nullptr;
    if (cudaMalloc(&d_status, 16) != cudaSuccess) return LADDER_ERR_CUDA;
    d_ns = reinterpret_cast<unsigned long long*>(d_status + 2);
    int rc = LADDER_OK;
    unsigned status = 0;
    unsigned long long ns = 0;
    if (cudaMemsetAsync(d_status, 0, 16, stream) != cudaSuccess) rc = LADDER_ERR_CUDA;
    if (rc == LADDER_OK) {
        watchdog_probe_kernel<<<1, 32, 0, stream>>>(d_status, d_ns, limit_ns);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess ||
            cudaMemcpy(&status, d_status, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = LADDER_ERR_CUDA;
    }
    cudaFree(d_status);
    if (rc != LADDER_OK) return rc;
    if (waited_ms) *waited_ms = (double)ns * 1e-6;
    return (status & ladder::kStatusTimeout) ? LADDER_ERR_TIMEOUT : LADDER_OK;
}
