// Emulated-FP64 path (BF16 digit slices on tcgen05).  Placeholder until the
// kernels land: plans for this precision are rejected as unsupported.
#include <cuda_runtime.h>

#include "ladder_internal.h"

namespace ladder {

bool emu_supported(int, int, int, int) { return false; }

cudaError_t launch_emu_prep(const ladder_plan_s&, const double*, const double*, void*, cudaStream_t) {
    return cudaErrorNotSupported;
}

cudaError_t launch_emu_block(const ladder_plan_s&, const BlockPair&, double*, void*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace ladder
