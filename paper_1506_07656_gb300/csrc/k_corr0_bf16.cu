// Bottom-level correlation on BF16 tensor cores (not built yet).
#include "dm_internal.cuh"

cudaError_t dm_launch_corr0_bf16(const DmGeom&, const float*, const float*, float, void*, void*, float*,
                                 unsigned char*, cudaStream_t) {
    return cudaErrorNotSupported;
}
