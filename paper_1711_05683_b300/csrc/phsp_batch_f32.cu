// phsp_batch_f32.cu -- the FP32 persistent batch kernel at each block size the autotuner may
// choose (its own translation unit, compiled in parallel with the runner's).
#include <cuda_runtime.h>

#include "phsp_batch.cuh"

namespace hydra {

const void* batch_kernel_f32(int block) {
    switch (block) {
        case 128: return reinterpret_cast<const void*>(&phsp_batch_kernel<float, float, 128>);
        case 512: return reinterpret_cast<const void*>(&phsp_batch_kernel<float, float, 512>);
        default: return reinterpret_cast<const void*>(&phsp_batch_kernel<float, float, 256>);
    }
}

void launch_batch_kernel_f32(int block, int grid, BatchHeader* hdr, TileSums* partials, cudaStream_t s) {
    if (block == 128) phsp_batch_kernel<float, float, 128><<<grid, 128, 0, s>>>(hdr, partials);
    else if (block == 512) phsp_batch_kernel<float, float, 512><<<grid, 512, 0, s>>>(hdr, partials);
    else phsp_batch_kernel<float, float, 256><<<grid, 256, 0, s>>>(hdr, partials);
}

}  // namespace hydra
