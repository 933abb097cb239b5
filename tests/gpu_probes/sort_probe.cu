// Test probe: runs the generator's sorting network for the intermediate-mass draws
// (sort_mass_draws<K>, phsp_device.cuh) on rows of K uint32 values, so that a test can compare
// it with a library sort.  Test infrastructure only; built by tests/test_gpu_sort_network.py.
#include <cuda_runtime.h>
#include <cstdint>
#include "phsp_device.cuh"

using namespace hydra;

namespace {

template <int K>
__global__ void k_sort(const uint32_t* in, uint64_t rows, uint32_t* out) {
    const uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < K; ++i) x[i] = in[r * K + i];
    sort_mass_draws<K>(x);
#pragma unroll
    for (int i = 0; i < K; ++i) out[r * K + i] = x[i];
}

template <int K>
int run(const uint32_t* h_in, uint64_t rows, uint32_t* h_out) {
    const size_t bytes = rows * K * sizeof(uint32_t);
    uint32_t *d_in = nullptr, *d_out = nullptr;
    if (cudaMalloc(&d_in, bytes) != cudaSuccess) return 1;
    if (cudaMalloc(&d_out, bytes) != cudaSuccess) {
        cudaFree(d_in);
        return 1;
    }
    cudaError_t err = cudaMemcpy(d_in, h_in, bytes, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) {
        k_sort<K><<<static_cast<unsigned>((rows + 255) / 256), 256>>>(d_in, rows, d_out);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpy(h_out, d_out, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d_in);
    cudaFree(d_out);
    return err == cudaSuccess ? 0 : 2;
}

}  // namespace

extern "C" int probe_sort(int k, const uint32_t* in, uint64_t rows, uint32_t* out) {
    switch (k) {
        case 1: return run<1>(in, rows, out);
        case 2: return run<2>(in, rows, out);
        case 3: return run<3>(in, rows, out);
        case 4: return run<4>(in, rows, out);
        case 5: return run<5>(in, rows, out);
        case 6: return run<6>(in, rows, out);
        case 7: return run<7>(in, rows, out);
        case 8: return run<8>(in, rows, out);
    }
    return 3;
}
