// Test probe: evaluates cuRAND's raw Philox4x32-10 block function (curand_Philox4x32_10 from
// curand_philox4x32_x.h) on given counters and keys, so a test can compare it with the
// oracle's Philox.  Built by the test suite only; not part of the library.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <cstdint>

__global__ void probe_kernel(const uint32_t* in, int count, uint32_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t* r = in + 6 * i;
    uint4 c = make_uint4(r[0], r[1], r[2], r[3]);
    uint2 k = make_uint2(r[4], r[5]);
    uint4 o = curand_Philox4x32_10(c, k);
    out[4 * i + 0] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
}

// in: count rows of (ctr0..3, key0..1); out: count rows of 4 words.  Returns a cudaError_t.
extern "C" int probe_curand_philox(const uint32_t* in_host, int count, uint32_t* out_host) {
    uint32_t *din = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&din, sizeof(uint32_t) * 6 * count);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(uint32_t) * 4 * count);
    if (e == cudaSuccess) e = cudaMemcpy(din, in_host, sizeof(uint32_t) * 6 * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        probe_kernel<<<(count + 127) / 128, 128>>>(din, count, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_host, dout, sizeof(uint32_t) * 4 * count, cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    return static_cast<int>(e);
}
