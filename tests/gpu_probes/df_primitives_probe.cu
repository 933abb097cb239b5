// Test probe: runs the library's double-float device primitives (phsp_df.cuh) on given inputs
// and returns the results as doubles, so that a test can compare them with exact values.
// Test infrastructure only; built by tests/test_gpu_df_primitives.py.
#include <cuda_runtime.h>
#include <cstdint>
#include "phsp_df.cuh"

using namespace hydra;

namespace {

__global__ void k_u32(int op, const uint32_t* x, int n, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    df v;
    if (op == 0) v = df_half_odd_u32(x[i]);        // (x + 1/2) 2^-31
    else if (op == 1) v = df_half_odd_centered(x[i]);  // (x - 2^31 + 1/2) 2^-31
    else if (op == 2) v = df_from_u32(x[i]);       // x
    else v = df_half_odd_raw(x[i]);                // x + 1/2
    out[2 * i] = static_cast<double>(v.hi);
    out[2 * i + 1] = static_cast<double>(v.lo);
}

__global__ void k_sincos(const uint32_t* x, int n, double* out) {
    df_sincos_table_init();
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        df s, c;
        df_sincos_2pi_u(x[i], s_sincos_table, &s, &c);
        out[4 * i] = s.hi;
        out[4 * i + 1] = s.lo;
        out[4 * i + 2] = c.hi;
        out[4 * i + 3] = c.lo;
    }
}

__global__ void k_frac64(const uint64_t* v, int n, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df f = df_frac_u64(v[i]);
    out[2 * i] = f.hi;
    out[2 * i + 1] = f.lo;
}

// prod_k p_k of k = 0..m-1 factors given as double-float pairs (hi, lo), times c
__global__ void k_weight(const float* p, int m, double c, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DfWeight w = df_weight_one();
    for (int k = 0; k < m; ++k) w = df_weight_mul(w, df{p[2 * k], p[2 * k + 1]});
    out[0] = df_weight_final(w, c);
}

// df (p[2i], p[2i+1]) to double: out[2i] the stored-kinematics conversion, out[2i+1] the exact one
__global__ void k_to_double(const float* p, int n, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df v{p[2 * i], p[2 * i + 1]};
    out[2 * i] = df_to_double(v);
    out[2 * i + 1] = df_to_double_exact(v);
}

int finish(const double* dev_out, double* host_out, size_t out_bytes) {
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpy(host_out, dev_out, out_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
    return 0;
}

}  // namespace

extern "C" {

// op 0..3 (see k_u32); out[2i], out[2i+1] = hi, lo
int probe_df_u32(int op, const uint32_t* x, int n, double* out) {
    uint32_t* dx = nullptr;
    double* dout = nullptr;
    if (cudaMalloc(&dx, n * sizeof(uint32_t)) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    cudaMemcpy(dx, x, n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    k_u32<<<(n + 127) / 128, 128>>>(op, dx, n, dout);
    const int rc = finish(dout, out, 2 * n * sizeof(double));
    cudaFree(dx);
    cudaFree(dout);
    return rc;
}

// out[4i..4i+3] = sin hi, sin lo, cos hi, cos lo of 2 pi (x + 1/2) 2^-32
int probe_df_sincos(const uint32_t* x, int n, double* out) {
    uint32_t* dx = nullptr;
    double* dout = nullptr;
    if (cudaMalloc(&dx, n * sizeof(uint32_t)) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, 4 * n * sizeof(double)) != cudaSuccess) return 1;
    cudaMemcpy(dx, x, n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    k_sincos<<<1, 256>>>(dx, n, dout);
    const int rc = finish(dout, out, 4 * n * sizeof(double));
    cudaFree(dx);
    cudaFree(dout);
    return rc;
}

// out[2i], out[2i+1] = hi, lo of v 2^-64
int probe_df_frac64(const uint64_t* v, int n, double* out) {
    uint64_t* dv = nullptr;
    double* dout = nullptr;
    if (cudaMalloc(&dv, n * sizeof(uint64_t)) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    cudaMemcpy(dv, v, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    k_frac64<<<(n + 127) / 128, 128>>>(dv, n, dout);
    const int rc = finish(dout, out, 2 * n * sizeof(double));
    cudaFree(dv);
    cudaFree(dout);
    return rc;
}

// out[0] = (prod of m double-float factors p[2k] + p[2k+1]) * c
int probe_df_weight(const float* p, int m, double c, double* out) {
    float* dp = nullptr;
    double* dout = nullptr;
    if (cudaMalloc(&dp, 2 * m * sizeof(float)) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, sizeof(double)) != cudaSuccess) return 1;
    cudaMemcpy(dp, p, 2 * m * sizeof(float), cudaMemcpyHostToDevice);
    k_weight<<<1, 32>>>(dp, m, c, dout);
    const int rc = finish(dout, out, sizeof(double));
    cudaFree(dp);
    cudaFree(dout);
    return rc;
}

// out[2i], out[2i+1] = df_to_double, df_to_double_exact of the pair (p[2i], p[2i+1])
int probe_df_to_double(const float* p, int n, double* out) {
    float* dp = nullptr;
    double* dout = nullptr;
    if (cudaMalloc(&dp, 2 * n * sizeof(float)) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, 2 * n * sizeof(double)) != cudaSuccess) return 1;
    cudaMemcpy(dp, p, 2 * n * sizeof(float), cudaMemcpyHostToDevice);
    k_to_double<<<(n + 127) / 128, 128>>>(dp, n, dout);
    const int rc = finish(dout, out, 2 * n * sizeof(double));
    cudaFree(dp);
    cudaFree(dout);
    return rc;
}

}  // extern "C"
