// phsp_host.h -- host-side helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "hydra_phsp.h"
#include "phsp_device.cuh"

namespace hydra {

struct MEConsts;

extern thread_local std::string g_last_error;

// Record a formatted message for hydra_last_error() and return st.
hydra_status fail(hydra_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
hydra_status cuda_fail(cudaError_t err, const char* what);

// Validate a decay and fill its launch constants (T = M - sum m in FP64, C_n, Philox keys).
hydra_status make_consts(double M, int n, const double* masses, uint64_t seed, DecayConsts* C);

// Validate a matrix element id and its parameters and fill both precisions.
hydra_status make_me(hydra_me_id me, int n, const double* params, int nparams, MEConsts* P);

// Arithmetic of FP64 generation (hydra_set_fp64_arith), shared by single and batched runs.
extern std::atomic<int> g_fp64_arith;

// Grid for a grid-stride kernel: min(blocks needed, resident blocks per SM x SMs).
int grid_for(const void* kernel, int block, uint64_t work_items);

// An NVTX range named after a C-ABI call (or a serving tick) for profiler timelines: pushed
// on construction, popped on destruction; a no-op check when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Release of the scratch owned by the other translation units (called by hydra_shutdown).
void release_extras_scratch();
void release_vegas_scratch();
void release_batch_run_scratch();

}  // namespace hydra
