/*
 * hydra_phsp.h -- C ABI of the B300 (sm_103a) phase-space Monte Carlo library.
 *
 * The library implements the data-parallel hot path of the phase-space Monte Carlo of
 * Hydra (arXiv:1711.05683, section 4.2 "Phase-Space Monte Carlo"): the Raubold-Lynch
 * N-body event generator with per-event weights (F. James, "Monte Carlo Phase Space",
 * CERN 68-15), and the weighted phase-space integral of a matrix element over its events
 * (section 3, "phase-space Monte Carlo integration").  The paper's user API is Listing 4:
 * PhaseSpace<N>(mother_mass, daughter_masses) and Generate(mother, events) filling a
 * structure-of-arrays container of N 4-vectors plus a weight per event.
 *
 * Conventions shared by every entry point
 *   - A decay is a parent of mass M > 0 at rest decaying to n daughters, 2 <= n <= 10,
 *     with masses m_i >= 0 and kinetic energy T = M - sum m_i > 0 (computed in FP64 on the
 *     host).  Masses are in any unit (GeV in the tests); outputs are in the same unit.
 *   - 4-vectors are (E, px, py, pz), energy first (Listing 4, Vector4R(M, 0, 0, 0)).
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed
 *     (key = (seed low word, seed high word)).  Event e of a call uses the counter-event
 *     index event_offset + e; draw d of that event is word d%4 of the Philox block with
 *     counter (index low word, index high word, d/4, 0).  Each event uses 3n-4 draws: the
 *     n-2 intermediate-mass draws, then (cos theta, phi) for each of the n-1 two-body
 *     decays, parent first.  Hence one call over [0, a+b) equals two calls over [0, a)
 *     and [a, a+b) (event_offset = a), bit for bit, at any launch shape.
 *   - Weights: w = C_n * prod_k p*_k, with C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M),
 *     so that E[w] = R_n = Int prod d3p_i/(2 E_i) delta4(P - sum p_i) (no 2 pi factors;
 *     the conventional Phi_n = R_n (2 pi)^(4-3n)).
 *   - Streams: hydra_stream_t is the CUDA runtime's cudaStream_t (NULL = legacy default
 *     stream).  Device pointers belong to the device current on the calling thread.
 *   - Errors: every entry point returns a hydra_status; nothing is thrown across the ABI.
 *     On an error nothing has been launched, except HYDRA_ERR_CUDA which reports a CUDA
 *     error from a launch or copy.  hydra_last_error() gives a message for the calling
 *     thread's most recent failure.
 *   - Memory: the caller owns every buffer passed in.  The library owns a small scratch
 *     area per device for the integral's partial sums (allocated on first use, released
 *     by hydra_shutdown).
 */
#ifndef HYDRA_PHSP_H
#define HYDRA_PHSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *hydra_stream_t;

typedef enum hydra_status {
    HYDRA_OK = 0,
    HYDRA_ERR_INVALID_ARG = 1,     /* bad value: non-finite/negative mass, M <= 0, NULL, ld < nevents, ... */
    HYDRA_ERR_BELOW_THRESHOLD = 2, /* sum of daughter masses >= M */
    HYDRA_ERR_UNSUPPORTED_N = 3,   /* n outside [2, 10] (or an ME id that needs another n) */
    HYDRA_ERR_MISALIGNED = 4,      /* buffer not 16-byte aligned or ld not a multiple of 4 */
    HYDRA_ERR_OOM = 5,             /* the library could not allocate its scratch memory */
    HYDRA_ERR_CUDA = 6,            /* a CUDA runtime call or kernel launch failed */
    HYDRA_ERR_TIMEOUT = 7,         /* a bounded device-side wait ran out */
    HYDRA_ERR_BUSY = 8             /* admission refused: over the memory budget */
} hydra_status;

typedef enum hydra_dtype {
    HYDRA_F32 = 0, /* FP32 kinematics, float outputs and weights */
    HYDRA_F64 = 1  /* FP64 kinematics, double outputs and weights */
} hydra_dtype;

typedef enum hydra_me_id {
    HYDRA_ME_FLAT = 0,      /* |ME|^2 = 1: the integral is the phase-space volume R_n */
    HYDRA_ME_DALITZ_2BW = 1 /* n = 3 only; params = (m0a, Ga, m0b, Gb, |c|, arg c):
                               |BW(s12; m0a, Ga) + |c| e^{i arg c} BW(s23; m0b, Gb)|^2,
                               BW(s; m0, G) = 1 / (m0^2 - s - i m0 G), s_ij = (p_i + p_j)^2 */
} hydra_me_id;

/* Kernels whose launch shape can be configured. */
typedef enum hydra_kernel_kind {
    HYDRA_KERNEL_GENERATE = 0, /* hydra_phsp_generate / hydra_phsp_generate_host */
    HYDRA_KERNEL_INTEGRATE = 1 /* hydra_phsp_integrate (all matrix elements) */
} hydra_kernel_kind;

/* Result of a phase-space integral of f = w |ME|^2 over n events. */
typedef struct hydra_integral {
    double mean;     /* sum_f / n: the MC estimate of Int |ME|^2 dR_n */
    double var_mean; /* variance of that mean: (sum_f2/n - mean^2) / (n - 1) */
    double sum_f;    /* sum of f */
    double sum_f2;   /* sum of f^2 */
    double sum_w;    /* sum of w (sum_w / n estimates R_n) */
    double sum_w2;   /* sum of w^2 */
    uint64_t n;      /* number of events */
} hydra_integral;

/* Message for the calling thread's most recent failing call ("" if none). */
const char *hydra_last_error(void);

/* Static name of a status code. */
const char *hydra_status_string(hydra_status status);

/*
 * Weight constant C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M) of the decay (host only).
 * Section 4.2, "weighted samples": w = C_n prod p*_k has mean R_n.
 * C_n (out, host) receives the value.  Errors: INVALID_ARG, UNSUPPORTED_N, BELOW_THRESHOLD.
 */
hydra_status hydra_phsp_volume_factor(double M, int n, const double *masses, double *C_n);

/*
 * Generate nevents weighted phase-space events (section 4.2; Listing 4's Generate).
 *
 *   M, n, masses  parent mass and the n daughter masses (host array of n doubles).
 *   nevents       events to generate; 0 is a no-op that returns HYDRA_OK.
 *   seed          Philox key.  event_offset: counter-event index of event 0 (see above);
 *                 event_offset + nevents must not exceed 2^64.
 *   dtype         HYDRA_F32 (float) or HYDRA_F64 (double) for kinematics and outputs.
 *   out           device buffer, structure of arrays [n][4][ld] of dtype: component c
 *                 (E, px, py, pz) of daughter i (masses[i]) for event e is at
 *                 out[(i*4 + c)*ld + e].  16-byte aligned; ld >= nevents, ld % 4 == 0.
 *   weights       device buffer of nevents dtype values, 16-byte aligned.
 *   stream        CUDA stream; the call is asynchronous with respect to the host.
 *
 * Errors: UNSUPPORTED_N, INVALID_ARG (M, masses, dtype, NULL buffers, ld < nevents,
 * offset overflow), BELOW_THRESHOLD, MISALIGNED, CUDA (launch failure).
 */
hydra_status hydra_phsp_generate(double M, int n, const double *masses, uint64_t nevents,
                                 uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                 void *out, uint64_t ld, void *weights, hydra_stream_t stream);

/*
 * hydra_phsp_generate with HOST output buffers (end-to-end use: events land in host memory).
 *
 * Same arguments and event definition as hydra_phsp_generate, except that out_host
 * ([n][4][ld], any ld >= nevents) and weights_host are host buffers; page-locked memory
 * (cudaMallocHost / cudaHostRegister) gives full copy bandwidth.  The library generates
 * chunks of 2^22 events into two device staging buffers it owns and copies each chunk to
 * the host on its own copy stream while the next chunk is generated on `stream`.  The call
 * blocks until every event is in host memory.  Errors: as hydra_phsp_generate (no
 * alignment rule for host buffers), plus OOM for the staging buffers.
 */
hydra_status hydra_phsp_generate_host(double M, int n, const double *masses, uint64_t nevents,
                                      uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                      void *out_host, uint64_t ld, void *weights_host,
                                      hydra_stream_t stream);

/*
 * Events of a moving parent (Listing 4, Generate(Mother, ...)): each event is generated in
 * the parent rest frame exactly as hydra_phsp_generate generates it, then every daughter is
 * taken to the frame where the parent has momentum p (energy sqrt(M^2 + p^2)) by the pure
 * boost E' = (P0 E + P.p)/M, p' = p + P (E' + E)/(P0 + M).  Weights are Lorentz invariant and
 * unchanged.  Give exactly one of:
 *   mother_p   host array of 3 doubles: one parent momentum for every event;
 *   mothers    device array [3][mld] of dtype: the momentum of event e's parent at
 *              mothers[c*mld + e] (c = x, y, z), mld >= nevents.
 * Other arguments, layout and errors as hydra_phsp_generate.  Asynchronous.
 */
hydra_status hydra_phsp_generate_boosted(double M, int n, const double *masses, uint64_t nevents,
                                         uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                         const double *mother_p, const void *mothers, uint64_t mld,
                                         void *out, uint64_t ld, void *weights, hydra_stream_t stream);

/*
 * Unweighting by accept-reject (section 4.2, "unweighted samples"): event e (counter-event
 * index event_offset + e, with n daughters and key `seed`) is kept when u_e w_max < w_e, where
 * u_e = (x + 1/2) 2^-32 and x is the event's draw 3n-4, the first draw after those of its
 * kinematics; the product and the comparison are in the weights' precision.
 *   weights     device array of nevents dtype values (from hydra_phsp_generate)
 *   w_max       the bound; <= 0 uses the largest weight of the sample
 *   indices     device array with room for nevents int64: receives the kept event indices
 *               in increasing order (deterministic)
 *   naccepted   host: number of kept events; w_max_used (host, optional): the bound used
 * Keeps about nevents / 4 bytes of device scratch (one accept bit and the tile counts and
 * offsets per event) until a larger call or hydra_shutdown.
 * Blocks until the count is on the host.  Errors: UNSUPPORTED_N, INVALID_ARG, OOM, CUDA.
 */
hydra_status hydra_phsp_unweight(int n, uint64_t nevents, uint64_t seed, uint64_t event_offset,
                                 hydra_dtype dtype, const void *weights, double w_max,
                                 int64_t *indices, uint64_t *naccepted, double *w_max_used,
                                 hydra_stream_t stream);

/*
 * Evaluation of a matrix element on stored events (section 4.2, "evaluation of model";
 * section 3, "parallel function evaluation on multidimensional data-sets"):
 * f_e = w_e |ME|^2(p_e) with s_ij = (p_i + p_j)^2 formed from the stored 4-vectors.
 *   events, ld   device SoA [n][4][ld] of dtype (may be NULL for HYDRA_ME_FLAT)
 *   weights      device array of nevents dtype values
 *   values       device array receiving f_e (dtype), or NULL
 *   result       host: mean, variance of the mean and sums of f and w, reduced in the fixed
 *                tile / segment order of hydra_phsp_integrate (deterministic)
 * With events, weights and values 16-byte aligned and ld a multiple of 4 (FP32) or 2 (FP64)
 * a lane reads runs of consecutive events with 16-byte loads; otherwise one event per lane
 * (the same values; the sums differ by rounding in their grouping).  FP64 events: the pair
 * masses and m0^2 - s in FP64, the rest of |ME|^2 in double-float (hydra_set_fp64_arith
 * selects FP64 throughout).
 * Blocking.  Errors: UNSUPPORTED_N, INVALID_ARG, OOM, CUDA.
 */
hydra_status hydra_phsp_evaluate(int n, uint64_t nevents, hydra_dtype dtype, hydra_me_id me,
                                 const double *params, int nparams, const void *events, uint64_t ld,
                                 const void *weights, void *values, hydra_integral *result,
                                 hydra_stream_t stream);

/*
 * VEGAS importance sampling over the phase-space variables (section 3, "self-adaptive
 * importance sampling"; section 4.1; G. P. Lepage, J. Comput. Phys. 27 (1978) 192):
 * Int |ME|^2 dR_n as the integral of F(u) = w(u) |ME|^2(event(u)) over the unit cube of the
 * D = 3n-4 Raubold-Lynch variables (u_0..u_{n-3} intermediate-mass uniforms, then one
 * (cos theta, phi) pair per top-down step), through a separable grid of `bins` bins per
 * dimension, refined after every iteration.  Iteration i draws `calls` points: y_d =
 * (x + 1/2) 2^-32 from Philox word d%4 of counter (s low, s high, d/4, i + 1) with key
 * `seed`; bin b = floor(y_d K); u_d = g_d[b] + (y_d K - b)(g_d[b+1] - g_d[b]); f = F(u) J with
 * J = prod_d K (g_d[b+1] - g_d[b]).  Estimate = mean of f, variance (<f^2> - <f>^2)/(calls-1)
 * (both reduced in the deterministic group / tile / segment tree of hydra_phsp_integrate, with
 * tiles of 512 points).  Each bin
 * collects sum f^2 (64-bit fixed point relative to the iteration's largest f^2, so the
 * histogram is order independent); refinement smooths it (1,2,1)/4 inside and (1,1)/2 at the
 * ends, weights each bin ((r - 1)/ln r)^alpha with r its share, and places the new edges at
 * equal shares of the total weight.  Iterations skip.. are combined with weights 1/var.
 * FP64 throughout.  bins = 1 is plain Monte Carlo.
 *   me, params   as hydra_phsp_integrate
 *   calls        points per iteration, 2 .. 2^36 (8 + 4 ceil((3n-4)/4) bytes of device scratch each)
 *   iterations   >= 1; bins: 1..256 with (3n-4) bins <= 6144; alpha >= 0; 0 <= skip < iterations
 *   est, var     host arrays of `iterations` doubles: each iteration's estimate and variance
 *   result       host double[3]: combined estimate, its standard deviation, chi^2 per degree
 *                of freedom of the combined iterations (0 for one)
 *   grid_out     host double[(3n-4)(bins+1)] receiving the final grid edges, or NULL
 * Blocking (one host synchronisation per call: the grids are refined on the device).
 * Errors: UNSUPPORTED_N, BELOW_THRESHOLD, INVALID_ARG, OOM, CUDA.
 */
hydra_status hydra_phsp_vegas(double M, int n, const double *masses, uint64_t seed, hydra_me_id me,
                              const double *params, int nparams, uint64_t calls, int iterations,
                              int bins, double alpha, int skip, double *est, double *var,
                              double *result, double *grid_out, hydra_stream_t stream);

/*
 * Copy selected events (e.g. the kept events of hydra_phsp_unweight) into a compact SoA
 * buffer: dst[(i*4 + c)*dst_ld + j] = src[(i*4 + c)*src_ld + indices[j]] for j < count, and
 * dst_weights[j] = src_weights[indices[j]] when both weight pointers are non-NULL.  Device
 * buffers of dtype; dst_ld >= count.  Asynchronous.  Errors: UNSUPPORTED_N, INVALID_ARG, CUDA.
 */
hydra_status hydra_phsp_gather(int n, hydra_dtype dtype, const void *src, uint64_t src_ld,
                               const void *src_weights, const int64_t *indices, uint64_t count,
                               void *dst, uint64_t dst_ld, void *dst_weights, hydra_stream_t stream);

/*
 * Phase-space integral of f = w |ME|^2 over nevents events (section 3, "phase-space Monte
 * Carlo integration"; the events are those hydra_phsp_generate would produce for the same
 * seed and event_offset, computed on the device and never stored).
 *
 *   kin_dtype     HYDRA_F32: FP32 kinematics and matrix element, FP64 accumulation;
 *                 HYDRA_F64: FP64-accurate kinematics and matrix element (double-float by
 *                 default, FP64 instructions after hydra_set_fp64_arith(HYDRA_FP64_NATIVE)),
 *                 f, w and all sums in FP64.
 *   me, params, nparams  matrix element id and its parameters (host array).
 *   result        host struct that receives the sums, mean and variance of the mean.
 *
 * Sums are accumulated in a fixed order that depends only on the event indices (tiles of
 * 2048 events in FP64, then FP64 compensated sums over tiles and segments), so the result
 * is the same bit for bit at every launch shape.  The call blocks until the result is on
 * the host.  Errors: as hydra_phsp_generate, plus UNSUPPORTED_N for an ME that needs
 * another n, INVALID_ARG for too few params or nevents == 0, OOM for scratch memory.
 */
hydra_status hydra_phsp_integrate(double M, int n, const double *masses, uint64_t nevents,
                                  uint64_t seed, uint64_t event_offset, hydra_dtype kin_dtype,
                                  hydra_me_id me, const double *params, int nparams,
                                  hydra_integral *result, hydra_stream_t stream);

/*
 * hydra_phsp_integrate without any memory allocation (the paper has no counterpart: this
 * entry point exists for callers of this library that cannot allocate device memory).
 *
 * Some callers cannot call cudaMalloc: processes that forbid dynamic device allocation once
 * they are running (real-time or certified hosts), plug-ins whose host application owns all
 * device memory through its own pool, and latency-critical loops where cudaMalloc/cudaFree
 * may synchronize the whole device and stall other streams.  This variant makes no
 * allocating call (no cudaMalloc, cudaFree or allocating library routine): its scratch is a
 * fixed array of 1,179,904 bytes (tile partials of one 2^26-event chunk, 2048 segment
 * partials, the result) compiled into the library as a static device variable, which every
 * GPU that loads the library holds until the process exits.
 *
 * Arguments, result and numerics are those of hydra_phsp_integrate, bit for bit, with one
 * extra limit: nevents <= 2^32 (larger counts return HYDRA_ERR_INVALID_ARG with a message).
 * Every call looks up the device address of the array on the current device
 * (cudaGetSymbolAddress) and ends by synchronising the stream, so it cannot be recorded in a
 * stream capture.  All calls share the one array, which keeps the previous call's contents;
 * every slot a call reads is written earlier in the same call, so nothing needs clearing.
 * Calls are serialized within the process by a lock and block until the result is on the
 * host; calls that overlap on the GPU (for instance issued around that lock) race on the
 * shared array and give wrong results.
 */
hydra_status hydra_phsp_integrate_noalloc(double M, int n, const double *masses, uint64_t nevents,
                                          uint64_t seed, uint64_t event_offset,
                                          hydra_dtype kin_dtype, hydra_me_id me,
                                          const double *params, int nparams,
                                          hydra_integral *result, hydra_stream_t stream);

/*
 * The raw random numbers of nevents events: the 3n-4 Philox4x32-10 draws of each event in
 * draw order (section 4.2's generator consumes them as described at the top of this file).
 * out: device buffer of uint32, structure of arrays out[d * ld + e], ld >= nevents.
 * Asynchronous.  Errors: UNSUPPORTED_N, INVALID_ARG, CUDA.
 */
hydra_status hydra_phsp_draws(int n, uint64_t nevents, uint64_t seed, uint64_t event_offset,
                              uint32_t *out, uint64_t ld, hydra_stream_t stream);

/*
 * Launch shape of a kernel for decays of n daughters in a precision: threads per block
 * (a multiple of 32 in [32, 512]) and events per thread (1, 2 or 4; each thread carries
 * that many independent events in lockstep, and the generator stores them as one vector).
 * Results do not depend on the shape: every event's arithmetic is the same, and integrals
 * use a fixed reduction tree.  Process-wide; used by the autotuner.  The library's defaults
 * are the shapes measured best on B300.  Errors: INVALID_ARG, UNSUPPORTED_N.
 */
hydra_status hydra_set_launch_config(hydra_kernel_kind kind, int n, hydra_dtype dtype, int block,
                                     int events_per_thread);
hydra_status hydra_get_launch_config(hydra_kernel_kind kind, int n, hydra_dtype dtype, int *block,
                                     int *events_per_thread);

/* ------------------------------------------------------------------------------------
 * Batches: many uneven requests in one persistent launch (CUDA-graph replay).
 *
 * A batch is a list of request slices.  The persistent kernel's warps take tiles of 2048
 * events from all slices in turn (an atomic tile counter), so thousands of small and large
 * requests with different n, masses and event counts keep every SM busy in one launch.
 * Each slice gives exactly the events (and, for integrals, exactly the bits) that the
 * single-request entry points give for the same arguments.
 * ------------------------------------------------------------------------------------ */
typedef enum hydra_request_kind {
    HYDRA_REQ_GENERATE = 0,
    HYDRA_REQ_INTEGRATE = 1
} hydra_request_kind;

typedef struct hydra_request {
    int32_t kind;           /* hydra_request_kind */
    int32_t n;              /* daughters, 2..10 */
    int32_t dtype;          /* hydra_dtype; all slices of one batch run share it */
    int32_t me;             /* integrate: hydra_me_id */
    double M;               /* parent mass */
    double masses[10];      /* daughter masses (first n used) */
    double params[6];       /* integrate: matrix-element parameters */
    uint64_t seed;          /* Philox key */
    uint64_t event_offset;  /* counter-event index of the request's event 0 */
    uint64_t first;         /* first event of this slice within the request */
    uint64_t count;         /* events in this slice (> 0) */
    /* generate: device buffers of this slice: event first + j of the request goes to
     * out[(i*4 + c)*ld + j] and weights[j]; 16-byte aligned, ld % 4 == 0, ld >= count. */
    void *out;
    uint64_t ld;
    void *weights;
    /* integrate: total events of the request; the slice must start on a multiple of 2^21
     * events and, unless it ends the request, hold a multiple of 2^21 events.  seg_partials
     * is a device array of 8 doubles per 2^21-event segment of the whole request, owned by
     * the caller and kept between the slices of one request.  When a slice ends the request
     * (first + count == total) its result is available from hydra_batch_result. */
    uint64_t total;
    double *seg_partials;
} hydra_request;

typedef struct hydra_batch hydra_batch; /* opaque; bound to the device current at creation */

/*
 * Create a batch runner for up to max_requests slices per run and up to max_integrate_tiles
 * tiles (2048 events each) of integral slices per run.  Allocates its device and pinned host
 * buffers and captures the CUDA graph of a run (tile-counter reset, persistent batch kernel,
 * segment reduction, finalization).  Errors: INVALID_ARG, OOM, CUDA.
 */
hydra_status hydra_batch_create(int max_requests, uint64_t max_integrate_tiles, hydra_batch **out);

/*
 * Enqueue one run of nreq slices on `stream` (asynchronous): one host-to-device copy of
 * the slice table, one graph launch (use_graph != 0) or the same kernels launched one by
 * one, and one device-to-host copy of the results of the integral slices.  The tiles are
 * handed out grouped by kind, matrix element and n (stable within a group); every event
 * depends only on its request and counter, so results do not depend on the table order.  A run may be
 * issued while the previous run of the same batch is still executing; the call waits for
 * that run's slice table to be consumed before reusing its staging memory.
 * Errors: INVALID_ARG (validation of every slice, capacity), UNSUPPORTED_N,
 * BELOW_THRESHOLD, MISALIGNED, CUDA.
 */
hydra_status hydra_batch_run(hydra_batch *batch, const hydra_request *reqs, int nreq, int use_graph,
                             hydra_stream_t stream);

/*
 * Result of slice i of the latest run (an integral slice that ended its request).  Blocks
 * until that run has finished.  Errors: INVALID_ARG (index, kind, or a slice that did not
 * end its request), CUDA.
 */
hydra_status hydra_batch_result(hydra_batch *batch, int i, hydra_integral *result);

/* Wait for the latest run and release the batch runner. */
hydra_status hydra_batch_destroy(hydra_batch *batch);

/*
 * Launch shape of the persistent batch kernel (no counterpart in the paper; the autotuner sets
 * it).  block: threads per block of FP32 runs, 128, 256 or 512 (FP64 runs: 256), read when a
 * runner is created (hydra_batch_create, hydra_phsp_batch_run); ept_by_n[n], n = 2..10: events
 * each thread of a generation tile computes in lockstep (FP32: 1, 2, or 4 for n <= 6; FP64: 2),
 * read by every run.  Entries 0 and 1 are ignored.  Results do not depend on the shape.
 * Process-wide.  Errors: INVALID_ARG.
 */
hydra_status hydra_set_batch_shape(hydra_dtype dtype, int block, const int32_t *ept_by_n);
hydra_status hydra_get_batch_shape(hydra_dtype dtype, int *block, int32_t *ept_by_n);

/* ------------------------------------------------------------------------------------
 * Whole requests under a device-memory budget (section 4.2's generation and section 3's
 * integration for many requests at once).
 * ------------------------------------------------------------------------------------ */
typedef enum hydra_dest {
    HYDRA_DEST_NONE = 0,   /* generated outputs are computed and dropped with their wave */
    HYDRA_DEST_HOST = 1,   /* out / weights are host buffers (page-locked memory copies fastest) */
    HYDRA_DEST_DEVICE = 2  /* out / weights are device buffers, written in place */
} hydra_dest;

typedef struct hydra_batch_request {
    int32_t kind;          /* HYDRA_REQ_GENERATE or HYDRA_REQ_INTEGRATE */
    int32_t n;             /* daughters, 2..10 */
    int32_t dtype;         /* hydra_dtype; all requests of one call share it */
    int32_t me;            /* integrate: hydra_me_id (FP32 or FP64 kinematics as dtype) */
    double M;              /* parent mass */
    double masses[10];     /* daughter masses (first n used) */
    double params[6];      /* integrate: matrix-element parameters */
    uint64_t seed;         /* Philox key */
    uint64_t event_offset; /* counter-event index of the request's event 0 */
    uint64_t nevents;      /* > 0 */
    int32_t dest;          /* generate: hydra_dest */
    int32_t status;        /* out: HYDRA_OK, or the validation error of this request */
    void *out;             /* generate, HOST or DEVICE: [n][4][ld] of dtype (DEVICE: 16-byte aligned) */
    uint64_t ld;           /* >= nevents (DEVICE: a multiple of 4) */
    void *weights;         /* generate, HOST or DEVICE: nevents values of dtype (DEVICE: 16-byte aligned) */
    hydra_integral result; /* integrate, out: as hydra_phsp_integrate */
} hydra_batch_request;

/*
 * Run nreq whole requests (generate or integrate, any n, masses and event counts) with at most
 * budget_bytes of device memory allocated by the call, and block until every output is in its
 * destination and every integral result is in its request.
 *
 * The call validates every request first (each one's status is set; on the first invalid one
 * it returns that error and launches nothing).  From the budget it takes the batch runner's
 * tables and tile partials and the integrals' segment storage (8 doubles per 2^21 events), and
 * the rest is the output arena.  Requests are packed in order into waves: a generate request
 * with destination NONE or HOST takes [4n+1][ld] values of the arena (ld = events rounded up
 * to 4), a request larger than the arena (half of it when any output goes to the host) is
 * split across waves, DEVICE outputs are written in place, and integrals run as slices of 2^26
 * events (at most 16 per wave).  Each wave is one run of a batch runner (hydra_batch_run: one
 * persistent launch, replayed from a CUDA graph, with the shape of hydra_set_batch_shape).
 * Outputs bound for the host are copied out of one half of the arena on a copy stream while
 * the next wave computes into the other half.  Every event and every integral is bit for bit
 * what hydra_phsp_generate / hydra_phsp_integrate give for the same arguments.
 *
 * Errors: the validation errors of hydra_phsp_generate and hydra_phsp_integrate (per request),
 * INVALID_ARG (no requests, mixed dtypes, a budget too small for these requests), OOM, CUDA.
 */
hydra_status hydra_phsp_batch_run(hydra_batch_request *reqs, int nreq, size_t budget_bytes, hydra_stream_t stream);

/* Waves and slices of the calling thread's latest successful hydra_phsp_batch_run. */
hydra_status hydra_phsp_batch_stats(uint64_t *waves, uint64_t *slices);

/*
 * Continuous-batching server (section 4.2's generation and section 3's integration as a
 * service): the serving loop in C++ over two batch runners.  Requests arrive over time; each
 * turn of the loop admits arrived requests while their memory fits two device rings (generated
 * FP32 outputs; integral segment partials, min(256 MiB, budget/16)) and the caller's pinned
 * ring, harvests finished ticks and landed copies, and, with fewer than two ticks in flight,
 * packs one slice of every active request, oldest first and up to max_tick_events events, into
 * one hydra_batch_run.  A generate request is one slice; its [n][4][ld] FP32 outputs and ld
 * weights (ld = nevents rounded up to a multiple of 4) are copied to the pinned ring on a copy
 * stream that waits for the tick, and it completes when that copy has landed.  An integral
 * (FP32 kinematics) advances by int_slice_segments x 2^21 events per tick and completes with
 * its last slice.  A request that can never fit, or that cannot be admitted while nothing is
 * active or in flight, is refused.  Every slice computes exactly the events of the
 * single-request entry points (same seed, event offset 0).
 */
typedef struct hydra_server hydra_server; /* opaque; bound to the device current at creation */

typedef struct hydra_serve_request {
    double arrival;    /* seconds after the start of the run; requests sorted by arrival */
    int32_t kind;      /* HYDRA_REQ_GENERATE or HYDRA_REQ_INTEGRATE */
    int32_t n;         /* daughters, 2..10 */
    double M;
    double masses[10];
    uint64_t nevents;  /* > 0 */
    uint64_t seed;
    int32_t me;        /* integrate: hydra_me_id */
    int32_t reserved;
    double params[6];  /* integrate: matrix-element parameters */
    double withdraw;   /* seconds after the start of the run (live service: after submission) at which
                        * the client withdraws the request if it is admitted and not yet fully
                        * launched (dropped between ticks, memory released); negative: never */
} hydra_serve_request;

typedef enum hydra_serve_status {
    HYDRA_SERVE_DONE = 0,
    HYDRA_SERVE_REFUSED = 1,   /* could never fit, or could not be admitted with nothing in flight */
    HYDRA_SERVE_WITHDRAWN = 2, /* withdrawn by the client (see withdraw) */
    HYDRA_SERVE_INVALID = 3,   /* failed the checks of hydra_phsp_generate / hydra_phsp_integrate */
    HYDRA_SERVE_TIMED_OUT = 4  /* not finished when the run's deadline passed */
} hydra_serve_status;

typedef struct hydra_serve_outcome {
    double latency;        /* seconds from arrival to completion (HYDRA_SERVE_DONE) */
    uint64_t host_offset;  /* generate with kept outputs: byte offset of its block in the pinned
                            * ring ([n][4][ld] floats, then ld weights); otherwise all ones */
    uint64_t ld;
    hydra_integral result; /* integrate */
    int32_t status;        /* hydra_serve_status */
    int32_t reserved;
} hydra_serve_outcome;

/*
 * budget_bytes   device memory of the two rings (allocated here, >= 16 MiB)
 * pinned         caller-owned page-locked host ring of pinned_bytes (generated outputs)
 * max_slices     requests admitted at once (and slices per tick)
 * keep_outputs   != 0: a generate request's pinned block is kept (host_offset) instead of
 *                released when it completes
 * Errors: INVALID_ARG, OOM, CUDA.
 */
hydra_status hydra_server_create(uint64_t budget_bytes, void *pinned, uint64_t pinned_bytes, int max_slices,
                                 int int_slice_segments, uint64_t max_tick_events, int keep_outputs,
                                 hydra_server **out);

/*
 * Serve nreq requests (blocking: returns when every request has an outcome).  time_scale
 * stretches the arrival times (0: all arrive at once).  outcomes[i] receives request i's status,
 * latency and result: a request that fails the checks of the single-request entry points is
 * answered HYDRA_SERVE_INVALID when it arrives and the others are served as usual.  wall_s the
 * run's wall time, ticks the batch runs.  The loop makes the server's device current and
 * restores the caller's on return.  Errors: INVALID_ARG (unsorted requests), BUSY (the server is
 * serving live requests), TIMEOUT (the deadline of hydra_server_set_deadline passed: no further
 * tick was launched, the ticks in flight were waited for, and unfinished requests are answered
 * HYDRA_SERVE_TIMED_OUT), and the batch runner's errors.
 */
hydra_status hydra_server_run(hydra_server *server, const hydra_serve_request *reqs, int nreq, double time_scale,
                              hydra_serve_outcome *outcomes, double *wall_s, uint64_t *ticks);

/*
 * Wall-clock limit of a run (hydra_server_run, or a live service started afterwards) in
 * seconds from its start; 0 (the default) is no limit.  The loop never spins past it: it checks
 * the clock on every turn and ends the run with HYDRA_ERR_TIMEOUT.  Errors: INVALID_ARG, BUSY.
 */
hydra_status hydra_server_set_deadline(hydra_server *server, double seconds);

/*
 * Live service: requests pushed from any thread while the loop runs on a worker thread the
 * library starts (same policy, rings and results as hydra_server_run; the arrival time of a
 * request is the moment it is submitted, its withdraw field counts from there).
 *   hydra_server_start   start the worker (BUSY if already started).
 *   hydra_server_submit  check the request as the single-request entry points do (their
 *                        errors are returned at once) and queue it; *ticket identifies it
 *                        (BUSY when the server is not started or is stopping).
 *   hydra_server_poll    wait up to timeout_s seconds for the ticket's outcome (kept outputs
 *                        at host_offset of the pinned ring, as for hydra_server_run); each
 *                        outcome is returned once.  TIMEOUT if not finished in time;
 *                        INVALID_ARG for an unknown or already returned ticket.
 *   hydra_server_stop    stop accepting, let the worker finish what was submitted for up to
 *                        timeout_s seconds, then end it as a deadline does (ticks in flight
 *                        waited for, the rest answered HYDRA_SERVE_TIMED_OUT, TIMEOUT
 *                        returned) and join it.  hydra_server_destroy stops a live server with
 *                        timeout 0.
 */
hydra_status hydra_server_start(hydra_server *server);
hydra_status hydra_server_submit(hydra_server *server, const hydra_serve_request *req, uint64_t *ticket);
hydra_status hydra_server_poll(hydra_server *server, uint64_t ticket, double timeout_s, hydra_serve_outcome *outcome);
hydra_status hydra_server_stop(hydra_server *server, double timeout_s);

/* Wait for the server's work and release it (its rings, runners and streams). */
hydra_status hydra_server_destroy(hydra_server *server);

/*
 * Arithmetic of FP64 generation (HYDRA_F64 in hydra_phsp_generate, hydra_phsp_generate_host
 * and batched generation).  B300's FP64 pipe is a small fraction of its FP32 pipe, so by
 * default the kinematics run in double-float arithmetic (pairs of FP32 numbers, ~48
 * significand bits, error-free sums and products plus Newton-corrected reciprocal, square
 * root and sine/cosine) with FP64 weights and FP64 outputs; HYDRA_FP64_NATIVE uses FP64
 * instructions throughout.  Both agree with an FP64 reference to ~1e-14 of the event scale.
 * Process-wide.  Errors: INVALID_ARG.
 */
typedef enum hydra_fp64_arith {
    HYDRA_FP64_NATIVE = 0,
    HYDRA_FP64_DOUBLE_FLOAT = 1
} hydra_fp64_arith;

hydra_status hydra_set_fp64_arith(hydra_fp64_arith arith);
hydra_fp64_arith hydra_get_fp64_arith(void);

/*
 * Arithmetic of Kallen's lambda in FP32 generation (HYDRA_F32 in hydra_phsp_generate and
 * hydra_phsp_generate_host; section 4.2's two-body momenta p = sqrt(lambda) / (2 M)).  The
 * default evaluates lambda(M_{k+1}^2, M_k^2, m^2) as the product of its four gap factors
 * Delta (Delta + 2 m)(Delta + 2 M_k)(Delta + 2 M_k + 2 m) in FP32: every factor is a sum of
 * non-negative terms, so the product has no cancellation and carries at most a few FP32
 * roundings, also at threshold.  HYDRA_LAMBDA_F64 multiplies the same four factors in FP64
 * and rounds the product once (FP64 instructions on every two-body step; the FP32 generator
 * then runs several times slower on B300, whose FP64 pipe is narrow).  Process-wide; other
 * entry points are unaffected.  Errors: INVALID_ARG.
 */
typedef enum hydra_lambda_arith {
    HYDRA_LAMBDA_FACTORED_F32 = 0,
    HYDRA_LAMBDA_F64 = 1
} hydra_lambda_arith;

hydra_status hydra_set_fp32_lambda(hydra_lambda_arith arith);
hydra_lambda_arith hydra_get_fp32_lambda(void);

/*
 * Device ceilings for rooflines (no counterpart in the paper: these measure the GPU the
 * library runs on).  hydra_probe_fma_rate runs independent chains of FP32 or FP64 fused
 * multiply-adds in registers on every SM and returns the rate in FMA instructions per second
 * (FLOP/s = 2x; for FP32 this is also the SM instruction-issue limit, one warp instruction per
 * scheduler per clock).  hydra_probe_write_bandwidth writes the caller's device buffer with
 * 16-byte stores `reps` times at each of eight launch shapes (4..32 blocks of 256 threads per
 * SM, one or four stores in flight per thread) and returns the best write-only rate in GB/s
 * (use a buffer far larger than L2).  Both block until done; iterations scale the FMA probe's
 * duration.
 * Errors: INVALID_ARG, MISALIGNED (buffer not 16-byte aligned), OOM, CUDA.
 */
hydra_status hydra_probe_fma_rate(hydra_dtype dtype, int iterations, double *fma_per_s, hydra_stream_t stream);
hydra_status hydra_probe_write_bandwidth(void *buffer, uint64_t bytes, int reps, double *gb_per_s,
                                         hydra_stream_t stream);

/*
 * Rate of one arithmetic operation in the arithmetic a generator runs (no counterpart in the
 * paper: the floating-point ceiling of the generators' rooflines counts the method's
 * operations at these rates).  Independent chains of the operation, 8 per thread, 256-thread
 * blocks on every SM; returns operations per second (a fused multiply-add counts one).
 *   HYDRA_ARITH_F32            FP32 instructions; square root and reciprocal are the
 *                              hardware approximations the FP32 kernels use
 *   HYDRA_ARITH_DOUBLE_FLOAT   double-float pairs with the FP64 generator's own operations
 *                              (FMA = a double-float product then sum)
 *   HYDRA_ARITH_F64            FP64 instructions (IEEE square root and reciprocal)
 * Blocks until done.  Errors: INVALID_ARG (unknown arithmetic or operation, iterations < 1),
 * OOM, CUDA.
 */
typedef enum hydra_probe_arith {
    HYDRA_ARITH_F32 = 0,
    HYDRA_ARITH_DOUBLE_FLOAT = 1,
    HYDRA_ARITH_F64 = 2
} hydra_probe_arith;

typedef enum hydra_probe_op {
    HYDRA_OP_ADD = 0,
    HYDRA_OP_MUL = 1,
    HYDRA_OP_FMA = 2,
    HYDRA_OP_SQRT = 3,
    HYDRA_OP_RCP = 4
} hydra_probe_op;

hydra_status hydra_probe_op_rate(hydra_probe_arith arith, hydra_probe_op op, int iterations, double *ops_per_s,
                                 hydra_stream_t stream);

/* Release the per-device scratch memory of the library (all devices).  Not thread safe
 * with respect to calls in flight. */
hydra_status hydra_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* HYDRA_PHSP_H */
