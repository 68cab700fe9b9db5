// cwb_internal.cuh -- shared declarations of the sm_103a componentwise boosting library.
//
// Device memory layout of one model (all owned by cwb_model, freed by cwb_free):
//   ind      [B][n_pad]   uint8 or uint16 index vectors, one row per binning (learners on the
//                         same feature with the same n_bins share a binning), rows train-first
//   y, w     [n_pad]      FP32 targets and weights (w omitted when all ones); y_lo holds the
//                         low part of FP64 targets
//   f, h     [n_pad][2]   primary and momentum model as compensated FP32 pairs (hi, lo)
//   c        [n_pad]      FP32 error-corrected residual (ACWB)
//   rw       [2][n_pad]   FP32 scatter inputs w*r (channel 0) and w*c (channel 1), zero past
//                         the active rows
//   zb       [K][S][4]    FP32 non-zero basis values at the design points (S = max n*)
//   zcol     [K][S]       int32 first non-zero column of each design point
//   crange   [K][D][2]    int32 contiguous bin range contributing to each column
//   ztab     [K][4 S]     FP32 the same design stored column by column (toff: column offsets)
//   G, P     [2][K][D][D] FP64 Gram matrix and cached inverse per phase
//   part     per-cluster histogram partials written by the scatter kernel
//   u        [2][B][S]    histograms per binning (binMatVec intermediate u)
//   trace    per iteration: mode, selected learners, FP64 fits, criteria
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "cwb.h"

namespace cwb {

constexpr int kMaxD = CWB_MAX_D;
constexpr int kMaxNnz = 4;              // degree <= 3
constexpr int kNumPhases = 2;
constexpr int kRowAlign = 256;          // n_pad multiple (elements)

// Error bits written by kernels into DevState::err.
enum : uint32_t {
    kErrTimeout = 1u,      // a bounded device wait ran out
    kErrNumeric = 2u,      // factorisation failed / df not reachable
    kErrIndex = 4u,        // an index fell outside its table (should never happen)
    kErrNonFinite = 8u,    // non-finite criterion
    kErrBound = 16u,       // a residual above the bound that set its fixed-point scale (should never happen)
};

enum : int32_t { kModeCWB = 0, kModeACWB = 1 };

// Iteration state kept on the device; every kernel reads it, only last blocks write it.
struct DevState {
    int32_t m;            // iterations whose fits are computed
    int32_t m_applied;    // iterations whose updates have been applied to f (and h)
    int32_t mode;         // mode of iteration m+1
    int32_t phase;        // cache used by CWB iterations (1 after an HCWB switch)
    int32_t counter;      // HCWB patience counter
    int32_t switch_iter;  // first CWB iteration of HCWB (1-based), 0 if none
    int32_t pend_mode;    // mode of iteration m (the one whose update may be pending)
    int32_t k_sel;        // learner of iteration m's primary fit
    int32_t k_cor;        // learner of iteration m's correction fit (ACWB)
    int32_t risk_valid;   // risk_prev holds a value
    uint32_t err;
    uint32_t ticket_rows;
    uint32_t ticket_solve;
    uint32_t pad0;
    double risk_prev;
    uint32_t rmax_bits[2];  // max |w r| and max |w c| of the current iteration (FP32 bits): atomicMax by the
                            // row pass, reset to 0 by the solve's last block
    int32_t cnt_log2[2];    // ceil(log2(largest per-cluster bin count)): [0] all rows, [1] HCWB training rows
    int32_t cnt_max[2];     // largest per-cluster bin count of the counting passes ([1]: persistent plan)
    uint32_t rprev_bits;    // max |w r| of the most recently computed residuals (FP32 bits)
    int32_t cnt_log2p;      // ceil(log2(largest per-CTA bin count)) of the persistent plan
    int32_t fix_exp;        // fixed-point exponent of the residuals the persistent path wrote last
    int32_t resid_path;     // 0: the latest residuals are FP32 in rw, 1: fixed point in rq (persistent path)
    int32_t resid_stale;    // HCWB: the row pass switched to CWB after computing ACWB residuals; the
                            // residual pass that follows it recomputes them for the CWB iteration
};

// How cwb_fit runs iterations: auto picks the persistent kernel when the model qualifies.
enum : int { kIterAuto = 0, kIterKernels = 1, kIterPersistent = 2 };

// Decomposition of the persistent iteration kernel (cwb_persist.cu).
struct PersistPlan {
    int FE, G, per_group, stages, nb, ctas;
    int64_t tiles;
    uint32_t ring_off, stage_stride;                           // ring of stages
    uint32_t f_off, y_off, sel_off, w_off, ylo_off, q_off;     // offsets within a stage (after the index box)
    uint32_t hist_off, vtab_off;
    size_t smem;
};

// Static description of the scatter decomposition (see k_scatter).
struct ScatterPlan {
    int f_lane;       // binnings side by side in a warp (lane-private histogram columns)
    int groups;       // ceil(B / f_lane)
    int fe;           // binnings per group actually streamed (balanced, <= f_lane)
    int bin_ranges;   // bin sub-ranges (only when one binning's bins do not fit shared memory)
    int nb_cta;       // bins held by one CTA
    int nbins_pad;    // bin_ranges * nb_cta (>= max n*)
    int ch_stride;    // shared-memory floats between the two channels' histograms
    int cmax;         // 1 (CWB) or 2 (ACWB/HCWB: residual and error-corrected residual)
    int cs;           // thread-block cluster size
    int clusters;     // clusters in the grid
    int slots;        // groups * bin_ranges
    int stages, nb_box, box_bytes, stage_rows;
    uint32_t ind_off, r_off, q_off, hist_off, bar_off, stage_ind_bytes, stage_r_bytes;
    int threads;
    size_t smem;      // dynamic shared memory bytes (incl. alignment slack)
    size_t part_floats;
    int stage_cb;     // bins per chunk of the cluster epilogue's transposing stage
    int active_ctas[4];  // resident scatter CTAs for cluster sizes 1, 2, 4, 8
    bool solve_stage_v;  // the solve stages each learner's design rows in shared memory
    bool solve_stage_z;  // ... and its column-major design
    bool int_acc;     // exact fixed-point int32 histograms (false: FP32 atomics for heavily skewed bins)
};

struct HostBinning {
    int feature;
    int nbins_spec;      // n_bins code requested
    int categories;      // > 0: categorical codes 0..categories-1, one design point per class
    int nstar;
    int exact;
    double xmin, xmax;
};

struct HostLearner {
    cwb_learner spec;
    int binning;
    int d;
    int nnz;
};

}  // namespace cwb

struct cwb_model {
    int device = 0;
    cudaStream_t stream = nullptr;        // work stream (user's or owned)
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr;
    cwb_config cfg{};
    int64_t n = 0, n_tr = 0, n_pad = 0;
    int32_t p = 0, K = 0, B = 0;
    bool hybrid = false, accel = false, weighted = false;
    int ind_bytes = 2;
    int d_max = 0, nstar_max = 0;
    double offset = 0.0;
    std::vector<cwb::HostBinning> bins;
    std::vector<cwb::HostLearner> lrn;
    cwb::ScatterPlan plan{};

    // device buffers
    void* ind = nullptr;
    float *y = nullptr, *y_lo = nullptr, *w = nullptr, *c = nullptr, *rw = nullptr;
    float *f = nullptr, *h = nullptr;     // [n_pad][2]: compensated hi, lo
    int32_t* perm = nullptr;              // new row -> original row (HCWB)
    float* zb = nullptr;
    double* zb64 = nullptr;
    int32_t* zcol = nullptr;
    int32_t* crange = nullptr;
    int32_t* toff = nullptr;              // [K][D] offset of column j in ztab
    float* ztab = nullptr;                // [K][4 S] column-major reduced design
    double *G = nullptr, *P = nullptr, *lambda = nullptr;
    double* Acrit = nullptr;              // [2][K][D][D] criterion matrix P G P - 2 P
    float2* Pdf = nullptr;                // [2][K][D][D] P as float-float pairs (hi, lo) for the solve
    float2* Adf = nullptr;                // [2][K][D][D] Acrit as float-float pairs
    int32_t *l_bin = nullptr, *l_d = nullptr, *l_nstar = nullptr, *l_type = nullptr;
    double *l_xmin = nullptr, *l_xmax = nullptr;
    int32_t *l_degree = nullptr, *l_nknots = nullptr, *l_feat = nullptr;   // l_degree: the class of a binary learner
    float* part = nullptr;                // [clusters][cmax][f_lane][nb_cta] per-cluster histograms
    int32_t* cluster_slot = nullptr;      // [clusters]
    int32_t* slot_c0 = nullptr;           // [slots + 1]
    CUtensorMap tmap;                     // 2D map of the index matrix [B][n_pad]
    double* theta_it = nullptr;           // [2][K][D]
    double* q_it = nullptr;               // [2][K]
    float* v = nullptr;                   // [2][K][S] fitted values Z^b theta of every learner per bin
    cwb::DevState* state = nullptr;
    double* risk_part = nullptr;
    int risk_blocks = 0;
    // trace
    int32_t trace_cap = 0;
    int32_t* tr_k = nullptr;              // [cap][2]
    int32_t* tr_mode = nullptr;           // [cap]
    double* tr_theta = nullptr;           // [cap][2][D]
    double* tr_q = nullptr;               // [cap][2]
    int32_t* forced = nullptr;            // [cap]
    double* coef = nullptr;               // [2][K][D] aggregated
    int32_t coef_valid_at = -1;
    int32_t done = 0;                     // iterations queued so far
    std::vector<int32_t> forced_host;     // pending host-side forced selections
    bool update_pending = false;          // the last iteration's update is not yet applied to f
    // per-kernel timing (cwb_profile): bit c of prof_mask brackets kernel class c
    bool prof_on = false;
    int prof_mask = 0;
    cudaEvent_t prof_ph[8] = {};          // placeholder events of the profiling graph
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t prof_launches[4] = {0, 0, 0, 0};
    // CUDA graphs: a block of kGraphIters iterations and a single iteration; the
    // profiling graph of one iteration carries event-record nodes around the
    // profiled kernels (their events are swapped before every launch)
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphExec_t graph1_exec = nullptr;
    cudaGraphExec_t prof_exec = nullptr;
    cudaGraph_t prof_graph = nullptr;     // kept alive: its event-record nodes address the exec's nodes
    std::vector<std::pair<int, std::pair<cudaGraphNode_t, cudaGraphNode_t>>> prof_nodes;
    int graph_iters = 0;
    bool graph_valid_for_batch = false;   // set by a batch capture, cleared when buffers or plans change
    bool use_pdl = true;                  // launch the iteration kernels with programmatic dependencies
    // persistent iteration kernel (plain CWB): plan, tensor map and buffers
    int iter_mode = cwb::kIterAuto;
    bool persist_ok = false;
    cwb::PersistPlan pplan{};
    CUtensorMap pmap;
    float* f2 = nullptr;                  // [n_pad][2] second f buffer (the persistent kernel alternates)
    long long* uacc = nullptr;            // [2][nb][B] exact histogram sums (bin-major)
    bool uacc_clean = true;               // both parities of uacc are zero
    unsigned* gbar = nullptr;             // barrier words, the two residual maxima, one arrival flag per CTA
    long long* ptime = nullptr;           // [4] phase times and iteration count (profiling)
    float* ztab_lo = nullptr;             // [K][4 S] low parts of the column-major design
    float* vmax = nullptr;                // [K] max |v_k| of the latest update tables
    double wmax = 1.0;                    // largest observation weight
    bool direct_enabled = true;           // CWB_DIRECT_Q=0 turns the direct fixed-point residuals off
    int sleep_waits = -1;                 // CWB_SLEEP_WAITS: 1 / 0 forces the scatter's suspend-time hint on / off
    long long wait_cycles = 4000000000LL; // limit of each device-side ring wait (SM clocks, ~2 s)
    int withhold_tile = -1;               // test hook (CWB_WITHHOLD_TILE): a scatter tile whose copies are never issued
    // row shards (cwb_shard_*): global binning ranges and row count, exchanged histogram sums
    bool shard = false;
    int64_t shard_n_global = 0;
    std::vector<double> shard_xmin, shard_xmax;   // per feature
    long long* u_shard = nullptr;         // [B][S] exact histogram sums (local, then the exchanged total)
    const long long* solve_u64 = nullptr; // set while a shard's solve is queued
};

namespace cwb {

// Error plumbing (thread-local message).
void set_error(const std::string& msg);
cwb_status cuda_status(cudaError_t e, const char* what);

#define CWB_CUDA_TRY(expr)                                                 \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return ::cwb::cuda_status(_e, #expr);       \
    } while (0)

#define CWB_TRY(expr)                                                      \
    do {                                                                   \
        cwb_status _s = (expr);                                            \
        if (_s != CWB_OK) return _s;                                       \
    } while (0)

cwb_status dev_alloc(void** p, size_t bytes, cudaStream_t s);

// Raises a kernel's dynamic shared-memory cap to the most the device allows next to the kernel's
// static shared memory.  The cap is per kernel and process-wide, while models need different amounts.
inline cudaError_t allow_max_dynamic_smem(const void* func, int device)
{
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}
void dev_free(void* p);

// Setup (cwb_setup.cu)
cwb_status setup_model(cwb_model* m, const void* X, int x_dtype, const void* y, const double* w,
                       const uint8_t* val_mask, int device_ptrs);

// Iterations (cwb_iter.cu)
cwb_status plan_scatter(cwb_model* m, int max_ctas = 0, int cs_req = 0);
void release_scatter_plan(cwb_model* m);
cwb_status autotune_scatter(cwb_model* m, int objective, int trials, double* best_us);
cwb_status scatter_count_pass(cwb_model* m);
cwb_status ensure_trace(cwb_model* m, int32_t cap);
cwb_status launch_iterations(cwb_model* m, int32_t iters);
cwb_status prepare_launch(cwb_model* m, int32_t iters);
void note_iterations_queued(cwb_model* m, int32_t iters);
void enqueue_iteration(cwb_model* m, cudaStream_t s, int mask);
cwb_status launch_final_update(cwb_model* m);
cwb_status materialize(cwb_model* m);
void release_graphs(cwb_model* m);
cwb_status launch_initial_rows(cwb_model* m);
cwb_status launch_aggregate(cwb_model* m);
cwb_status read_device_error(cwb_model* m);
cwb_status profile_collect(cwb_model* m);
void profile_release(cwb_model* m);

// Row shards (cwb_setup.cu, cwb_iter.cu)
cwb_status build_caches(cwb_model* m, const double* cnt, int phases);
cwb_status shard_stats(cwb_model* m, double* counts_h, double sums_h[2], int32_t* cnt_log2);
cwb_status shard_finish(cwb_model* m, const double* counts_h, const double sums_h[2], int32_t cnt_log2);
cwb_status shard_rows(cwb_model* m, float* rmax, int device_ptrs);
cwb_status shard_scatter(cwb_model* m, const float* rmax, int rmax_device, long long* u, int u_device);
cwb_status shard_solve(cwb_model* m, const long long* u, int device_ptrs);

// Persistent iteration kernel (cwb_persist.cu)
cwb_status plan_persistent(cwb_model* m);
cwb_status init_residual_bound(cwb_model* m);

// Plain CWB with exact fixed-point histograms: the row pass writes the residuals as int32 fixed
// point with a scale from residual_bound (known before the pass), so the scatter needs no conversion
// step.  Accelerated, hybrid and sharded models and the persistent path keep the converter.
inline bool direct_q(const cwb_model* m)
{
    return !m->accel && !m->hybrid && !m->shard && m->plan.int_acc && m->direct_enabled &&
           m->iter_mode != kIterPersistent;
}
cwb_status launch_persistent(cwb_model* m, int32_t iters);
cwb_status persistent_profile(cwb_model* m, double ms[3], int64_t* iters, bool reset);
cwb_status persistent_residuals(cwb_model* m, float* out_dev);

// Model creation with an explicit iteration mode (kIterAuto, kIterKernels, kIterPersistent) and,
// when the model creates its own stream, that stream's priority (0: the default)
cwb_status create_model(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p, const void* y,
                        const double* w, const cwb_learner* bl, int32_t K, int32_t device_ptrs, cwb_model** out,
                        int iter_mode, int stream_priority = 0);

// Predict / fitted (cwb_api.cu)
cwb_status launch_predict(const cwb_model* m, const void* Xnew, int x_dtype, int64_t n_new, float* out_dev);

}  // namespace cwb
