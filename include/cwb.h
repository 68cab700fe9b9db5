/*
 * cwb.h -- C ABI of the GB300 (sm_103a) componentwise boosting library.
 *
 * The library fits additive models by componentwise gradient boosting on
 * binned numerical features (Schalk, Bischl, Ruegamer, arXiv 2110.03513):
 *
 *   CWB   App. A.1, Algorithm 1  -- every base learner is fitted to the pseudo
 *         residuals, the one with the smallest SSE updates the model;
 *   ACWB  Sec. 3.2, Algorithm 3  -- Nesterov momentum: a primary model f, a
 *         momentum model h and a second (error-corrected) fit per iteration;
 *   HCWB  Sec. 3.2.3, Algorithm 4 -- ACWB on training rows until the validation
 *         risk stops improving for `patience` iterations, then CWB on all rows.
 *
 * Each base learner is univariate (Sec. 2.2): a cubic P-spline (B-spline basis
 * with a difference penalty, App. A.2) or a linear learner (1, x).  Features
 * are discretised per learner into n* design points with an index vector
 * (Sec. 3.1.1); every iteration computes Z_k^T W r through the index vector
 * (binMatVec, Algorithm 2) and solves with the cached (Z_k^T W Z_k + lambda K)^-1.
 *
 * Conventions for every entry point:
 *  - Matrices of observations are feature-major (column-major): X[j * n + i]
 *    is feature j of row i.
 *  - `device_ptrs` = 0: pointer arguments are host memory; = 1: they are
 *    device memory on the model's device (CUDA global memory).  Host buffers
 *    may be pageable or pinned.
 *  - Output buffers are allocated by the caller.
 *  - Nothing crosses the ABI as an exception; every failure returns a
 *    cwb_status and leaves a message readable through cwb_last_error() on the
 *    calling thread.  CUDA errors are reported as CWB_ECUDA.
 *  - A model is not thread-safe: calls on one model must not overlap.
 *    Different models may be used from different threads.
 *  - Work is issued on the model's stream (cwb_config.stream).  Calls that
 *    return host data synchronise that stream; cwb_fit does not, unless a
 *    device-side error has to be read back (see cwb_fit).
 */
#ifndef CWB_H
#define CWB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cwb_model cwb_model;   /* opaque; owns all device state of one fit */

typedef enum {
    CWB_OK = 0,
    CWB_EINVAL = 1,     /* invalid argument or unsupported combination */
    CWB_ENOMEM = 2,     /* device or host allocation failed */
    CWB_ECUDA = 3,      /* a CUDA call failed */
    CWB_ENUMERIC = 4,   /* a factorisation failed or df cannot be reached */
    CWB_ETIMEOUT = 5,   /* a device-side wait ran out (the kernel returned early) */
    CWB_ESTATE = 6      /* call not valid in the model's current state */
} cwb_status;

typedef enum { CWB_LOSS_L2 = 0, CWB_LOSS_BINOMIAL = 1 } cwb_loss;
typedef enum { CWB_OPT_CWB = 0, CWB_OPT_ACWB = 1, CWB_OPT_HCWB = 2 } cwb_optimizer;
typedef enum {
    CWB_BL_PSPLINE = 0,             /* P-spline (Sec. 2.2) */
    CWB_BL_LINEAR = 1,              /* linear effect (1, x) */
    CWB_BL_CATEGORICAL = 2,         /* ridge representation of a categorical feature (App. B.1) */
    CWB_BL_CATEGORICAL_BINARY = 3   /* sparse binary representation: one class of a categorical feature */
} cwb_bl_type;
typedef enum { CWB_F32 = 0, CWB_F64 = 1 } cwb_dtype;

/* n_bins codes (cwb_learner.n_bins) */
#define CWB_BINS_EXACT 0     /* design points = the sorted unique values of the feature */
#define CWB_BINS_SQRT (-1)   /* n* = floor(sqrt(n)) equidistant design points (Sec. 3.1.1) */

/* Limits */
#define CWB_MAX_D 64          /* basis dimension per learner */
#define CWB_MAX_BINS 65535    /* design points per learner (uint16 index vector) */

/*
 * One univariate base learner (Sec. 2.2; categorical learners App. B.1).
 *
 * Categorical learners read their feature as class codes: every value must be an
 * integer in [0, c) with c = n_knots (CWB_EINVAL otherwise).  Each class is one
 * design point, so the lookup k_i is the code itself and n_bins is ignored.  The
 * ridge learner has d = c coefficients, the dummy design and the identity penalty
 * (so (Z^T W Z + lambda I) is diagonal with the class weights n_k + lambda, and
 * df1 = sum_k n_k / (n_k + lambda)); c <= CWB_MAX_D.  The binary learner has one
 * unpenalised coefficient for the class `level` (its class mean); c <= CWB_MAX_BINS.
 * Learners of either kind on the same feature with the same c share one binning,
 * i.e. one histogram per iteration.  Prediction maps any value that is not a valid
 * code to a zero contribution.
 */
typedef struct {
    int32_t type;        /* cwb_bl_type */
    int32_t feature;     /* column of X, 0 <= feature < p */
    int32_t degree;      /* B-spline degree, 0..3 (P-spline only; 3 = cubic) */
    int32_t n_knots;     /* P-spline: interior equidistant knots, d = n_knots + degree + 1;
                            categorical: number of classes c >= 2 */
    int32_t diff_order;  /* order of the difference penalty, 1 <= diff_order < d (P-spline only) */
    double df;           /* > 0: lambda is chosen so that tr(H_k) = df (App. A.2, Eq. df1) */
    double lambda;       /* used when df <= 0 (P-spline, categorical ridge); linear and binary
                            learners are unpenalised */
    int32_t n_bins;      /* CWB_BINS_EXACT, CWB_BINS_SQRT, or an explicit n* >= 2 (numeric learners) */
    int32_t level;       /* categorical binary: the class it indicates, 0 <= level < n_knots */
} cwb_learner;

/* Optimiser settings (Algorithm 1, 3, 4 inputs). */
typedef struct {
    int32_t loss;              /* cwb_loss; binomial needs y in {0, 1} */
    int32_t opt;               /* cwb_optimizer */
    double nu;                 /* learning rate nu > 0 */
    double gamma;              /* momentum parameter gamma >= 0 (ACWB/HCWB) */
    int32_t iterations;        /* default M for cwb_fit(model, 0) */
    int32_t patience;          /* pat_0 >= 0 (HCWB) */
    const uint8_t* val_mask;   /* HCWB: n entries, 1 = validation row; same memory kind as X */
    void* stream;              /* cudaStream_t to issue work on; NULL: the model creates and owns a stream */
    int32_t device;            /* CUDA device ordinal; -1 = the calling thread's current device */
} cwb_config;

/* Per-learner description after setup. */
typedef struct {
    int32_t d;            /* basis dimension */
    int32_t nstar;        /* number of design points n* */
    int32_t binning;      /* index of the shared binning (learners on the same feature and n_bins share one) */
    int32_t reserved;
    double xmin, xmax;    /* training range of the feature */
    double lambda;        /* smoothing parameter of the first phase (train rows for HCWB) */
    double lambda_full;   /* smoothing parameter on all rows (HCWB second phase; = lambda otherwise) */
} cwb_learner_info;

/*
 * cwb_create -- set up a model: copy and bin the data, build the reduced designs,
 * choose lambda per learner from its df and cache the inverse of
 * Z_k^T W Z_k + lambda K_k (Sec. 2.4, Sec. 3.1.2: factorise once before boosting).
 *
 *   cfg         optimiser settings (copied; the val_mask is read during the call only)
 *   X           p x n feature-major observations, dtype x_dtype (CWB_F32 or CWB_F64)
 *   n, p        rows (>= 2) and features (>= 1)
 *   y           n targets, same dtype as X
 *   w           n observation weights (> 0) in FP64, or NULL for w = 1 (App. A.2, W_k = diag(w))
 *   bl, K       K >= 1 base learners
 *   device_ptrs 0: X, y, w, val_mask are host pointers; 1: device pointers.  Either way
 *               the model keeps its own copies; the caller's buffers are only read
 *               during this call.
 *   out         receives the new model (NULL on failure)
 *
 * Errors: CWB_EINVAL for bad sizes, non-finite features or targets, a constant feature (max == min), n* outside
 * [2, 65535], d > CWB_MAX_D, binomial targets outside {0, 1}, a categorical feature
 * holding a value that is not a class code 0..c-1, or HCWB without a validation mask
 * holding at least one training and one validation row;
 * CWB_ENUMERIC if a Gram matrix is singular or df is not reachable;
 * CWB_ENOMEM / CWB_ECUDA on device failures.
 */
cwb_status cwb_create(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p,
                      const void* y, const double* w, const cwb_learner* bl, int32_t K,
                      int32_t device_ptrs, cwb_model** out);

/*
 * cwb_create_many -- the setup of many fits at once (Sec. 2.4 and Sec. 3.1.2: binning, bin counts,
 * Z^T W Z, df -> lambda and the factorisations are computed once, before boosting).  Request i holds
 * the arguments of one cwb_create call; `threads` host threads (<= 0: up to 16) create the models
 * concurrently, each on its own stream (cfg.stream is honoured when set), so the setup kernels and the
 * host-side steps of different fits overlap on the GPU.  Each model equals the one cwb_create would
 * return for the same request.  out[i] receives model i (NULL if its creation failed); status[i]
 * (nullable) its status.  Returns CWB_OK when every request succeeded, else the status of the first
 * failing request (its message names the request index).  device_ptrs applies to every request.
 */
typedef struct {
    cwb_config cfg;
    const void* X;          /* p x n features, as in cwb_create */
    int32_t x_dtype;
    int64_t n;
    int32_t p;
    const void* y;
    const double* w;        /* nullable */
    const cwb_learner* bl;
    int32_t K;
} cwb_fit_request;
cwb_status cwb_create_many(const cwb_fit_request* reqs, int32_t count, int32_t device_ptrs, int32_t threads,
                           cwb_model** out, cwb_status* status);

/*
 * cwb_fit -- run `iterations` boosting iterations (<= 0: cfg.iterations) on the
 * device, continuing from the model's current state (fits are resumable).  One
 * iteration is: pseudo residuals, binMatVec scatter of W r into every binning's
 * histogram (Algorithm 2), Z^T u, theta = P (Z^T u), the SSE criterion, argmin
 * over learners and the update f += nu Z_k theta_k (Algorithm 1; Algorithm 3 for
 * ACWB with two fits per iteration).  No host synchronisation happens between
 * iterations; the call returns once the work is queued on the model's stream
 * (as CUDA graphs).  The update of the last iteration is folded into the next
 * iteration's row pass; calls that read the fitted values, the trace or the
 * coefficients apply it first.  A device-side wait that ran out is reported by
 * the next call that synchronises, as CWB_ETIMEOUT (the kernel that waited has
 * returned; the model's state is then undefined, other models are unaffected);
 * a non-finite residual or criterion (a diverging fit), or a residual above the
 * bound of its fixed-point scale (which the bound rules out), as CWB_ENUMERIC.  The
 * limit of the waits is about two seconds; the environment variable
 * CWB_WAIT_CYCLES, read when a model is created, sets it in SM clock cycles.
 */
cwb_status cwb_fit(cwb_model* m, int32_t iterations);

/*
 * cwb_predict -- evaluate offset + sum_k g_k(x)^T theta_k (primary model, aggregated
 * parameters; Sec. 2.3, Sec. 3.2.1) at n_new new rows.  Xnew is p x n_new
 * feature-major (dtype x_dtype); values are clamped to each learner's training
 * range.  `out` receives n_new FP32 predictions on the link scale.  Memory kind of
 * Xnew and out follows device_ptrs.  Synchronises the model's stream.
 */
cwb_status cwb_predict(const cwb_model* m, const void* Xnew, int32_t x_dtype, int64_t n_new, float* out,
                       int32_t device_ptrs);

/*
 * cwb_get_coefficients -- aggregated parameters of learner k (eq. (1) additivity;
 * Sec. 3.2.1 for ACWB/HCWB).  which = 0: primary model theta_f; which = 1: momentum
 * model theta_h (zeros for CWB).  theta receives min(d_k, cap) FP64 values (host
 * memory); *offset (nullable) receives the constant initial model.
 */
cwb_status cwb_get_coefficients(const cwb_model* m, int32_t k, int32_t which, double* theta, int32_t cap,
                                double* offset);

/*
 * cwb_get_trace -- selected learners per iteration (0-based), host memory.
 * k_sel[t] for t < min(cap, done); k_cor (nullable) the correction learner of
 * ACWB iterations, -1 for CWB iterations; *switch_iter (nullable) the first CWB
 * iteration of HCWB (1-based) or 0; *done (nullable) iterations run so far.
 */
cwb_status cwb_get_trace(const cwb_model* m, int32_t* k_sel, int32_t* k_cor, int32_t cap, int32_t* switch_iter,
                         int32_t* done);

/*
 * cwb_get_criteria -- per iteration t < min(cap, done), the best and second-best
 * value of Q_k = theta^T G theta - 2 theta^T s (SSE_k minus the common r^T W r)
 * of the primary fit, FP64, host memory.  For checking near ties.
 */
cwb_status cwb_get_criteria(const cwb_model* m, double* q_best, double* q_second, int32_t cap);

/*
 * cwb_get_fitted -- the primary model at the n training rows (original row order),
 * FP32, memory kind per device_ptrs.  Synchronises the model's stream.
 */
cwb_status cwb_get_fitted(const cwb_model* m, float* f, int32_t device_ptrs);

/* cwb_get_learner_info -- setup results of learner k. */
cwb_status cwb_get_learner_info(const cwb_model* m, int32_t k, cwb_learner_info* info);

/*
 * cwb_get_learner_matrices -- FP64 d x d row-major G = Z^T W Z and P = (G + lambda K)^-1
 * of learner k for phase 0 (first phase) or 1 (all rows, HCWB).  Either pointer may be NULL.
 */
cwb_status cwb_get_learner_matrices(const cwb_model* m, int32_t k, int32_t phase, double* G, double* P);

/* cwb_get_bin_index -- index vector of learner k (n entries, original row order, 0-based), host int32. */
cwb_status cwb_get_bin_index(const cwb_model* m, int32_t k, int32_t* ind);

/*
 * cwb_force_selection -- testing hook: for the next `count` iterations the primary
 * learner is `k_forced[t]` instead of the argmin (k_forced host int32, -1 = no
 * override).  Used to keep comparing against the FP64 oracle past a near tie.
 */
cwb_status cwb_force_selection(cwb_model* m, const int32_t* k_forced, int32_t count);

/*
 * cwb_profile -- per-kernel timing.  `enable` = 0 switches it off, CWB_PROF_ALL
 * brackets every kernel class, otherwise an OR of CWB_PROF_ROWS, CWB_PROF_SCATTER
 * and CWB_PROF_SOLVE selects the classes.  While enabled, iterations are launched
 * one by one from a one-iteration CUDA graph whose event-record nodes (CUDA events
 * on the model's stream) bracket the selected kernels; unselected kernels run
 * without events between them.  Changing the setting clears the accumulated figures.
 */
#define CWB_PROF_ALL 1
#define CWB_PROF_ROWS 0x10
#define CWB_PROF_SCATTER 0x20
#define CWB_PROF_SOLVE 0x40
cwb_status cwb_profile(cwb_model* m, int32_t enable);

/*
 * cwb_get_profile -- accumulated device time (ms) and launch counts per kernel
 * class since profiling was enabled: index 0 = row pass (update / pseudo
 * residuals), 1 = binMatVec scatter, 2 = per-learner solve (sum of the cluster
 * partial histograms, Z^T u, theta, criterion, update table, argmin), 3 = reserved
 * (always 0).  `ms` and `launches` hold `cap` entries (host memory, either may be
 * NULL).  Synchronises the model's stream.
 */
cwb_status cwb_get_profile(cwb_model* m, double* ms, int64_t* launches, int32_t cap);

/*
 * cwb_get_residuals -- the scatter input of the most recent iteration, in the
 * caller's row order: channel 0 = w * r (pseudo residuals), channel 1 = w * c
 * (error-corrected residuals, ACWB/HCWB).  Rows outside the fitting set of that
 * iteration read 0.  `out` holds n FP32 values in host memory.
 */
cwb_status cwb_get_residuals(const cwb_model* m, int32_t channel, float* out);

/*
 * cwb_get_scatter_plan -- the decomposition chosen for the binMatVec scatter, for
 * tuning and reports.  values (host int32, `cap` entries) receive in order:
 * binnings per warp (lane-private columns), binnings per group, groups, bin ranges,
 * bins per CTA, cluster size, clusters, pipeline stages, threads per CTA,
 * dynamic shared memory bytes, 1 if histograms use exact int32 fixed point,
 * then the scatter CTAs that can be resident at cluster sizes 1, 2, 4 and 8,
 * then 1 if cwb_fit runs the model's iterations as one persistent kernel (see
 * CWB_ITER_MODE below), that kernel's ring stages, CTAs and shared memory bytes.
 * The cluster size is the largest that keeps nearly every SM busy; the
 * environment variable CWB_CLUSTER_SIZE (1, 2, 4, 8 or 16), read when a model is
 * created, overrides it when that size can be resident.  CWB_F_LANE (a power of
 * two), read likewise, caps the binnings side by side in a warp.
 *
 * CWB_ITER_MODE, read when a model is created: unset or "kernels" runs every
 * iteration as three kernels (pseudo residuals, binMatVec scatter, solve with the
 * argmin) launched from CUDA graphs; "persistent" runs plain CWB models (one
 * residual channel, histograms that fit one CTA) as one cooperative kernel per
 * cwb_fit call with grid-wide barriers between the phases of an iteration
 * (cwb_create fails with CWB_EINVAL for a model that does not qualify).  Both
 * compute the same iteration; results agree within the oracle tolerances.
 *
 * In the three-kernel path, plain CWB models with fixed-point histograms have
 * the row pass write the residuals as int32 fixed point directly, at a scale set
 * by a bound on max |w r| known before the pass (the previous maximum plus the
 * pending update's largest step; max w for the binomial loss), so the scatter
 * needs no conversion step.  CWB_DIRECT_Q=0, read when a model is created, keeps
 * the conversion inside the scatter (scale from the measured maximum) instead.
 * The scatter's ring waits sleep with a suspend-time hint when its ring has six or
 * more stages; CWB_SLEEP_WAITS=1 or 0, read when a model is created, forces the
 * hint on or off.
 */
cwb_status cwb_get_scatter_plan(const cwb_model* m, int32_t* values, int32_t cap);

/*
 * cwb_predict_noalloc -- cwb_predict for host buffers that performs no device
 * memory allocation.  (The paper has no counterpart; this is a deployment aid.)
 *
 * Some callers cannot allocate device memory at prediction time: real-time
 * serving loops, where cudaMalloc can stall on the driver's allocator and
 * cudaFree waits for all work on the device; and processes whose device memory
 * is handed out by another framework's allocator under a fixed budget, where an
 * allocation made behind that allocator's back can fail or push the process
 * over its budget.  cwb_predict copies host inputs into freshly allocated device
 * buffers; this entry point instead stages Xnew and the predictions through one
 * fixed scratch array of CWB_NOALLOC_SCRATCH_BYTES (16 MiB) that the library
 * declares at file scope in device memory.  Every GPU that loads the library
 * holds that array until the process exits.
 *
 *   Xnew   host, p x n_new feature-major, dtype x_dtype (CWB_F32 or CWB_F64)
 *   out    host, n_new FP32 predictions (same values as cwb_predict)
 *
 * Size limit: the Xnew bytes rounded up to 256, plus 4 * n_new bytes, must fit
 * in CWB_NOALLOC_SCRATCH_BYTES; larger requests (however large n_new is) fail
 * with CWB_EINVAL before any device work, with a message naming the limit
 * (split the rows into several calls).
 * The first call on a device looks up the scratch array's device address with
 * that device current (no allocation); make that first call before any stream
 * capture begins.  All calls in the process share the one array and it keeps the
 * previous call's contents; nothing in it needs to start at zero because every
 * byte read is written earlier in the same call.  Calls that overlap on the GPU
 * (different threads or streams, even on different models) race on the array:
 * serialise them.  Synchronises the model's stream before returning.
 */
#define CWB_NOALLOC_SCRATCH_BYTES (16u << 20)
cwb_status cwb_predict_noalloc(const cwb_model* m, const void* Xnew, int32_t x_dtype, int64_t n_new, float* out);

/*
 * cwb_autotune -- pick the scatter decomposition (grid size and cluster size) for this model by
 * timing `trials` scatter launches of each candidate on the model's own data.  objective 0: the
 * fastest scatter (the model has the GPU to itself); 1: the least SM-time, CTAs x time (models that
 * share the GPU, e.g. in a batch or a server).  Changes no fitting state; graphs captured earlier are
 * rebuilt on the next fit.  best_us (nullable) receives the chosen plan's time per scatter launch.
 * Synchronises the model's stream.
 */
cwb_status cwb_autotune(cwb_model* m, int32_t objective, int32_t trials, double* best_us);

/*
 * Batched fits -- many independent models advanced together (for example CV folds x a
 * hyperparameter grid).  cwb_batch_fit queues `iterations` iterations of every model: each model's
 * next `iters_per_launch` iterations are one branch of a single CUDA graph, so one graph launch runs
 * them for all models at once and independent branches share the GPU.  Afterwards every model is in
 * the state cwb_fit(model, iterations) would leave (same kernels, same plan), and work later queued
 * on a model's own stream waits for the batch.  Models must live on one device and stay alive while
 * the batch exists; a model must not be fitted through cwb_fit while a batch launch on it is queued.
 * cwb_batch_fit returns once the work is queued; cwb_batch_synchronize waits and reports device
 * errors of every model.
 */
typedef struct cwb_batch cwb_batch;
cwb_status cwb_batch_create(cwb_model* const* models, int32_t count, int32_t iters_per_launch, cwb_batch** out);
cwb_status cwb_batch_fit(cwb_batch* b, int32_t iterations);
cwb_status cwb_batch_synchronize(cwb_batch* b);
void cwb_batch_free(cwb_batch* b);

/*
 * Fit server -- continuous batching of fit requests on one GPU.  Submitted requests queue on the
 * host and are admitted in arrival order while the sum of the admitted fits' estimated device
 * footprints stays within hbm_budget_bytes (and at most max_active fits run).  Each admitted fit
 * is created on a stream of its own and advanced in slices of slice_iterations iterations (up to two
 * slices queued per fit), so the iterations of different fits interleave on the GPU; when a fit has
 * run cfg.iterations iterations it is retired and its slot and memory go to the next request.
 *   cwb_server_submit  host buffers X, y, w and the learners follow cwb_create; X, y and w must stay
 *                      valid until the request completes (val_mask and the learners are copied).
 *                      Returns the request id.  A request larger than the whole budget: CWB_EINVAL.
 *   cwb_server_poll    one scheduling round (admit, queue slices, retire); with wait != 0 it repeats
 *                      until at least one request completes or nothing is left.  Completed ids go to
 *                      done_ids (cap entries), their number to n_done.
 *   cwb_server_take    hands over a completed request's model (the caller frees it with cwb_free);
 *                      a request that failed reports CWB_ESTATE and its message.
 *   cwb_server_stats   pending, active, admitted, completed, bytes in use, budget (host int64).
 *   cwb_server_free    frees the server, its running fits and completed fits not taken.
 * The server is not thread-safe.
 */
typedef struct cwb_server cwb_server;
typedef struct {
    int32_t device;
    uint64_t hbm_budget_bytes;
    int32_t max_active;          /* <= 0: 64 */
    int32_t slice_iterations;    /* <= 0: 32 */
} cwb_server_config;
cwb_status cwb_server_create(const cwb_server_config* cfg, cwb_server** out);
cwb_status cwb_server_submit(cwb_server* s, const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n,
                             int32_t p, const void* y, const double* w, const cwb_learner* bl, int32_t K, int64_t* id);
cwb_status cwb_server_poll(cwb_server* s, int32_t wait, int64_t* done_ids, int32_t cap, int32_t* n_done);
cwb_status cwb_server_take(cwb_server* s, int64_t id, cwb_model** out);
cwb_status cwb_server_stats(const cwb_server* s, int64_t* values, int32_t cap);
void cwb_server_free(cwb_server* s);

/*
 * Row shards -- the rows of one fit split over several GPUs (one process and one model per GPU).
 * binMatVec sums over rows (Algorithm 2), so every shard scatters its own rows and the
 * histograms are added across shards; every shard then runs the same solve and argmin on the
 * same totals and keeps its rows' f in step.  The caller moves the data between shards (an
 * all-reduce of its communication library, or a plain sum when the shards share a process):
 *
 *   setup      cwb_shard_create on each shard's rows with the feature ranges and the row count of
 *              all shards (n* = floor(sqrt(n_global)) for CWB_BINS_SQRT), then cwb_shard_stats
 *              (bin counts [B][S] and {sum of y, rows}: SUM over shards; the bin-count bound of
 *              the scatter: MAX) and cwb_shard_finish with the totals: Z^T Z, lambda and the
 *              cached inverse from the counts of all rows, the offset from all rows.
 *   iteration  cwb_shard_rows (pending update, pseudo residuals of the shard's rows, their
 *              max |r|: MAX over shards), cwb_shard_scatter with that maximum (the common
 *              fixed-point scale; u = the shard's exact histogram sums, int64 [B][S]: SUM over
 *              shards; integer sums, so the total does not depend on the order of the
 *              additions), cwb_shard_solve with the total.
 *
 * Plain CWB, unweighted rows, equidistant (or categorical) binnings.  B and S come from
 * cwb_shard_sizes.  Buffers follow device_ptrs (device buffers on the shard's device let
 * the exchange run without host copies).  cwb_fit is not available on a shard; the getters
 * (trace, coefficients, fitted values of the shard's rows, prediction) are.
 */
typedef struct {
    int64_t n_global;     /* rows of all shards together */
    const double* xmin;   /* p per-feature minima over all shards' rows (host memory) */
    const double* xmax;   /* p per-feature maxima over all shards' rows (host memory) */
} cwb_shard_config;
cwb_status cwb_shard_create(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p, const void* y,
                            const cwb_learner* bl, int32_t K, int32_t device_ptrs, const cwb_shard_config* sc,
                            cwb_model** out);
cwb_status cwb_shard_sizes(const cwb_model* m, int32_t* B, int32_t* S);
cwb_status cwb_shard_stats(cwb_model* m, double* counts, double* sums, int32_t* cnt_log2);
cwb_status cwb_shard_finish(cwb_model* m, const double* counts, const double* sums, int32_t cnt_log2);
cwb_status cwb_shard_rows(cwb_model* m, float* rmax, int32_t device_ptrs);
cwb_status cwb_shard_scatter(cwb_model* m, const float* rmax, int64_t* u, int32_t device_ptrs);
cwb_status cwb_shard_solve(cwb_model* m, const int64_t* u, int32_t device_ptrs);

/* cwb_synchronize -- wait for the model's queued work; reports device-side errors. */
cwb_status cwb_synchronize(cwb_model* m);

/* cwb_last_error -- message of the last failure on the calling thread ("" if none). */
const char* cwb_last_error(void);

/* cwb_free -- release a model and all its device memory; NULL is a no-op. */
void cwb_free(cwb_model* m);

#ifdef __cplusplus
}
#endif

#endif /* CWB_H */
