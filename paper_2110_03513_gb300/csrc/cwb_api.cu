// cwb_api.cu -- the C ABI (include/cwb.h): argument checks, model lifecycle,
// prediction and read-back.  All arithmetic of the method runs in kernels;
// host code here validates, allocates, orders launches and copies results.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

#include "cwb_internal.cuh"
#include "cwb_bspline.cuh"
#include "cwb_noalloc_size.h"

namespace cwb {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

cwb_status cuda_status(cudaError_t e, const char* what)
{
    set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? CWB_ENOMEM : CWB_ECUDA;
}

cwb_status dev_alloc(void** p, size_t bytes, cudaStream_t)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                  cudaGetErrorString(e));
        return CWB_ENOMEM;
    }
    return CWB_OK;
}

void dev_free(void* p)
{
    if (p) cudaFree(p);
}

namespace {

// g_k(x)^T theta of one learner at a raw value x.  Categorical learners (App. B.1) take the raw value: a valid class code selects its
// coefficient, anything else contributes nothing.  Numeric learners clamp x to the
// training range.  For a binary learner q holds the class it indicates.
__device__ double learner_eval(double x, int type, int q, int nk, double xmin, double xmax, const double* theta)
{
    if (type == CWB_BL_CATEGORICAL || type == CWB_BL_CATEGORICAL_BINARY) {
        if (!(x >= 0.0 && x < (double)nk && x == floor(x))) return 0.0;
        const int code = (int)x;
        if (type == CWB_BL_CATEGORICAL) return theta[code];
        return code == q ? theta[0] : 0.0;
    }
    x = fmin(fmax(x, xmin), xmax);
    if (type == CWB_BL_LINEAR) return theta[0] + theta[1] * x;
    // P-spline: g_k(x)^T theta over the q + 1 non-zero B-splines at x
    double N[kMaxNnz];
    const int c0 = bspline_nonzero(x, xmin, xmax, q, nk, N);
    double acc = 0.0;
    for (int t = 0; t <= q; ++t) acc += N[t] * theta[c0 + t];
    return acc;
}

template <typename T>
__global__ void k_predict(const T* __restrict__ X, int64_t n_new, int K, int D, const int32_t* __restrict__ l_feat,
                          const int32_t* __restrict__ l_type, const int32_t* __restrict__ l_degree,
                          const int32_t* __restrict__ l_nknots, const double* __restrict__ l_xmin,
                          const double* __restrict__ l_xmax, const double* __restrict__ coef, double offset,
                          float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_new; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = offset;
        for (int k = 0; k < K; ++k) {
            const double x = (double)X[(int64_t)l_feat[k] * n_new + i];
            acc += learner_eval(x, l_type[k], l_degree[k], l_nknots[k], l_xmin[k], l_xmax[k], coef + (int64_t)k * D);
        }
        out[i] = (float)acc;
    }
}

// Fitted values in the caller's row order; f holds compensated (hi, lo) pairs.
__global__ void k_unpermute(const float* __restrict__ f, const int32_t* __restrict__ perm, int64_t n,
                            float* __restrict__ out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[perm ? perm[q] : q] = f[2 * q] + f[2 * q + 1];
}

int grid_1d(int64_t work, int device)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int64_t g = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)std::max(sms, 1) * 8));
}

// Makes the model's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void free_model(cwb_model* m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    void* bufs[] = {m->ind, m->y, m->y_lo, m->w, m->f, m->h, m->c, m->rw, m->perm, m->zb, m->zb64, m->zcol, m->crange, m->toff, m->ztab, m->G,
                    m->P, m->Acrit, m->Pdf, m->Adf, m->lambda, m->l_bin, m->l_d, m->l_nstar, m->l_type, m->l_xmin, m->l_xmax, m->l_degree,
                    m->l_nknots, m->l_feat, m->part, m->cluster_slot, m->slot_c0, m->theta_it, m->q_it, m->v, m->state, m->risk_part, m->tr_k,
                    m->tr_mode, m->tr_theta, m->tr_q, m->forced, m->coef, m->f2, m->uacc, m->gbar, m->ptime, m->ztab_lo,
                    m->vmax, m->u_shard};
    for (void* p : bufs) dev_free(p);
    profile_release(m);
    release_graphs(m);
    for (cudaEvent_t e : m->prof_ph)
        if (e) cudaEventDestroy(e);
    if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

cwb_status validate_learner(const cwb_learner& b, int32_t p, int k)
{
    auto bad = [&](const std::string& why) {
        set_error("learner " + std::to_string(k) + ": " + why);
        return CWB_EINVAL;
    };
    if (b.feature < 0 || b.feature >= p) return bad("feature index out of range");
    if (b.type < CWB_BL_PSPLINE || b.type > CWB_BL_CATEGORICAL_BINARY) return bad("unknown base-learner type");
    if (b.type == CWB_BL_CATEGORICAL) {
        if (b.n_knots < 2 || b.n_knots > CWB_MAX_D) return bad("a ridge learner needs 2 <= classes <= CWB_MAX_D");
        if (!(b.df > 0.0) && !(b.lambda >= 0.0)) return bad("need df > 0 or lambda >= 0");
        return CWB_OK;
    }
    if (b.type == CWB_BL_CATEGORICAL_BINARY) {
        if (b.n_knots < 2 || b.n_knots > CWB_MAX_BINS) return bad("a binary learner needs 2 <= classes <= 65535");
        if (b.level < 0 || b.level >= b.n_knots) return bad("level must be in [0, classes)");
        return CWB_OK;
    }
    if (b.n_bins != CWB_BINS_EXACT && b.n_bins != CWB_BINS_SQRT && (b.n_bins < 2 || b.n_bins > CWB_MAX_BINS))
        return bad("n_bins must be CWB_BINS_EXACT, CWB_BINS_SQRT or in [2, 65535]");
    if (b.type == CWB_BL_PSPLINE) {
        if (b.degree < 0 || b.degree > 3) return bad("degree must be in [0, 3]");
        if (b.n_knots < 0) return bad("n_knots must be >= 0");
        int d = b.n_knots + b.degree + 1;
        if (d > CWB_MAX_D) return bad("basis dimension exceeds CWB_MAX_D");
        if (b.diff_order < 1 || b.diff_order >= d) return bad("diff_order must be in [1, d)");
        if (!(b.df > 0.0) && !(b.lambda >= 0.0)) return bad("need df > 0 or lambda >= 0");
        if (b.df > 0.0 && !(b.df > b.diff_order)) return bad("df must exceed the penalty null-space dimension");
    }
    return CWB_OK;
}

cwb_status create_impl(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p, const void* y,
                       const double* w, const cwb_learner* bl, int32_t K, int32_t device_ptrs, cwb_model** out,
                       int iter_mode, const cwb_shard_config* sc = nullptr, int stream_priority = 0)
{
    if (!out) { set_error("out is NULL"); return CWB_EINVAL; }
    *out = nullptr;
    if (!cfg || !X || !y || !bl) { set_error("NULL argument"); return CWB_EINVAL; }
    if (n < 2 || n > (int64_t)INT32_MAX) { set_error("n must be in [2, 2^31-1]"); return CWB_EINVAL; }
    if (p < 1 || K < 1) { set_error("p and K must be >= 1"); return CWB_EINVAL; }
    if (x_dtype != CWB_F32 && x_dtype != CWB_F64) { set_error("x_dtype must be CWB_F32 or CWB_F64"); return CWB_EINVAL; }
    if (cfg->loss != CWB_LOSS_L2 && cfg->loss != CWB_LOSS_BINOMIAL) { set_error("unknown loss"); return CWB_EINVAL; }
    if (cfg->opt < CWB_OPT_CWB || cfg->opt > CWB_OPT_HCWB) { set_error("unknown optimizer"); return CWB_EINVAL; }
    if (!(cfg->nu > 0.0) || !isfinite(cfg->nu)) { set_error("nu must be > 0"); return CWB_EINVAL; }
    if (!(cfg->gamma >= 0.0) || !isfinite(cfg->gamma)) { set_error("gamma must be >= 0"); return CWB_EINVAL; }
    if (cfg->iterations < 0 || cfg->patience < 0) { set_error("iterations and patience must be >= 0"); return CWB_EINVAL; }
    if (cfg->opt == CWB_OPT_HCWB && !cfg->val_mask) { set_error("HCWB needs a validation mask"); return CWB_EINVAL; }
    for (int k = 0; k < K; ++k) CWB_TRY(validate_learner(bl[k], p, k));
    if (sc) {
        if (cfg->opt != CWB_OPT_CWB) { set_error("row shards run plain CWB"); return CWB_EINVAL; }
        if (w) { set_error("row shards take unweighted rows"); return CWB_EINVAL; }
        if (!sc->xmin || !sc->xmax || sc->n_global < n) { set_error("bad shard configuration"); return CWB_EINVAL; }
        for (int k = 0; k < K; ++k)
            if (bl[k].n_bins == CWB_BINS_EXACT && bl[k].type != CWB_BL_CATEGORICAL &&
                bl[k].type != CWB_BL_CATEGORICAL_BINARY) {
                set_error("row shards need equidistant binnings (the unique values differ per shard)");
                return CWB_EINVAL;
            }
    }

    cwb_model* m = new cwb_model();
    int dev = cfg->device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    }
    m->device = dev;
    DeviceGuard guard(dev);
    if (!guard.ok) {
        delete m;
        set_error("cannot select CUDA device " + std::to_string(dev));
        return CWB_ECUDA;
    }
    m->cfg = *cfg;
    m->cfg.val_mask = nullptr;
    m->cfg.device = dev;
    m->n = n;
    m->p = p;
    m->K = K;
    m->hybrid = cfg->opt == CWB_OPT_HCWB;
    m->accel = cfg->opt != CWB_OPT_CWB;
    m->iter_mode = sc ? kIterKernels : iter_mode;
    if (sc) {
        m->shard = true;
        m->shard_n_global = sc->n_global;
        m->shard_xmin.assign(sc->xmin, sc->xmin + p);
        m->shard_xmax.assign(sc->xmax, sc->xmax + p);
    }
    if (const char* wc = std::getenv("CWB_WAIT_CYCLES")) {
        // limit of the device-side ring waits in SM clocks (default ~2 s); a short limit makes a
        // wait run out on purpose (failure-path tests)
        const long long v = std::atoll(wc);
        if (v > 0) m->wait_cycles = v;
    }
    if (const char* wt = std::getenv("CWB_WITHHOLD_TILE")) {
        // failure-path test hook: the first scatter CTA arms this tile's ring stage but never issues its
        // copies, so the waits on it run out and the kernel returns CWB_ETIMEOUT
        m->withhold_tile = std::atoi(wt);
    }
    if (const char* dq = std::getenv("CWB_DIRECT_Q")) m->direct_enabled = std::atoi(dq) != 0;
    if (const char* sw = std::getenv("CWB_SLEEP_WAITS")) m->sleep_waits = std::atoi(sw) != 0 ? 1 : 0;
    if (const char* mode = std::getenv("CWB_ITER_MODE")) {
        // "kernels" or unset: three kernels per iteration (rows, scatter, solve) launched from CUDA
        // graphs; "persistent": one persistent cooperative kernel for plain CWB models that qualify
        if (iter_mode == kIterAuto && std::strcmp(mode, "kernels") == 0) m->iter_mode = kIterKernels;
        else if (iter_mode == kIterAuto && std::strcmp(mode, "persistent") == 0) m->iter_mode = kIterPersistent;
    }
    if (cfg->stream) {
        m->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        cudaError_t e = cudaStreamCreateWithPriority(&m->stream, cudaStreamNonBlocking, stream_priority);
        if (e != cudaSuccess) {
            delete m;
            return cuda_status(e, "cudaStreamCreate");
        }
        m->own_stream = true;
    }
    // learners on the same feature with the same binning share one index vector; categorical
    // learners on one feature with the same number of classes share the class-code binning
    std::map<std::tuple<int, int, int>, int> bmap;
    for (int k = 0; k < K; ++k) {
        HostLearner L;
        L.spec = bl[k];
        const bool cat = bl[k].type == CWB_BL_CATEGORICAL || bl[k].type == CWB_BL_CATEGORICAL_BINARY;
        auto key = std::make_tuple(bl[k].feature, cat ? 1 : 0, cat ? bl[k].n_knots : bl[k].n_bins);
        auto it = bmap.find(key);
        if (it == bmap.end()) {
            HostBinning hb{};
            hb.feature = bl[k].feature;
            hb.nbins_spec = cat ? bl[k].n_knots : bl[k].n_bins;
            hb.categories = cat ? bl[k].n_knots : 0;
            it = bmap.emplace(key, (int)m->bins.size()).first;
            m->bins.push_back(hb);
        }
        L.binning = it->second;
        if (bl[k].type == CWB_BL_LINEAR) {
            L.d = 2;
            L.nnz = 2;
        } else if (bl[k].type == CWB_BL_CATEGORICAL) {
            L.d = bl[k].n_knots;
            L.nnz = 1;
        } else if (bl[k].type == CWB_BL_CATEGORICAL_BINARY) {
            L.d = 1;
            L.nnz = 1;
        } else {
            L.d = bl[k].n_knots + bl[k].degree + 1;
            L.nnz = bl[k].degree + 1;
        }
        m->lrn.push_back(L);
    }
    m->B = (int)m->bins.size();

    cwb_status st = setup_model(m, X, x_dtype, y, w, cfg->val_mask, device_ptrs);
    if (st == CWB_OK) {
        for (int k = 0; k < K; ++k) {
            const cwb_learner& b = bl[k];
            if (b.type == CWB_BL_PSPLINE && m->bins[m->lrn[k].binning].nstar < 2) st = CWB_EINVAL;
        }
    }
    if (st == CWB_OK) st = plan_scatter(m);
    if (st == CWB_OK) {
        const int S = m->nstar_max, D = m->d_max;
        std::vector<int32_t> feat(K);
        for (int k = 0; k < K; ++k) feat[k] = bl[k].feature;
        int32_t* l_feat = nullptr;
        st = dev_alloc((void**)&m->theta_it, sizeof(double) * 2 * K * D, m->stream);
        if (st == CWB_OK) st = dev_alloc((void**)&m->q_it, sizeof(double) * 2 * K, m->stream);
        if (st == CWB_OK) st = dev_alloc((void**)&m->v, sizeof(float) * 2 * (size_t)K * S, m->stream);
        if (st == CWB_OK) st = dev_alloc((void**)&m->state, sizeof(DevState), m->stream);
        if (st == CWB_OK) st = dev_alloc((void**)&m->coef, sizeof(double) * 2 * K * D, m->stream);
        if (st == CWB_OK) st = dev_alloc((void**)&m->vmax, sizeof(float) * K, m->stream);
        if (st == CWB_OK && m->shard)
            st = dev_alloc((void**)&m->u_shard, sizeof(long long) * (size_t)m->B * m->nstar_max, m->stream);
        if (st == CWB_OK) st = dev_alloc((void**)&l_feat, sizeof(int32_t) * K, m->stream);
        if (st == CWB_OK) {
            m->risk_blocks = 0;
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            st = dev_alloc((void**)&m->risk_part, sizeof(double) * (size_t)std::max(sms, 1) * 8, m->stream);
        }
        if (st == CWB_OK) {
            cudaError_t e = cudaMemcpyAsync(l_feat, feat.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, m->stream);
            if (e != cudaSuccess) st = cuda_status(e, "cudaMemcpyAsync");
        }
        if (st == CWB_OK) {
            DevState s0{};
            s0.m = 0;
            s0.m_applied = 0;
            s0.mode = m->accel ? kModeACWB : kModeCWB;
            s0.phase = 0;
            s0.k_sel = -1;
            s0.k_cor = -1;
            s0.pend_mode = kModeCWB;
            cudaError_t e = cudaMemcpyAsync(m->state, &s0, sizeof(s0), cudaMemcpyHostToDevice, m->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * 2 * (size_t)K * S, m->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(m->coef, 0, sizeof(double) * 2 * K * D, m->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(m->vmax, 0, sizeof(float) * K, m->stream);
            if (e != cudaSuccess) st = cuda_status(e, "state init");
        }
        if (st == CWB_OK) st = scatter_count_pass(m);
        if (st == CWB_OK && !m->accel && !m->shard) st = init_residual_bound(m);
        if (st == CWB_OK) st = plan_persistent(m);
        if (st == CWB_OK && m->iter_mode == kIterPersistent && !m->persist_ok) {
            set_error("CWB_ITER_MODE=persistent: this model does not qualify for the persistent iteration kernel");
            st = CWB_EINVAL;
        }
        if (st == CWB_OK) st = ensure_trace(m, std::max(cfg->iterations, 1));
        if (st == CWB_OK) st = launch_initial_rows(m);
        if (st == CWB_OK) {
            cudaError_t e = cudaStreamSynchronize(m->stream);
            if (e != cudaSuccess) st = cuda_status(e, "create");
        }
        if (st == CWB_OK) st = read_device_error(m);
        if (st == CWB_OK) m->l_feat = l_feat;
        else dev_free(l_feat);
    }
    if (st != CWB_OK) {
        free_model(m);
        return st;
    }
    *out = m;
    return CWB_OK;
}

}  // namespace

cwb_status create_model(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p, const void* y,
                        const double* w, const cwb_learner* bl, int32_t K, int32_t device_ptrs, cwb_model** out,
                        int iter_mode, int stream_priority)
{
    set_error("");
    try {
        return create_impl(cfg, X, x_dtype, n, p, y, w, bl, K, device_ptrs, out, iter_mode, nullptr, stream_priority);
    } catch (const std::exception& e) {
        set_error(std::string("host exception: ") + e.what());
        return CWB_ENOMEM;
    }
}

cwb_status launch_predict(const cwb_model* m, const void* Xnew, int x_dtype, int64_t n_new, float* out_dev)
{
    const int g = grid_1d(n_new, m->device);
    if (x_dtype == CWB_F64)
        k_predict<<<g, 256, 0, m->stream>>>((const double*)Xnew, n_new, m->K, m->d_max, m->l_feat, m->l_type,
                                            m->l_degree, m->l_nknots, m->l_xmin, m->l_xmax, m->coef, m->offset,
                                            out_dev);
    else
        k_predict<<<g, 256, 0, m->stream>>>((const float*)Xnew, n_new, m->K, m->d_max, m->l_feat, m->l_type,
                                            m->l_degree, m->l_nknots, m->l_xmin, m->l_xmax, m->coef, m->offset,
                                            out_dev);
    CWB_CUDA_TRY(cudaGetLastError());
    return CWB_OK;
}

}  // namespace cwb

using namespace cwb;

extern "C" {

cwb_status cwb_create(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p, const void* y,
                      const double* w, const cwb_learner* bl, int32_t K, int32_t device_ptrs, cwb_model** out)
{
    return create_model(cfg, X, x_dtype, n, p, y, w, bl, K, device_ptrs, out, kIterAuto);
}

cwb_status cwb_create_many(const cwb_fit_request* reqs, int32_t count, int32_t device_ptrs, int32_t threads,
                           cwb_model** out, cwb_status* status)
{
    set_error("");
    if (!reqs || !out || count < 0) { set_error("cwb_create_many: bad argument"); return CWB_EINVAL; }
    if (count == 0) return CWB_OK;
    for (int32_t i = 0; i < count; ++i) out[i] = nullptr;
    try {
        int nt = threads > 0 ? threads : std::min(16, (int)std::max(1u, std::thread::hardware_concurrency()));
        nt = std::max(1, std::min(nt, (int)count));
        std::vector<cwb_status> st((size_t)count, CWB_OK);
        std::vector<std::string> msg((size_t)count);
        std::atomic<int32_t> next{0};
        // each worker takes the next request and creates its model (own stream, own temporaries); the
        // setup kernels and the host-side steps of different requests overlap
        auto work = [&]() {
            for (;;) {
                const int32_t i = next.fetch_add(1);
                if (i >= count) break;
                const cwb_fit_request& r = reqs[i];
                st[i] = create_model(&r.cfg, r.X, r.x_dtype, r.n, r.p, r.y, r.w, r.bl, r.K, device_ptrs, &out[i],
                                     kIterAuto);
                if (st[i] != CWB_OK) msg[i] = g_last_error;
            }
        };
        std::vector<std::thread> pool;
        try {
            for (int t = 1; t < nt; ++t) pool.emplace_back(work);
        } catch (const std::exception&) {
            // fewer threads than asked (the host refused more): the ones running take every request
        }
        work();
        for (std::thread& t : pool) t.join();
        cwb_status first = CWB_OK;
        for (int32_t i = 0; i < count; ++i) {
            if (status) status[i] = st[i];
            if (st[i] != CWB_OK && first == CWB_OK) {
                first = st[i];
                set_error("cwb_create_many: request " + std::to_string(i) + ": " + msg[i]);
            }
        }
        return first;
    } catch (const std::exception& e) {
        set_error(std::string("cwb_create_many: host exception: ") + e.what());
        return CWB_ENOMEM;
    }
}

cwb_status cwb_fit(cwb_model* m, int32_t iterations)
{
    set_error("");
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    int32_t it = iterations > 0 ? iterations : m->cfg.iterations;
    if (it <= 0) return CWB_OK;
    if (m->shard) {
        set_error("a row shard runs its iterations through cwb_shard_rows / cwb_shard_scatter / cwb_shard_solve");
        return CWB_ESTATE;
    }
    try {
        CWB_TRY(launch_iterations(m, it));   // the last update is applied when f is next read
    } catch (const std::exception& e) {
        set_error(std::string("host exception: ") + e.what());
        return CWB_ENOMEM;
    }
    return CWB_OK;
}

cwb_status cwb_synchronize(cwb_model* m)
{
    set_error("");
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return read_device_error(m);
}

cwb_status cwb_predict(const cwb_model* mc, const void* Xnew, int32_t x_dtype, int64_t n_new, float* out,
                       int32_t device_ptrs)
{
    set_error("");
    cwb_model* m = const_cast<cwb_model*>(mc);
    if (!m || !Xnew || !out) { set_error("NULL argument"); return CWB_EINVAL; }
    if (n_new < 0) { set_error("n_new must be >= 0"); return CWB_EINVAL; }
    if (x_dtype != CWB_F32 && x_dtype != CWB_F64) { set_error("x_dtype must be CWB_F32 or CWB_F64"); return CWB_EINVAL; }
    if (n_new == 0) return CWB_OK;
    DeviceGuard guard(m->device);
    CWB_TRY(launch_aggregate(m));
    const size_t xsz = (x_dtype == CWB_F64 ? 8 : 4) * (size_t)n_new * m->p;
    void* xd = const_cast<void*>(Xnew);
    float* od = out;
    if (!device_ptrs) {
        CWB_TRY(dev_alloc(&xd, xsz, m->stream));
        CWB_TRY(dev_alloc((void**)&od, sizeof(float) * n_new, m->stream));
        cudaError_t e = cudaMemcpyAsync(xd, Xnew, xsz, cudaMemcpyHostToDevice, m->stream);
        if (e != cudaSuccess) { dev_free(xd); dev_free(od); return cuda_status(e, "cudaMemcpyAsync"); }
    }
    cwb_status st = launch_predict(m, xd, x_dtype, n_new, od);
    if (st == CWB_OK && !device_ptrs) {
        cudaError_t e = cudaMemcpyAsync(out, od, sizeof(float) * n_new, cudaMemcpyDeviceToHost, m->stream);
        if (e != cudaSuccess) st = cuda_status(e, "cudaMemcpyAsync");
    }
    if (st == CWB_OK) {
        cudaError_t e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = cuda_status(e, "predict");
    }
    if (!device_ptrs) { dev_free(xd); dev_free(od); }
    if (st == CWB_OK) st = read_device_error(m);
    return st;
}

cwb_status cwb_get_coefficients(const cwb_model* mc, int32_t k, int32_t which, double* theta, int32_t cap,
                                double* offset)
{
    set_error("");
    cwb_model* m = const_cast<cwb_model*>(mc);
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    if (k < 0 || k >= m->K || (which != 0 && which != 1) || (cap > 0 && !theta)) {
        set_error("bad learner index, which or buffer");
        return CWB_EINVAL;
    }
    DeviceGuard guard(m->device);
    CWB_TRY(launch_aggregate(m));
    const int d = m->lrn[k].d;
    const int cnt = std::min(d, std::max(cap, 0));
    if (cnt > 0)
        CWB_CUDA_TRY(cudaMemcpyAsync(theta, m->coef + ((int64_t)which * m->K + k) * m->d_max, sizeof(double) * cnt,
                                     cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (offset) *offset = m->offset;
    return read_device_error(m);
}

cwb_status cwb_get_trace(const cwb_model* mc, int32_t* k_sel, int32_t* k_cor, int32_t cap, int32_t* switch_iter,
                         int32_t* done)
{
    set_error("");
    cwb_model* m = const_cast<cwb_model*>(mc);
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    CWB_TRY(materialize(m));
    const int32_t cnt = std::min(std::max(cap, 0), m->done);
    std::vector<int32_t> tk(2 * (size_t)std::max(cnt, 1));
    if (cnt > 0)
        CWB_CUDA_TRY(cudaMemcpyAsync(tk.data(), m->tr_k, sizeof(int32_t) * 2 * cnt, cudaMemcpyDeviceToHost, m->stream));
    DevState st;
    CWB_CUDA_TRY(cudaMemcpyAsync(&st, m->state, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int32_t t = 0; t < cnt; ++t) {
        if (k_sel) k_sel[t] = tk[2 * t];
        if (k_cor) k_cor[t] = tk[2 * t + 1];
    }
    if (switch_iter) *switch_iter = (st.switch_iter > 0 && st.switch_iter <= m->done) ? st.switch_iter : 0;
    if (done) *done = m->done;
    return read_device_error(m);
}

cwb_status cwb_get_criteria(const cwb_model* mc, double* q_best, double* q_second, int32_t cap)
{
    set_error("");
    cwb_model* m = const_cast<cwb_model*>(mc);
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    const int32_t cnt = std::min(std::max(cap, 0), m->done);
    std::vector<double> tq(2 * (size_t)std::max(cnt, 1));
    if (cnt > 0)
        CWB_CUDA_TRY(cudaMemcpyAsync(tq.data(), m->tr_q, sizeof(double) * 2 * cnt, cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int32_t t = 0; t < cnt; ++t) {
        if (q_best) q_best[t] = tq[2 * t];
        if (q_second) q_second[t] = tq[2 * t + 1];
    }
    return read_device_error(m);
}

cwb_status cwb_get_fitted(const cwb_model* mc, float* f, int32_t device_ptrs)
{
    set_error("");
    cwb_model* m = const_cast<cwb_model*>(mc);
    if (!m || !f) { set_error("NULL argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    CWB_TRY(materialize(m));
    float* od = f;
    if (!device_ptrs) CWB_TRY(dev_alloc((void**)&od, sizeof(float) * m->n, m->stream));
    k_unpermute<<<grid_1d(m->n, m->device), 256, 0, m->stream>>>(m->f, m->perm, m->n, od);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !device_ptrs)
        e = cudaMemcpyAsync(f, od, sizeof(float) * m->n, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (!device_ptrs) dev_free(od);
    if (e != cudaSuccess) return cuda_status(e, "cwb_get_fitted");
    return read_device_error(m);
}

cwb_status cwb_get_learner_info(const cwb_model* m, int32_t k, cwb_learner_info* info)
{
    set_error("");
    if (!m || !info || k < 0 || k >= m->K) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    const HostLearner& L = m->lrn[k];
    const HostBinning& hb = m->bins[L.binning];
    double lam[2] = {0.0, 0.0};
    CWB_CUDA_TRY(cudaMemcpyAsync(&lam[0], m->lambda + k, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaMemcpyAsync(&lam[1], m->lambda + m->K + k, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    info->d = L.d;
    info->nstar = hb.nstar;
    info->binning = L.binning;
    info->reserved = 0;
    info->xmin = hb.xmin;
    info->xmax = hb.xmax;
    info->lambda = lam[0];
    info->lambda_full = m->hybrid ? lam[1] : lam[0];
    return CWB_OK;
}

cwb_status cwb_get_learner_matrices(const cwb_model* m, int32_t k, int32_t phase, double* G, double* P)
{
    set_error("");
    if (!m || k < 0 || k >= m->K || phase < 0 || phase > 1) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    const int d = m->lrn[k].d, D = m->d_max;
    const int ph = m->hybrid ? phase : 0;
    std::vector<double> buf((size_t)D * D);
    for (int which = 0; which < 2; ++which) {
        double* dst = which == 0 ? G : P;
        if (!dst) continue;
        const double* src = (which == 0 ? m->G : m->P) + ((int64_t)ph * m->K + k) * D * D;
        CWB_CUDA_TRY(cudaMemcpyAsync(buf.data(), src, sizeof(double) * D * D, cudaMemcpyDeviceToHost, m->stream));
        CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) dst[i * d + j] = buf[(size_t)i * D + j];
    }
    return CWB_OK;
}

cwb_status cwb_get_bin_index(const cwb_model* m, int32_t k, int32_t* ind)
{
    set_error("");
    if (!m || !ind || k < 0 || k >= m->K) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    const int b = m->lrn[k].binning;
    const size_t nb = (size_t)m->ind_bytes * m->n;
    std::vector<uint8_t> raw(nb);
    std::vector<int32_t> perm;
    CWB_CUDA_TRY(cudaMemcpyAsync(raw.data(), (const uint8_t*)m->ind + (size_t)m->ind_bytes * b * m->n_pad, nb,
                                 cudaMemcpyDeviceToHost, m->stream));
    if (m->perm) {
        perm.resize(m->n);
        CWB_CUDA_TRY(cudaMemcpyAsync(perm.data(), m->perm, sizeof(int32_t) * m->n, cudaMemcpyDeviceToHost, m->stream));
    }
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int64_t q = 0; q < m->n; ++q) {
        int v = m->ind_bytes == 1 ? raw[q] : ((const uint16_t*)raw.data())[q];
        ind[m->perm ? perm[q] : q] = v;
    }
    return CWB_OK;
}

cwb_status cwb_get_residuals(const cwb_model* m, int32_t channel, float* out)
{
    set_error("");
    if (!m || !out || channel < 0 || channel > 1) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    std::vector<float> raw(m->n);
    std::vector<int32_t> perm;
    DevState st;
    CWB_CUDA_TRY(cudaMemcpyAsync(&st, m->state, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (st.resid_path == 1) {
        // the persistent path forms w r inside its scatter: recompute it at the model's current f
        // (channel 1 is not used by plain CWB)
        if (channel == 1) {
            for (int64_t q = 0; q < m->n; ++q) out[q] = 0.0f;
            return CWB_OK;
        }
        CWB_TRY(persistent_residuals(const_cast<cwb_model*>(m), m->rw));
        CWB_CUDA_TRY(cudaMemcpyAsync(raw.data(), m->rw, sizeof(float) * m->n, cudaMemcpyDeviceToHost, m->stream));
    } else {
        CWB_CUDA_TRY(cudaMemcpyAsync(raw.data(), m->rw + (int64_t)channel * m->n_pad, sizeof(float) * m->n,
                                     cudaMemcpyDeviceToHost, m->stream));
    }
    if (st.resid_path == 2) {
        // the row pass wrote w r as int32 fixed point, w r * 2^fix_exp (channel 1 is not used)
        CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
        const double sc = ldexp(1.0, -st.fix_exp);
        for (int64_t q = 0; q < m->n; ++q) {
            int32_t v;
            std::memcpy(&v, &raw[q], sizeof(v));
            raw[q] = channel == 1 ? 0.0f : (float)((double)v * sc);
        }
    }
    if (m->perm) {
        perm.resize(m->n);
        CWB_CUDA_TRY(cudaMemcpyAsync(perm.data(), m->perm, sizeof(int32_t) * m->n, cudaMemcpyDeviceToHost, m->stream));
    }
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int64_t q = 0; q < m->n; ++q) out[m->perm ? perm[q] : q] = raw[q];
    return CWB_OK;
}

cwb_status cwb_force_selection(cwb_model* m, const int32_t* k_forced, int32_t count)
{
    set_error("");
    if (!m || (count > 0 && !k_forced) || count < 0) { set_error("bad argument"); return CWB_EINVAL; }
    m->forced_host.assign(k_forced, k_forced + count);
    return CWB_OK;
}

cwb_status cwb_autotune(cwb_model* m, int32_t objective, int32_t trials, double* best_us)
{
    set_error("");
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    if (objective != 0 && objective != 1) { set_error("objective must be 0 or 1"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return autotune_scatter(m, objective, trials, best_us);
}

cwb_status cwb_profile(cwb_model* m, int32_t enable)
{
    set_error("");
    if (!m) { set_error("model is NULL"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    CWB_TRY(profile_collect(m));
    for (int i = 0; i < 4; ++i) {
        m->prof_ms[i] = 0.0;
        m->prof_launches[i] = 0;
    }
    if (m->persist_ok) {
        double ms3[3];
        int64_t its = 0;
        CWB_TRY(persistent_profile(m, ms3, &its, true));
    }
    const int mask = enable == CWB_PROF_ALL ? 0x7 : ((enable >> 4) & 0x7);
    if (mask != m->prof_mask && m->prof_exec) {
        cudaGraphExecDestroy(m->prof_exec);
        if (m->prof_graph) cudaGraphDestroy(m->prof_graph);
        m->prof_exec = nullptr;
        m->prof_graph = nullptr;
        m->prof_nodes.clear();
    }
    m->prof_mask = mask;
    m->prof_on = mask != 0;
    return CWB_OK;
}

cwb_status cwb_get_profile(cwb_model* m, double* ms, int64_t* launches, int32_t cap)
{
    set_error("");
    if (!m || cap < 0) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    CWB_TRY(profile_collect(m));
    if (m->persist_ok) {
        // phase times of the persistent kernel (rows, scatter, solve with the argmin), per iteration
        double ms3[3];
        int64_t its = 0;
        CWB_TRY(persistent_profile(m, ms3, &its, true));
        for (int i = 0; i < 3; ++i) {
            m->prof_ms[i] += ms3[i];
            m->prof_launches[i] += its;
        }
    }
    for (int i = 0; i < cap && i < 4; ++i) {
        if (ms) ms[i] = m->prof_ms[i];
        if (launches) launches[i] = m->prof_launches[i];
    }
    return CWB_OK;
}

cwb_status cwb_get_scatter_plan(const cwb_model* m, int32_t* values, int32_t cap)
{
    set_error("");
    if (!m || (cap > 0 && !values)) { set_error("bad argument"); return CWB_EINVAL; }
    const ScatterPlan& P = m->plan;
    const bool pers = m->persist_ok && m->iter_mode != kIterKernels;
    const int32_t v[19] = {P.f_lane, P.fe, P.groups, P.bin_ranges, P.nb_cta, P.cs, P.clusters, P.stages, P.threads,
                           (int32_t)P.smem, P.int_acc ? 1 : 0, P.active_ctas[0], P.active_ctas[1], P.active_ctas[2],
                           P.active_ctas[3], pers ? 1 : 0, pers ? m->pplan.stages : 0, pers ? m->pplan.ctas : 0,
                           pers ? (int32_t)m->pplan.smem : 0};
    for (int i = 0; i < cap && i < 19; ++i) values[i] = v[i];
    return CWB_OK;
}

// Fixed device scratch for cwb_predict_noalloc: staged Xnew followed by the predictions.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CWB_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on `dev` (looked up once per device, with that device current).
cwb_status noalloc_scratch(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("cwb_predict_noalloc supports device ordinals below 64");
        return CWB_EINVAL;
    }
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    return CWB_OK;
}
}  // namespace

cwb_status cwb_predict_noalloc(const cwb_model* mc, const void* Xnew, int32_t x_dtype, int64_t n_new, float* out)
{
    set_error("");
    cwb_model* m = const_cast<cwb_model*>(mc);
    if (!m || !Xnew || !out) { set_error("NULL argument"); return CWB_EINVAL; }
    if (n_new < 0) { set_error("n_new must be >= 0"); return CWB_EINVAL; }
    if (x_dtype != CWB_F32 && x_dtype != CWB_F64) { set_error("x_dtype must be CWB_F32 or CWB_F64"); return CWB_EINVAL; }
    if (n_new == 0) return CWB_OK;
    const int64_t xsz = (x_dtype == CWB_F64) ? 8 : 4;
    uint64_t need = 0;
    if (!cwb_noalloc_need(n_new, m->p, xsz, (uint64_t)CWB_NOALLOC_SCRATCH_BYTES, &need)) {
        set_error("cwb_predict_noalloc: " + std::to_string(n_new) + " rows of " + std::to_string(m->p) +
                  " features do not fit in the scratch limit of " + std::to_string((size_t)CWB_NOALLOC_SCRATCH_BYTES) +
                  " bytes (each row takes " + std::to_string(xsz * m->p + 4) +
                  " bytes, plus up to 255 of alignment); split the rows into several calls");
        return CWB_EINVAL;
    }
    const size_t x_bytes = (size_t)xsz * (size_t)n_new * (size_t)m->p;     // <= need, no wrap-around
    const size_t out_off = (x_bytes + 255) & ~(size_t)255;
    DeviceGuard guard(m->device);
    unsigned char* base = nullptr;
    CWB_TRY(noalloc_scratch(m->device, &base));
    CWB_TRY(launch_aggregate(m));
    CWB_CUDA_TRY(cudaMemcpyAsync(base, Xnew, x_bytes, cudaMemcpyHostToDevice, m->stream));
    float* out_dev = reinterpret_cast<float*>(base + out_off);
    CWB_TRY(launch_predict(m, base, x_dtype, n_new, out_dev));
    CWB_CUDA_TRY(cudaMemcpyAsync(out, out_dev, sizeof(float) * (size_t)n_new, cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return read_device_error(m);
}

cwb_status cwb_shard_create(const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p, const void* y,
                            const cwb_learner* bl, int32_t K, int32_t device_ptrs, const cwb_shard_config* sc,
                            cwb_model** out)
{
    set_error("");
    if (!sc) {
        if (out) *out = nullptr;
        set_error("shard configuration is NULL");
        return CWB_EINVAL;
    }
    try {
        return create_impl(cfg, X, x_dtype, n, p, y, nullptr, bl, K, device_ptrs, out, kIterKernels, sc);
    } catch (const std::exception& e) {
        set_error(std::string("host exception: ") + e.what());
        return CWB_ENOMEM;
    }
}

cwb_status cwb_shard_sizes(const cwb_model* m, int32_t* B, int32_t* S)
{
    set_error("");
    if (!m || !m->shard) { set_error("not a row shard"); return CWB_EINVAL; }
    if (B) *B = m->B;
    if (S) *S = m->nstar_max;
    return CWB_OK;
}

cwb_status cwb_shard_stats(cwb_model* m, double* counts, double* sums, int32_t* cnt_log2)
{
    set_error("");
    if (!m || !m->shard || !counts || !sums || !cnt_log2) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    return shard_stats(m, counts, sums, cnt_log2);
}

cwb_status cwb_shard_finish(cwb_model* m, const double* counts, const double* sums, int32_t cnt_log2)
{
    set_error("");
    if (!m || !m->shard || !counts || !sums) { set_error("bad argument"); return CWB_EINVAL; }
    if (m->done > 0) { set_error("cwb_shard_finish comes before the first iteration"); return CWB_ESTATE; }
    DeviceGuard guard(m->device);
    return shard_finish(m, counts, sums, cnt_log2);
}

cwb_status cwb_shard_rows(cwb_model* m, float* rmax, int32_t device_ptrs)
{
    set_error("");
    if (!m || !m->shard || !rmax) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    return shard_rows(m, rmax, device_ptrs);
}

cwb_status cwb_shard_scatter(cwb_model* m, const float* rmax, int64_t* u, int32_t device_ptrs)
{
    set_error("");
    if (!m || !m->shard || !rmax || !u) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    return shard_scatter(m, rmax, device_ptrs, reinterpret_cast<long long*>(u), device_ptrs);
}

cwb_status cwb_shard_solve(cwb_model* m, const int64_t* u, int32_t device_ptrs)
{
    set_error("");
    if (!m || !m->shard || !u) { set_error("bad argument"); return CWB_EINVAL; }
    DeviceGuard guard(m->device);
    return shard_solve(m, reinterpret_cast<const long long*>(u), device_ptrs);
}

const char* cwb_last_error(void) { return g_last_error.c_str(); }

void cwb_free(cwb_model* m)
{
    if (!m) return;
    DeviceGuard guard(m->device);
    free_model(m);
}

}  // extern "C"
