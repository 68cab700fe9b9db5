// cwb_batch.cu -- many fits on one GPU: batched graphs and a continuous-batching server.
//
//   cwb_batch   a fixed set of models advanced together: every model's next K iterations
//               are one branch of a single CUDA graph, so one graph launch runs K iterations
//               of all of them and independent branches share the GPU.
//   cwb_server  a request loop: fit requests queue on the host, are admitted while their
//               estimated device footprint fits a budget, run in slices of iterations on their
//               own streams (interleaved on the GPU) and are handed back when done.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cwb_internal.cuh"

using namespace cwb;

// ---------------------------------------------------------------------------- batch

struct cwb_batch {
    int device = 0;
    std::vector<cwb_model*> models;
    int32_t k = 32;                       // iterations per branch in the main graph
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t exec_k = nullptr, exec_1 = nullptr;
    std::vector<int32_t> cap_at_capture;  // trace capacity each model had when the graphs were captured
};

namespace {

void batch_release_graphs(cwb_batch* b)
{
    if (b->exec_k) cudaGraphExecDestroy(b->exec_k);
    if (b->exec_1) cudaGraphExecDestroy(b->exec_1);
    b->exec_k = b->exec_1 = nullptr;
}

// One graph: for every model, its next `iters` chained iterations captured on the model's capture
// stream as a graph of its own, added to the batch graph as an independent child-graph node.
cwb_status batch_capture_once(cwb_batch* b, int32_t iters, cudaGraphExec_t* out)
{
    cudaGraph_t parent = nullptr;
    CWB_CUDA_TRY(cudaGraphCreate(&parent, 0));
    cwb_status st = CWB_OK;
    for (size_t i = 0; i < b->models.size() && st == CWB_OK; ++i) {
        cwb_model* m = b->models[i];
        cudaGraph_t child = nullptr;
        cudaError_t e = cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            st = cuda_status(e, "cudaStreamBeginCapture (batch)");
            break;
        }
        for (int32_t t = 0; t < iters; ++t) enqueue_iteration(m, m->capture_stream, 0);
        cudaError_t el = cudaGetLastError();
        e = cudaStreamEndCapture(m->capture_stream, &child);
        if (el != cudaSuccess) st = cuda_status(el, "batch: iteration launches");
        else if (e != cudaSuccess) st = cuda_status(e, "cudaStreamEndCapture (batch)");
        if (st == CWB_OK) {
            cudaGraphNode_t node = nullptr;
            e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, child);
            if (e != cudaSuccess) st = cuda_status(e, "cudaGraphAddChildGraphNode");
        }
        if (child) cudaGraphDestroy(child);
    }
    if (st == CWB_OK) {
        cudaError_t e = cudaGraphInstantiate(out, parent, 0);
        if (e != cudaSuccess) st = cuda_status(e, "cudaGraphInstantiate (batch)");
    }
    cudaGraphDestroy(parent);
    return st;
}

// With programmatic dependencies between each model's kernels if the driver accepts them inside
// child graphs, otherwise with plain stream order.
cwb_status batch_capture(cwb_batch* b, int32_t iters, cudaGraphExec_t* out)
{
    if (batch_capture_once(b, iters, out) == CWB_OK) return CWB_OK;
    cudaGetLastError();
    for (cwb_model* m : b->models) m->use_pdl = false;
    cwb_status st = batch_capture_once(b, iters, out);
    for (cwb_model* m : b->models) m->use_pdl = true;
    return st;
}

}  // namespace

extern "C" {

cwb_status cwb_batch_create(cwb_model* const* models, int32_t count, int32_t iters_per_launch, cwb_batch** out)
{
    set_error("");
    if (!out || !models || count <= 0) {
        set_error("cwb_batch_create: models and out are required, count > 0");
        return CWB_EINVAL;
    }
    *out = nullptr;
    auto* b = new cwb_batch();
    b->device = models[0]->device;
    b->k = iters_per_launch > 0 ? iters_per_launch : 32;
    for (int32_t i = 0; i < count; ++i) {
        if (!models[i] || models[i]->device != b->device) {
            delete b;
            set_error("cwb_batch_create: every model must be non-NULL and on the same device");
            return CWB_EINVAL;
        }
        b->models.push_back(models[i]);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    b->joins.resize(count, nullptr);
    for (int32_t i = 0; i < count && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
    for (cwb_model* m : b->models)
        if (e == cudaSuccess && !m->capture_stream) e = cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cwb_batch_free(b);
        return cuda_status(e, "cwb_batch_create");
    }
    *out = b;
    return CWB_OK;
}

cwb_status cwb_batch_fit(cwb_batch* b, int32_t iterations)
{
    set_error("");
    if (!b) { set_error("batch is NULL"); return CWB_EINVAL; }
    if (iterations <= 0) return CWB_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    const int32_t full = iterations / b->k, rest = iterations % b->k;
    // traces must hold every queued iteration; a reallocation changes pointers baked into graphs
    bool recapture = !b->exec_k;
    b->cap_at_capture.resize(b->models.size(), 0);
    for (size_t i = 0; i < b->models.size(); ++i) {
        cwb_model* m = b->models[i];
        CWB_TRY(prepare_launch(m, iterations));
        if (m->trace_cap != b->cap_at_capture[i] || !m->graph_valid_for_batch) recapture = true;
    }
    if (recapture) {
        batch_release_graphs(b);
        for (size_t i = 0; i < b->models.size(); ++i) {
            b->cap_at_capture[i] = b->models[i]->trace_cap;
            b->models[i]->graph_valid_for_batch = true;
        }
    }
    // the models' own queued work (creation, earlier fits, getters) precedes the batch
    for (size_t i = 0; i < b->models.size(); ++i) {
        CWB_CUDA_TRY(cudaEventRecord(b->joins[i], b->models[i]->stream));
        CWB_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->joins[i], 0));
    }
    if (full > 0) {
        if (!b->exec_k) CWB_TRY(batch_capture(b, b->k, &b->exec_k));
        for (int32_t r = 0; r < full; ++r) CWB_CUDA_TRY(cudaGraphLaunch(b->exec_k, b->stream));
    }
    if (rest > 0) {
        if (!b->exec_1) CWB_TRY(batch_capture(b, 1, &b->exec_1));
        for (int32_t r = 0; r < rest; ++r) CWB_CUDA_TRY(cudaGraphLaunch(b->exec_1, b->stream));
    }
    // later work on each model's own stream waits for the batch
    CWB_CUDA_TRY(cudaEventRecord(b->done, b->stream));
    for (cwb_model* m : b->models) {
        CWB_CUDA_TRY(cudaStreamWaitEvent(m->stream, b->done, 0));
        note_iterations_queued(m, iterations);
    }
    return CWB_OK;
}

cwb_status cwb_batch_synchronize(cwb_batch* b)
{
    set_error("");
    if (!b) { set_error("batch is NULL"); return CWB_EINVAL; }
    CWB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (cwb_model* m : b->models) CWB_TRY(cwb_synchronize(m));
    return CWB_OK;
}

void cwb_batch_free(cwb_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_release_graphs(b);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------- server

namespace {

struct Request {
    int64_t id = 0;
    cwb_config cfg{};
    const void* X = nullptr;
    int32_t x_dtype = CWB_F32;
    int64_t n = 0;
    int32_t p = 0;
    const void* y = nullptr;
    const double* w = nullptr;
    std::vector<cwb_learner> bl;
    std::vector<uint8_t> val_mask;        // copied: the config's pointer need not outlive submit
    uint64_t footprint = 0;
    uint64_t index_bytes = 0;             // the index matrix's bytes (read once per iteration)
};

struct Active {
    Request req;
    cwb_model* m = nullptr;
    int32_t queued = 0;                   // iterations launched
    std::vector<cudaEvent_t> slice_done;  // ring of in-flight slice events
    int head = 0, in_flight = 0;
};

}  // namespace

struct cwb_server {
    cwb_server_config cfg{};
    int64_t next_id = 1;
    std::deque<Request> pending;
    std::vector<Active> active;
    std::unordered_map<int64_t, cwb_model*> finished;
    std::unordered_map<int64_t, std::string> failed;
    uint64_t in_use = 0;
    int64_t admitted = 0, completed = 0;
};

namespace {

constexpr int kSlicesInFlight = 2;

// Device bytes a fit holds while it runs (index matrix, row vectors, design tables, caches), plus
// the feature copy its creation stages.  An estimate from the request alone; also records the index
// matrix's bytes in the request.
uint64_t estimate_footprint(Request& r)
{
    const uint64_t n_pad = ((uint64_t)r.n + 255) / 256 * 256;
    std::vector<std::pair<int, int>> bins;
    int d_max = 2;
    uint64_t nstar_max = 2;
    for (const cwb_learner& l : r.bl) {
        const bool cat = l.type == CWB_BL_CATEGORICAL || l.type == CWB_BL_CATEGORICAL_BINARY;
        const auto key = std::make_pair(l.feature, cat ? -3 - l.n_knots : l.n_bins);   // categorical: by classes
        if (std::find(bins.begin(), bins.end(), key) == bins.end()) bins.push_back(key);
        if (l.type == CWB_BL_PSPLINE) d_max = std::max(d_max, l.n_knots + l.degree + 1);
        if (l.type == CWB_BL_CATEGORICAL) d_max = std::max(d_max, l.n_knots);
        if (cat) {
            nstar_max = std::max(nstar_max, (uint64_t)l.n_knots);
            continue;
        }
        uint64_t ns = l.n_bins > 1 ? (uint64_t)l.n_bins : (l.n_bins == CWB_BINS_SQRT ? 1 : (uint64_t)r.n);
        if (l.n_bins == CWB_BINS_SQRT) {
            ns = 1;
            while ((ns + 1) * (ns + 1) <= (uint64_t)r.n) ++ns;
        }
        nstar_max = std::max(nstar_max, ns);
    }
    const uint64_t B = bins.size(), K = r.bl.size();
    const bool accel = r.cfg.opt != CWB_OPT_CWB;
    const uint64_t elem = nstar_max <= 256 ? 1 : 2;
    uint64_t bytes = B * n_pad * elem;                                  // index matrix
    r.index_bytes = bytes;
    bytes += n_pad * (4 + 4 + 4 + 8 + 8);                               // y, y_lo, w, f, rw
    if (accel) bytes += n_pad * (8 + 4 + 4 + 4);                        // h, c, second channel, perm
    bytes += K * nstar_max * (16 + 4 + 16 + 8 + 8);                     // zb, zcol, ztab, v, zb64
    bytes += 8 * K * (uint64_t)d_max * d_max * 8;                       // G, P, A and their float pairs per phase
    bytes += 152ull * 32 * nstar_max * 4 * (accel ? 2 : 1);             // cluster partial histograms
    bytes += (uint64_t)r.p * r.n * (r.x_dtype == CWB_F64 ? 8 : 4);      // staged features during creation
    bytes += 64ull << 20;                                               // traces, tables, slack
    return bytes;
}

// Stream priority of a request: fits with less work (index bytes x iterations) run on streams of
// higher priority, so that their kernels are dispatched ahead of those of long fits when SMs free up
// (shortest work first: small requests finish without waiting behind the long ones; the long fits
// take the SMs whenever the short ones have nothing queued).
int request_priority(const Request& r, uint64_t footprint_index_bytes)
{
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const double work = (double)footprint_index_bytes * (double)std::max(1, r.cfg.iterations);
    const int levels = least - greatest + 1;              // greatest is the most negative (highest) priority
    int level = (int)std::floor(std::log10(std::max(work, 1.0))) - 8;
    level = std::max(0, std::min(levels - 1, level));
    return greatest + level;
}

bool slice_finished(Active& a)
{
    while (a.in_flight > 0) {
        cudaEvent_t e = a.slice_done[(a.head + kSlicesInFlight - a.in_flight) % kSlicesInFlight];
        cudaError_t q = cudaEventQuery(e);
        if (q == cudaErrorNotReady) return false;
        if (q != cudaSuccess) return false;
        --a.in_flight;
    }
    return true;
}

void retire(cwb_server* s, size_t idx, bool ok, const std::string& why)
{
    Active& a = s->active[idx];
    for (cudaEvent_t e : a.slice_done)
        if (e) cudaEventDestroy(e);
    a.slice_done.clear();
    if (ok) s->finished[a.req.id] = a.m;
    else {
        s->failed[a.req.id] = why;
        cwb_free(a.m);
    }
    s->in_use -= a.req.footprint;
    s->completed += 1;
    s->active.erase(s->active.begin() + idx);
}

}  // namespace

extern "C" {

cwb_status cwb_server_create(const cwb_server_config* cfg, cwb_server** out)
{
    set_error("");
    if (!cfg || !out) { set_error("cwb_server_create: NULL argument"); return CWB_EINVAL; }
    if (cfg->hbm_budget_bytes == 0) { set_error("cwb_server_create: hbm_budget_bytes must be > 0"); return CWB_EINVAL; }
    auto* s = new cwb_server();
    s->cfg = *cfg;
    if (s->cfg.max_active <= 0) s->cfg.max_active = 64;
    if (s->cfg.slice_iterations <= 0) s->cfg.slice_iterations = 32;
    *out = s;
    return CWB_OK;
}

cwb_status cwb_server_submit(cwb_server* s, const cwb_config* cfg, const void* X, int32_t x_dtype, int64_t n, int32_t p,
                             const void* y, const double* w, const cwb_learner* bl, int32_t K, int64_t* id)
{
    set_error("");
    if (!s || !cfg || !X || !y || !bl || K <= 0 || n <= 0 || p <= 0 || !id) {
        set_error("cwb_server_submit: bad argument");
        return CWB_EINVAL;
    }
    if (cfg->iterations <= 0) { set_error("cwb_server_submit: cfg.iterations must be > 0"); return CWB_EINVAL; }
    Request r;
    r.id = s->next_id++;
    r.cfg = *cfg;
    r.cfg.stream = nullptr;              // every admitted fit runs on a stream of its own
    r.cfg.device = s->cfg.device;
    r.X = X;
    r.x_dtype = x_dtype;
    r.n = n;
    r.p = p;
    r.y = y;
    r.w = w;
    r.bl.assign(bl, bl + K);
    if (cfg->val_mask) {
        r.val_mask.assign(cfg->val_mask, cfg->val_mask + n);
        r.cfg.val_mask = nullptr;
    }
    r.footprint = estimate_footprint(r);
    if (r.footprint > s->cfg.hbm_budget_bytes) {
        set_error("cwb_server_submit: the request needs about " + std::to_string(r.footprint) +
                  " bytes, more than the server's budget");
        return CWB_EINVAL;
    }
    *id = r.id;
    s->pending.push_back(std::move(r));
    return CWB_OK;
}

cwb_status cwb_server_poll(cwb_server* s, int32_t wait, int64_t* done_ids, int32_t cap, int32_t* n_done)
{
    set_error("");
    if (!s || (cap > 0 && !done_ids)) { set_error("cwb_server_poll: bad argument"); return CWB_EINVAL; }
    int32_t got = 0;
    for (;;) {
        // admission: FIFO while the footprint fits the budget and a slot is free
        while (!s->pending.empty() && (int32_t)s->active.size() < s->cfg.max_active &&
               s->in_use + s->pending.front().footprint <= s->cfg.hbm_budget_bytes) {
            Request r = std::move(s->pending.front());
            s->pending.pop_front();
            Active a;
            if (!r.val_mask.empty()) r.cfg.val_mask = r.val_mask.data();
            // server fits interleave their iterations with other fits on the GPU: the three-kernel path
            // (a persistent kernel would hold every SM for its whole slice)
            cwb_status st = create_model(&r.cfg, r.X, r.x_dtype, r.n, r.p, r.y, r.w, r.bl.data(), (int32_t)r.bl.size(), 0,
                                         &a.m, kIterKernels, request_priority(r, r.index_bytes));
            if (st != CWB_OK) {
                s->failed[r.id] = cwb_last_error();
                s->completed += 1;
                if (got < cap) done_ids[got] = r.id;
                ++got;
                continue;
            }
            a.slice_done.assign(kSlicesInFlight, nullptr);
            for (auto& e : a.slice_done) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            s->in_use += r.footprint;
            a.req = std::move(r);
            s->active.push_back(std::move(a));
            s->admitted += 1;
        }
        // scheduling round: keep up to kSlicesInFlight slices queued per fit; retire finished fits
        for (size_t i = 0; i < s->active.size();) {
            Active& a = s->active[i];
            const int32_t M = a.req.cfg.iterations;
            slice_finished(a);
            if (a.queued >= M && a.in_flight == 0) {
                cwb_status st = cwb_synchronize(a.m);
                const int64_t id = a.req.id;
                retire(s, i, st == CWB_OK, st == CWB_OK ? "" : cwb_last_error());
                if (got < cap) done_ids[got] = id;
                ++got;
                continue;
            }
            while (a.queued < M && a.in_flight < kSlicesInFlight) {
                const int32_t slice = std::min(s->cfg.slice_iterations, M - a.queued);
                cwb_status st = cwb_fit(a.m, slice);
                if (st != CWB_OK) break;
                cudaEventRecord(a.slice_done[a.head], a.m->stream);
                a.head = (a.head + 1) % kSlicesInFlight;
                a.in_flight += 1;
                a.queued += slice;
            }
            ++i;
        }
        if (got > 0 || !wait || (s->active.empty() && s->pending.empty())) break;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (n_done) *n_done = std::min(got, cap);
    return CWB_OK;
}

cwb_status cwb_server_take(cwb_server* s, int64_t id, cwb_model** out)
{
    set_error("");
    if (!s || !out) { set_error("cwb_server_take: NULL argument"); return CWB_EINVAL; }
    *out = nullptr;
    auto f = s->failed.find(id);
    if (f != s->failed.end()) {
        set_error("request " + std::to_string(id) + " failed: " + f->second);
        s->failed.erase(f);
        return CWB_ESTATE;
    }
    auto it = s->finished.find(id);
    if (it == s->finished.end()) {
        set_error("request " + std::to_string(id) + " is not finished (or was already taken)");
        return CWB_ESTATE;
    }
    *out = it->second;
    s->finished.erase(it);
    return CWB_OK;
}

cwb_status cwb_server_stats(const cwb_server* s, int64_t* values, int32_t cap)
{
    set_error("");
    if (!s || (cap > 0 && !values)) { set_error("cwb_server_stats: bad argument"); return CWB_EINVAL; }
    const int64_t v[6] = {(int64_t)s->pending.size(), (int64_t)s->active.size(), s->admitted, s->completed,
                          (int64_t)s->in_use, (int64_t)s->cfg.hbm_budget_bytes};
    for (int32_t i = 0; i < cap && i < 6; ++i) values[i] = v[i];
    return CWB_OK;
}

void cwb_server_free(cwb_server* s)
{
    if (!s) return;
    while (!s->active.empty()) {
        cwb_synchronize(s->active.back().m);
        retire(s, s->active.size() - 1, false, "server freed");
    }
    for (auto& kv : s->finished) cwb_free(kv.second);
    delete s;
}

}  // extern "C"
