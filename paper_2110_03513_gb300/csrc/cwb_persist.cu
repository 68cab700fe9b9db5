// cwb_persist.cu -- plain CWB iterations as one persistent, cooperative kernel.
//
// One CTA per SM, all resident (cooperative launch).  An iteration of Algorithm 1 is two phases
// separated by grid barriers:
//
//   scatter  (binMatVec, Algorithm 2, with the row pass folded in)  CTA (binning group g, row
//            range) streams its tiles with TMA into a ring: the index box of the group's
//            binnings, and the rows' f, y (and w, the low parts of FP64 targets) and the index
//            column of the learner chosen last.  Two converter warps apply the pending update
//            f += nu v_k*[ind_k*], write the new f (group 0; f is double-buffered because both
//            groups read the same rows) and turn the weighted pseudo residuals w r into int32
//            fixed point (scale 2^S from a bound on max |w r| known before the pass, see
//            residual_bound).  Sixteen consumer warps add them into lane-private int32
//            shared-memory histograms, which are then added exactly into a bin-major int64
//            array u[bin][binning] (integer sums: independent of the order of the additions).
//   solve    (one CTA per learner)  s = Z^b^T u in float-float arithmetic from the exact sums,
//            theta = P s, the criterion Q = s^T (P G P - 2 P) s (= SSE - r^T W r), the update
//            table v_k = Z^b theta and max |v_k|.
//
// The barrier after the solve carries the argmin: CTA 0 waits for every CTA, takes the argmin
// over the criteria (ties: lowest k), writes the trace and the state, and releases the others
// with the selected learner.  The index boxes of the next iteration's first ring stages are
// issued while the solve runs (the index matrix never changes).  Every wait (mbarriers, grid
// barriers) is bounded: once a limit runs out the kernel sets kErrTimeout and runs to its end.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "cwb_internal.cuh"
#include "cwb_device.cuh"

namespace cwb {

namespace {

constexpr int kPWarps = 16;                          // consumer warps of the scatter phase
constexpr int kPConv = 2;                            // converter warps (row pass)
constexpr int kPLoader = kPWarps + kPConv;           // warp index of the loader
constexpr int kPThreads = (kPWarps + kPConv + 1) * 32;
constexpr int kPStageRows = 256;                     // rows per ring stage
constexpr int kPMaxStages = 8;
constexpr int kPSyncHead = 4;                        // sync words before the arrival flags
constexpr long long kBarrierCycles = 4000000000LL;   // ~2 s at 2 GHz per grid barrier

struct PArgs {
    DevState* state;
    unsigned* sync;           // [0] release word, [1] selected learner, [2..3] residual maxima, [4..] arrivals
    long long* ptime;         // [4] phase times (ns) and iterations, or NULL
    int iters;
    int64_t n, n_pad;
    const void* ind;
    const float* y;
    const float* y_lo;
    const float* w;
    float* fa;                // f double buffer [n_pad][2]: iteration i of the launch reads fa (i even) or fb
    float* fb;
    int loss;
    float nu_hi, nu_lo, wmax;
    int K, D, S, B;
    const int32_t* l_bin;
    const int32_t* l_d;
    const int32_t* l_nstar;
    float* v;                 // [K][S] update tables (channel 0 of the [2][K][S] array)
    float* vmax;              // [K] max |v_k|
    // scatter plan
    int FE, G, per_group, stages, nb;
    int64_t tiles;
    uint32_t ring_off, stage_stride, f_off, y_off, sel_off, w_off, ylo_off, q_off;
    uint32_t hist_off, vtab_off;
    long long* uacc;          // [2][nb][B] exact sums of the fixed-point histograms
    // solve
    const float* zb;          // [K][S][4]
    const int32_t* zcol;      // [K][S]
    const int32_t* crange;    // [K][D][2]
    const int32_t* toff;      // [K][D]
    const float* ztab;        // [K][4 S] column-major design (FP32 high parts)
    const float* ztab_lo;     // [K][4 S] low parts (float-float design)
    const float2* Pdf;        // [K][D][D] phase-0 cache, float-float pairs
    const float2* Adf;
    double* theta_it;         // [2][K][D]
    double* q_it;             // [2][K]
    // trace
    int32_t* tr_k;
    int32_t* tr_mode;
    double* tr_q;
    double* tr_theta;
    const int32_t* forced;
    int trace_cap;
    long long wait_cycles;    // limit of each ring wait (SM clocks); copies in flight are drained with kWaitCycles
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long globaltimer()
{
    long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier, arrival half: every CTA publishes that it reached generation gen + 1.
__device__ __forceinline__ void barrier_arrive(unsigned* sync, unsigned gen)
{
    __syncthreads();
    if (threadIdx.x == 0) st_release_gpu(sync + kPSyncHead + blockIdx.x, gen + 1u);
}

// CTA 0, warp 0: wait (bounded) until every CTA has arrived at generation gen + 1.
__device__ __forceinline__ void barrier_gather(unsigned* sync, unsigned gen, uint32_t* err)
{
    const long long deadline = clock64() + kBarrierCycles;
    const int lane = threadIdx.x & 31;
    for (;;) {
        bool mine = true;
        for (int c = lane; c < (int)gridDim.x; c += 32) mine &= ld_acquire_gpu(sync + kPSyncHead + c) >= gen + 1u;
        if (__all_sync(0xffffffffu, mine)) break;
        if (clock64() > deadline) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            break;
        }
    }
}

// Every CTA but 0, thread 0: wait (bounded) for CTA 0's release of generation gen + 1.
__device__ __forceinline__ void barrier_wait_release(unsigned* sync, unsigned gen, uint32_t* err)
{
    const long long deadline = clock64() + kBarrierCycles;
    while (ld_acquire_gpu(sync) < gen + 1u) {
        if (clock64() > deadline) {
            atomicOr(err, kErrTimeout);
            break;
        }
    }
}

template <typename IndT>
__device__ __forceinline__ void lds_ind4(const unsigned char* p, int out[4]);
template <>
__device__ __forceinline__ void lds_ind4<uint16_t>(const unsigned char* p, int out[4])
{
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    out[0] = u.x & 0xffff;
    out[1] = u.x >> 16;
    out[2] = u.y & 0xffff;
    out[3] = u.y >> 16;
}
template <>
__device__ __forceinline__ void lds_ind4<uint8_t>(const unsigned char* p, int out[4])
{
    const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
    out[0] = u & 0xff;
    out[1] = (u >> 8) & 0xff;
    out[2] = (u >> 16) & 0xff;
    out[3] = u >> 24;
}

template <typename IndT>
__global__ void __launch_bounds__(kPThreads, 1) k_iter(const __grid_constant__ CUtensorMap tmap, PArgs a)
{
    constexpr int U = 16 / sizeof(IndT);                   // rows per 16-byte unit
    constexpr int row_bytes = kPStageRows * (int)sizeof(IndT);
    constexpr int nunits = row_bytes / 16;                 // units of one binning per stage
    constexpr int UN = nunits / kPWarps;                   // units per consumer warp and stage
    constexpr int E = 128 / (int)sizeof(IndT);             // rows per 128-byte box row
    constexpr int RPL = kPStageRows / (kPConv * 32);       // rows per converter lane and stage
    static_assert(RPL == 4, "converter lanes handle four rows");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[kPMaxStages], ready[kPMaxStages], empty[kPMaxStages];
    __shared__ float red_f[kPThreads / 32];
    __shared__ int red_i[kPThreads / 32];
    __shared__ unsigned s_ksel;
    __shared__ DF s_s[kMaxD], s_t[kMaxD];
    __shared__ double s_th[kMaxD];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kPThreads / 32;
    int* hist = reinterpret_cast<int*>(smem + a.hist_off);
    float* vtab = reinterpret_cast<float*>(smem + a.vtab_off);
    uint32_t* err = &a.state->err;

    // this CTA's share of the scatter: group g, tile range [t_lo, t_hi)
    const int g = blockIdx.x % a.G, jg = blockIdx.x / a.G;
    const bool scat = jg < a.per_group;
    const int64_t t_lo = scat ? a.tiles * jg / a.per_group : 0;
    const int64_t t_hi = scat ? a.tiles * (jg + 1) / a.per_group : 0;
    const int ntiles = (int)(t_hi - t_lo);
    const int nst = a.stages;

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], kPConv);
            mbar_init(&empty[s], kPWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < a.nb * 32; i += blockDim.x) hist[i] = 0;
    // iteration state at launch (CTA 0 changes it only at the release of the first argmin)
    const DevState st0 = *a.state;
    __syncthreads();
    int m_loc = st0.m;
    bool pending = st0.m > st0.m_applied && st0.k_sel >= 0;
    int k_sel = st0.k_sel;
    uint32_t rprev_bits = st0.rprev_bits;
    const int cnt_log2 = st0.cnt_log2p;
    const long long wait_limit = a.wait_cycles;
    unsigned gen = 0;

    // loader bookkeeping: tiles are numbered continuously across iterations (T = iter * ntiles + it)
    const bool loader = warp == kPLoader && lane == 0;
    const uint32_t box_bytes = (uint32_t)(a.FE * row_bytes);
    auto tx_bytes = [&](bool pend) -> uint32_t {
        return box_bytes + kPStageRows * 12u + (pend ? (uint32_t)row_bytes : 0u) + (a.w ? kPStageRows * 4u : 0u) +
               (a.y_lo ? kPStageRows * 4u : 0u);
    };
    int64_t issued_idx = 0;           // tiles whose index box was issued (stage armed)
    int64_t issued_rows = 0;          // tiles whose row copies were issued
    auto stage_of = [&](int64_t T, int& s, uint32_t& ph) {
        s = (int)(T % nst);
        ph = (uint32_t)((T / nst) & 1);
    };
    auto issue_index = [&](int64_t T, uint32_t tx) -> bool {   // waits for the stage, arms it, copies the box
        int s;
        uint32_t ph;
        stage_of(T, s, ph);
        if (T >= nst && !mbar_wait(&empty[s], ph ^ 1u, clock64() + wait_limit)) return false;
        const int64_t row0 = (t_lo + (T % ntiles)) * kPStageRows;
        mbar_arrive_expect_tx(&full[s], tx);
        tma_load_3d(smem + a.ring_off + (size_t)s * a.stage_stride, &tmap, 0, g * a.FE, (int)(row0 / E), &full[s]);
        return true;
    };
    auto issue_rows = [&](int64_t T, const float* fcur, int b_sel) {
        int s;
        uint32_t ph;
        stage_of(T, s, ph);
        const int64_t row0 = (t_lo + (T % ntiles)) * kPStageRows;
        unsigned char* st = smem + a.ring_off + (size_t)s * a.stage_stride;
        bulk_load(st + a.f_off, fcur + 2 * row0, kPStageRows * 8, &full[s]);
        bulk_load(st + a.y_off, a.y + row0, kPStageRows * 4, &full[s]);
        if (b_sel >= 0)
            bulk_load(st + a.sel_off, static_cast<const IndT*>(a.ind) + (int64_t)b_sel * a.n_pad + row0, row_bytes, &full[s]);
        if (a.w) bulk_load(st + a.w_off, a.w + row0, kPStageRows * 4, &full[s]);
        if (a.y_lo) bulk_load(st + a.ylo_off, a.y_lo + row0, kPStageRows * 4, &full[s]);
    };
    bool load_ok = true;
    if (loader && ntiles > 0) {
        const uint32_t tx = tx_bytes(pending);
        for (int64_t T = 0; T < std::min<int64_t>(nst, ntiles); ++T) {
            issue_index(T, tx);
            ++issued_idx;
        }
    }

    long long t_ph0 = 0, t_ph1 = 0;
    const DF nu = {a.nu_hi, a.nu_lo};

    for (int iter = 0; iter < a.iters; ++iter) {
        if (a.ptime && blockIdx.x == 0 && tid == 0) t_ph0 = globaltimer();
        const int par = (m_loc + 1) & 1;      // parity of the iteration computed now (m_loc + 1)
        const float* fcur = (iter & 1) ? a.fb : a.fa;
        float* fnxt = (iter & 1) ? a.fa : a.fb;
        const int b_sel = pending ? a.l_bin[k_sel] : -1;
        const float vmax_sel = pending ? __ldcg(a.vmax + k_sel) : 0.0f;
        const int S_exp = fixed_scale(residual_bound(a.loss, pending, rprev_bits, vmax_sel, a.nu_hi, a.wmax), cnt_log2);
        const float scale = pow2f(S_exp);
        // the selected learner's update table, and its coefficients for the trace
        if (pending) {
            const float* vs = a.v + (int64_t)k_sel * a.S;
            for (int l = tid; l < a.S; l += blockDim.x) vtab[l] = __ldcg(vs + l);
            if (blockIdx.x == 0 && m_loc >= 1 && m_loc - 1 < a.trace_cap)
                for (int e = tid; e < a.D; e += blockDim.x)
                    a.tr_theta[((int64_t)2 * (m_loc - 1)) * a.D + e] = __ldcg(a.theta_it + (int64_t)k_sel * a.D + e);
        }
        __syncthreads();
        // ---------------------------------------------------------------- scatter (with the row pass)
        const int64_t T0 = (int64_t)iter * ntiles;
        float rmax = 0.0f;
        bool bad = false;
        if (warp == kPLoader) {
            if (loader && ntiles > 0) {
                // (the rows' f was written by other CTAs' generic stores before the last grid barrier)
                asm volatile("fence.proxy.async.global;" ::: "memory");
                // row tiles of the stages armed ahead, then the rest of this iteration's tiles
                for (; issued_rows < issued_idx; ++issued_rows) issue_rows(issued_rows, fcur, b_sel);
                const uint32_t tx = tx_bytes(pending);
                for (; load_ok && issued_idx < T0 + ntiles; ++issued_idx) {
                    if (!issue_index(issued_idx, tx)) {
                        load_ok = false;
                        atomicOr(err, kErrTimeout);
                        break;
                    }
                    issue_rows(issued_idx, fcur, b_sel);
                    ++issued_rows;
                }
            }
        } else if (warp >= kPWarps) {
            // converter warp c: rows [128 c, 128 c + 128) of every tile, four per lane
            const int c = warp - kPWarps;
            const int r0 = c * 128 + lane * RPL;
            for (int it = 0; it < ntiles; ++it) {
                int s;
                uint32_t ph;
                stage_of(T0 + it, s, ph);
                if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, clock64() + wait_limit))) {
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    break;
                }
                const unsigned char* st = smem + a.ring_off + (size_t)s * a.stage_stride;
                const float4 fa4 = *reinterpret_cast<const float4*>(st + a.f_off + r0 * 8);
                const float4 fb4 = *reinterpret_cast<const float4*>(st + a.f_off + r0 * 8 + 16);
                const float4 y4 = *reinterpret_cast<const float4*>(st + a.y_off + r0 * 4);
                const float4 w4 = a.w ? *reinterpret_cast<const float4*>(st + a.w_off + r0 * 4) : make_float4(1.f, 1.f, 1.f, 1.f);
                const float4 l4 = a.y_lo ? *reinterpret_cast<const float4*>(st + a.ylo_off + r0 * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
                DF fv[4] = {{fa4.x, fa4.y}, {fa4.z, fa4.w}, {fb4.x, fb4.y}, {fb4.z, fb4.w}};
                if (pending) {
                    int idx[4];
                    lds_ind4<IndT>(st + a.sel_off + r0 * (int)sizeof(IndT), idx);
#pragma unroll
                    for (int t = 0; t < 4; ++t) fv[t] = df_add(fv[t], df_mul_f(nu, vtab[idx[t]]));
                }
                const int64_t row = (t_lo + it) * kPStageRows + r0;
                const float yv[4] = {y4.x, y4.y, y4.z, y4.w}, wv[4] = {w4.x, w4.y, w4.z, w4.w},
                            lv[4] = {l4.x, l4.y, l4.z, l4.w};
                int q[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    float r = 0.0f;
                    if (row + t < a.n) r = wv[t] * neg_gradient(a.loss, yv[t], lv[t], fv[t]);
                    if (!(fabsf(r) <= 3.0e38f)) {
                        bad = true;
                        r = 0.0f;
                    }
                    rmax = fmaxf(rmax, fabsf(r));
                    q[t] = __float2int_rn(r * scale);
                }
                *reinterpret_cast<int4*>(const_cast<unsigned char*>(st) + a.q_off + r0 * 4) = make_int4(q[0], q[1], q[2], q[3]);
                if (g == 0) {
                    *reinterpret_cast<float4*>(fnxt + 2 * row) = make_float4(fv[0].hi, fv[0].lo, fv[1].hi, fv[1].lo);
                    *reinterpret_cast<float4*>(fnxt + 2 * row + 4) = make_float4(fv[2].hi, fv[2].lo, fv[3].hi, fv[3].lo);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&ready[s]);
            }
        } else {
            const int f = lane;
            const bool active = f < a.FE && g * a.FE + f < a.B;
            int* hf = hist + f;
            for (int it = 0; it < ntiles; ++it) {
                int s;
                uint32_t ph;
                stage_of(T0 + it, s, ph);
                if (!__all_sync(0xffffffffu, mbar_wait(&ready[s], ph, clock64() + wait_limit))) {
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    break;
                }
                const unsigned char* st = smem + a.ring_off + (size_t)s * a.stage_stride;
                const int* q_st = reinterpret_cast<const int*>(st + a.q_off);
                uint4 raw[UN];
                int rv[UN][U];
                if (active) {
#pragma unroll
                    for (int k = 0; k < UN; ++k) {
                        // unit `pos` of binning f sits in 128-byte box row R = (pos / 8) FE + f at the
                        // 16-byte slot (pos % 8) ^ (R % 8) (128-byte swizzle)
                        const int pos = warp * UN + k;
                        const int R = (pos >> 3) * a.FE + f;
                        raw[k] = *reinterpret_cast<const uint4*>(st + R * 128 + (((pos & 7) ^ (R & 7)) << 4));
#pragma unroll
                        for (int t4 = 0; t4 < U / 4; ++t4) {
                            const int4 r4 = reinterpret_cast<const int4*>(q_st + pos * U)[t4];
                            rv[k][4 * t4] = r4.x;
                            rv[k][4 * t4 + 1] = r4.y;
                            rv[k][4 * t4 + 2] = r4.z;
                            rv[k][4 * t4 + 3] = r4.w;
                        }
                    }
                }
                // the stage is free as soon as its values are in registers
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                if (active) {
#pragma unroll
                    for (int k = 0; k < UN; ++k) {
                        int idx[U];
                        unpack16<IndT>(raw[k], idx);
#pragma unroll
                        for (int t = 0; t < U; ++t) atomicAdd(hf + (idx[t] << 5), rv[k][t]);
                    }
                }
            }
        }
        // the new f is read by the next iteration's bulk copies (async proxy)
        if (warp >= kPWarps && warp < kPLoader && g == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        // residual maximum of this iteration (the converters' rows)
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        const bool anybad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            red_f[warp] = rmax;
            red_i[warp] = anybad ? 1 : 0;
        }
        __syncthreads();
        if (tid == 0) {
            float mx = 0.0f;
            int b = 0;
            for (int w2 = 0; w2 < nwarps; ++w2) {
                mx = fmaxf(mx, red_f[w2]);
                b |= red_i[w2];
            }
            if (scat) atomicMax(&a.sync[2 + par], __float_as_uint(mx));
            if (b) atomicOr(err, kErrNonFinite);
        }
        if (scat) {
            // exact int64 sums, bin-major u[bin][binning]; a warp adds one bin of 32 binnings
            // (coalesced), CTAs start at different bins so that they do not queue on the same
            // lines; the histogram is cleared for the next iteration as it is read
            long long* u_par = a.uacc + (int64_t)par * a.nb * a.B;
            const int off = (int)((int64_t)jg * a.nb / a.per_group);
            for (int e = tid; e < a.nb * 32; e += blockDim.x) {
                const int f = e & 31;
                int l = (e >> 5) + off;
                if (l >= a.nb) l -= a.nb;
                const int hv = hist[l * 32 + f];
                hist[l * 32 + f] = 0;
                if (hv != 0 && f < a.FE && g * a.FE + f < a.B)
                    atomicAdd(reinterpret_cast<unsigned long long*>(u_par + (int64_t)l * a.B + g * a.FE + f),
                              (unsigned long long)(long long)hv);
            }
        }
        // the next iteration's first index boxes while the solve runs
        if (loader && ntiles > 0 && iter + 1 < a.iters && load_ok) {
            const int64_t T1 = (int64_t)(iter + 1) * ntiles;
            const uint32_t tx = tx_bytes(true);
            for (; issued_idx < T1 + std::min<int64_t>(nst, ntiles); ++issued_idx) {
                if (!issue_index(issued_idx, tx)) {
                    load_ok = false;
                    atomicOr(err, kErrTimeout);
                    break;
                }
            }
        }
        // ---------------------------------------------------------------- barrier: u, f and the maximum complete
        barrier_arrive(a.sync, gen);
        if (blockIdx.x == 0) {
            if (warp == 0) barrier_gather(a.sync, gen, err);
            __syncthreads();
            if (tid == 0) st_release_gpu(a.sync, gen + 1u);
        } else if (tid == 0) {
            barrier_wait_release(a.sync, gen, err);
        }
        gen += 1u;
        __syncthreads();
        if (a.ptime && blockIdx.x == 0 && tid == 0) t_ph1 = globaltimer();
        // ---------------------------------------------------------------- solve
        {
            // clear the other parity's sums (the next iteration's) and maximum
            long long* u_next = a.uacc + (int64_t)(par ^ 1) * a.nb * a.B;
            for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < (int64_t)a.nb * a.B; e += (int64_t)gridDim.x * blockDim.x)
                u_next[e] = 0;
            if (blockIdx.x == 0 && tid == 0) a.sync[2 + (par ^ 1)] = 0u;
            const float inv_scale = pow2f(-S_exp);
            const long long* u_par = a.uacc + (int64_t)par * a.nb * a.B;
            for (int k = blockIdx.x; k < a.K; k += gridDim.x) {
                const int b = a.l_bin[k], d = a.l_d[k], ns = a.l_nstar[k];
                // s_j = sum over the bins of column j's range of z_lj u_l: half a warp per column
                {
                    const int hw = warp * 2 + (lane >> 4), hl = lane & 15;
                    const unsigned hmask = (lane >> 4) ? 0xffff0000u : 0x0000ffffu;
                    for (int j = hw; j < d; j += 2 * nwarps) {
                        const int lo = __ldg(a.crange + ((int64_t)k * a.D + j) * 2);
                        const int hi = __ldg(a.crange + ((int64_t)k * a.D + j) * 2 + 1);
                        const int off = __ldg(a.toff + (int64_t)k * a.D + j);
                        const float* zh = a.ztab + (int64_t)k * kMaxNnz * a.S + off - lo;
                        const float* zl = a.ztab_lo + (int64_t)k * kMaxNnz * a.S + off - lo;
                        DF acc = {0.0f, 0.0f};
                        for (int l = lo + hl; l < hi; l += 16) {
                            const DF ul = df_scale(df_of_ll(__ldcg(u_par + (int64_t)l * a.B + b)), inv_scale);
                            acc = df_add(acc, df_mul(DF{__ldg(zh + l), __ldg(zl + l)}, ul));
                        }
                        for (int o = 8; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o, hmask));
                        if (hl == 0) s_s[j] = acc;
                    }
                }
                __syncthreads();
                // theta = P s and t = A s (eight lanes per row), Q = s . t
                const float2* Pk = a.Pdf + (int64_t)k * a.D * a.D;
                const float2* Ak = a.Adf + (int64_t)k * a.D * a.D;
                for (int base = 0; base < 2 * d * 8; base += blockDim.x) {
                    const int e = base + tid;
                    const bool valid = e < 2 * d * 8;
                    const int mat = (valid && e >= d * 8) ? 1 : 0;
                    const int r = e - mat * d * 8;
                    const int i = r >> 3, qq = r & 7;
                    const float2* Mx = mat ? Ak : Pk;
                    DF p = {0.0f, 0.0f};
                    if (valid)
                        for (int j = qq; j < d; j += 8) {
                            const float2 mij = __ldg(Mx + i * a.D + j);
                            p = df_add(p, df_mul(DF{mij.x, mij.y}, s_s[j]));
                        }
#pragma unroll 1
                    for (int o = 1; o < 8; o <<= 1) p = df_add(p, df_shfl_xor(p, o));
                    if (valid && qq == 0) {
                        if (mat) s_t[i] = df_mul(p, s_s[i]);
                        else s_th[i] = (double)p.hi + (double)p.lo;
                    }
                }
                __syncthreads();
                if (warp == 0) {
                    DF x = {0.0f, 0.0f};
                    for (int i = lane; i < d; i += 32) x = df_add(x, s_t[i]);
#pragma unroll 1
                    for (int o = 16; o > 0; o >>= 1) x = df_add(x, df_shfl_xor(x, o));
                    if (lane == 0) a.q_it[k] = (double)x.hi + (double)x.lo;
                }
                for (int i = tid; i < a.D; i += blockDim.x) a.theta_it[(int64_t)k * a.D + i] = i < d ? s_th[i] : 0.0;
                // update table v_k = Z^b theta (FP32) and max |v_k|
                float vm = 0.0f;
                for (int l = tid; l < ns; l += blockDim.x) {
                    const int c0 = __ldg(a.zcol + (int64_t)k * a.S + l);
                    const float4 z = __ldg(reinterpret_cast<const float4*>(a.zb) + (int64_t)k * a.S + l);
                    float acc = 0.0f;
                    if (c0 < a.D) acc = fmaf(z.x, (float)s_th[c0], acc);
                    if (c0 + 1 < a.D) acc = fmaf(z.y, (float)s_th[c0 + 1], acc);
                    if (c0 + 2 < a.D) acc = fmaf(z.z, (float)s_th[c0 + 2], acc);
                    if (c0 + 3 < a.D) acc = fmaf(z.w, (float)s_th[c0 + 3], acc);
                    a.v[(int64_t)k * a.S + l] = acc;
                    vm = fmaxf(vm, fabsf(acc));
                }
                for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
                if (lane == 0) red_f[warp] = vm;
                __syncthreads();
                if (tid == 0) {
                    float mx = 0.0f;
                    for (int w2 = 0; w2 < nwarps; ++w2) mx = fmaxf(mx, red_f[w2]);
                    a.vmax[k] = mx;
                }
                __syncthreads();
            }
        }
        // ---------------------------------------------------------------- barrier with the argmin
        barrier_arrive(a.sync, gen);
        if (blockIdx.x == 0) {
            if (warp == 0) {
                barrier_gather(a.sync, gen, err);
                const long long kInf = order_key(INFINITY);
                Best2 x = {kInf, kInf, -1};
                bool badq = false;
#pragma unroll 1
                for (int kk = lane; kk < a.K; kk += 32) {
                    const long long qt = __ldcg(reinterpret_cast<const long long*>(a.q_it) + kk);
                    long long key = (qt & 0x7fffffffffffffffLL) == 0 ? 0LL : order_key(__longlong_as_double(qt));
                    if ((qt & 0x7ff0000000000000LL) == 0x7ff0000000000000LL) {
                        badq = true;
                        key = kInf;
                    }
                    x = best2_merge(x, Best2{key, kInf, kk});
                }
#pragma unroll 1
                for (int o = 16; o > 0; o >>= 1) x = best2_merge(x, best2_shfl(x, o));
                badq = __any_sync(0xffffffffu, badq);
                if (lane == 0) {
                    const int it = m_loc;
                    const bool trace_ok = it < a.trace_cap;
                    int kb = x.k1 < 0 ? 0 : x.k1;
                    if (trace_ok && a.forced) {
                        const int fk = a.forced[it];
                        if (fk >= 0 && fk < a.K) kb = fk;
                    }
                    DevState* S_ = a.state;
                    if (trace_ok) {
                        a.tr_k[2 * it] = kb;
                        a.tr_k[2 * it + 1] = -1;
                        a.tr_mode[it] = kModeCWB;
                        a.tr_q[2 * it] = key_value(x.q1);
                        a.tr_q[2 * it + 1] = key_value(x.q2);
                    } else {
                        atomicOr(err, kErrIndex);
                    }
                    if (badq) atomicOr(err, kErrNonFinite);
                    if (pending) S_->m_applied = m_loc;
                    S_->k_sel = kb;
                    S_->k_cor = -1;
                    S_->pend_mode = kModeCWB;
                    S_->m = it + 1;
                    S_->fix_exp = S_exp;
                    S_->resid_path = 1;
                    s_ksel = (unsigned)kb;
                    a.sync[1] = (unsigned)kb;
                    st_release_gpu(a.sync, gen + 1u);
                }
            }
        } else if (tid == 0) {
            barrier_wait_release(a.sync, gen, err);
            s_ksel = ld_acquire_gpu(a.sync + 1);
        }
        gen += 1u;
        __syncthreads();
        k_sel = (int)s_ksel;
        if (k_sel < 0 || k_sel >= a.K) k_sel = 0;
        rprev_bits = __ldcg(a.sync + 2 + par);
        m_loc += 1;
        pending = true;
        if (a.ptime && blockIdx.x == 0 && tid == 0) {
            const long long t2 = globaltimer();
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ptime + 1), (unsigned long long)(t_ph1 - t_ph0));
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ptime + 2), (unsigned long long)(t2 - t_ph1));
            atomicAdd(reinterpret_cast<unsigned long long*>(a.ptime + 3), 1ull);
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.state->rprev_bits = rprev_bits;
        a.state->rmax_bits[0] = 0u;
        a.state->rmax_bits[1] = 0u;
    }
    // no bulk copy may be in flight when the CTA retires (only possible after a wait ran out)
    if (loader && ntiles > 0 && !load_ok) {
        const long long d2 = clock64() + kWaitCycles;
        for (int64_t T = std::max<int64_t>(0, issued_idx - nst); T < issued_idx; ++T) {
            int s;
            uint32_t ph;
            stage_of(T, s, ph);
            mbar_wait(&full[s], ph, d2);
        }
    }
}

// Residuals of the current model, w r = w (-dL/df) at f (the scatter input of the most recent
// iteration on the persistent path, before its fixed-point rounding).
__global__ void k_resid_now(int64_t n, int loss, const float* __restrict__ y, const float* __restrict__ y_lo,
                            const float* __restrict__ w, const float* __restrict__ f, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (w ? w[i] : 1.0f) * neg_gradient(loss, y[i], y_lo ? y_lo[i] : 0.0f, DF{f[2 * i], f[2 * i + 1]});
}

template <typename IndT>
__global__ void __launch_bounds__(512) k_pcount(const IndT* __restrict__ ind, int64_t n, int64_t n_pad, int B, int FE,
                                                int G, int per_group, int64_t tiles, int nb, DevState* state)
{
    extern __shared__ int hc[];           // [nb][32]
    const int g = blockIdx.x % G, jg = blockIdx.x / G;
    if (jg >= per_group) return;
    const int64_t r_lo = tiles * jg / per_group * kPStageRows;
    const int64_t r_hi = std::min<int64_t>(n, tiles * (jg + 1) / per_group * kPStageRows);
    for (int i = threadIdx.x; i < nb * 32; i += blockDim.x) hc[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int b = g * FE + lane;
    if (lane < FE && b < B)
        for (int64_t q = r_lo + warp; q < r_hi; q += nw) atomicAdd(&hc[(int)ind[(int64_t)b * n_pad + q] * 32 + lane], 1);
    __syncthreads();
    int mx = 0;
    for (int i = threadIdx.x; i < nb * 32; i += blockDim.x) mx = max(mx, hc[i]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) atomicMax(&state->cnt_max[1], mx);
}

__global__ void k_pcount_log2(DevState* state)
{
    if (threadIdx.x != 0) return;
    const int c = state->cnt_max[1];
    int l = 0;
    while ((1 << l) < c && l < 30) ++l;
    state->cnt_log2p = l;
}

// max |w r| of the residuals at the current model (the bound's input before the first
// persistent iteration) and the largest weight.
__global__ void k_init_rmax(int64_t n, int loss, const float* __restrict__ y, const float* __restrict__ y_lo,
                            const float* __restrict__ w, const float* __restrict__ f, uint32_t* out /* [2] */)
{
    float rm = 0.0f, wm = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float wv = w ? w[i] : 1.0f;
        const float r = wv * neg_gradient(loss, y[i], y_lo ? y_lo[i] : 0.0f, DF{f[2 * i], f[2 * i + 1]});
        if (fabsf(r) <= 3.0e38f) rm = fmaxf(rm, fabsf(r));
        wm = fmaxf(wm, wv);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], __float_as_uint(rm));
        atomicMax(&out[1], __float_as_uint(wm));
    }
}

int num_sms_p(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

using EncodeTiledFnP = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

// Plans the persistent path for plain CWB models whose histograms fit one CTA's shared memory
// beside a ring of at least three stages; sets m->persist_ok.  Allocates its buffers (the second
// f buffer, the exact sums, the barrier words) and runs the counting pass for the fixed-point
// scale.
// The inputs of residual_bound known at creation: the largest weight (m->wmax) and, before the
// first iteration, max |w r| of the residuals at the offset (the state's rprev_bits).
cwb_status init_residual_bound(cwb_model* m)
{
    cudaStream_t s = m->stream;
    const int sms = num_sms_p(m->device);
    uint32_t* mx = nullptr;
    if (cudaMallocAsync((void**)&mx, sizeof(uint32_t) * 2, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation for the residual bound failed");
        return CWB_ENOMEM;
    }
    uint32_t mx_h[2] = {0u, 0u};
    DevState st;
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(uint32_t) * 2, s);
    if (e == cudaSuccess) {
        k_init_rmax<<<std::max(1, std::min(4 * sms, (int)((m->n + 255) / 256))), 256, 0, s>>>(
            m->n, m->cfg.loss, m->y, m->y_lo, m->w, m->f, mx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mx_h, mx, sizeof(mx_h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, m->state, sizeof(st), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(mx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "residual bound at creation");
    float wmax_f = 1.0f;
    std::memcpy(&wmax_f, &mx_h[1], sizeof(float));
    m->wmax = wmax_f > 0.0f ? wmax_f : 1.0f;
    if (st.m == 0 && st.rprev_bits == 0u) {
        CWB_CUDA_TRY(cudaMemcpyAsync(&m->state->rprev_bits, &mx_h[0], sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        CWB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return CWB_OK;
}

cwb_status plan_persistent(cwb_model* m)
{
    m->persist_ok = false;
    // opt-in (CWB_ITER_MODE=persistent): on the 1M x 50 workload it measured slower than the
    // three-kernel path (see the design notes), so auto mode keeps the kernels
    if (m->accel || m->iter_mode != kIterPersistent) return CWB_OK;
    const int sms = num_sms_p(m->device);
    int optin = 0, coop = 0;
    CWB_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    CWB_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, m->device));
    if (!coop) return CWB_OK;
    PersistPlan P{};
    const int elem = m->ind_bytes;
    P.nb = (m->nstar_max + 3) & ~3;
    const int F = 32;
    P.G = (m->B + F - 1) / F;
    P.FE = (m->B + P.G - 1) / P.G;
    P.per_group = sms / P.G;
    if (P.per_group < 1) return CWB_OK;
    P.tiles = (m->n + kPStageRows - 1) / kPStageRows;
    // stage: index box (1024-byte aligned for the 128-byte swizzle), f, y, the selected index
    // column, w, the low parts of y, and the fixed-point residuals
    const uint32_t box = (uint32_t)(P.FE * kPStageRows * elem);
    uint32_t o = (box + 1023u) / 1024u * 1024u;
    P.f_off = o;
    o += kPStageRows * 8;
    P.y_off = o;
    o += kPStageRows * 4;
    P.sel_off = o;
    o += kPStageRows * elem;
    P.w_off = o;
    if (m->w) o += kPStageRows * 4;
    P.ylo_off = o;
    if (m->y_lo) o += kPStageRows * 4;
    P.q_off = o;
    o += kPStageRows * 4;
    P.stage_stride = (o + 1023u) / 1024u * 1024u;
    const size_t hist = (size_t)P.nb * 32 * 4;
    const size_t vtab = ((size_t)m->nstar_max * 4 + 15) / 16 * 16;
    const size_t static_smem = 4096;
    const long long budget = (long long)optin - 1024 - (long long)static_smem - (long long)hist - (long long)vtab;
    if (budget < 3 * (long long)P.stage_stride) return CWB_OK;
    P.stages = (int)std::min<long long>(kPMaxStages, budget / (long long)P.stage_stride);
    P.ring_off = 0;
    P.hist_off = P.stages * P.stage_stride;
    P.vtab_off = (uint32_t)(P.hist_off + hist);
    P.smem = (size_t)P.vtab_off + vtab + 1024;
    P.ctas = sms;
    // every CTA must be resident at once
    const void* kf = m->ind_bytes == 1 ? (const void*)k_iter<uint8_t> : (const void*)k_iter<uint16_t>;
    CWB_CUDA_TRY(allow_max_dynamic_smem(kf, m->device));
    int per_sm = 0;
    CWB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, kPThreads, P.smem));
    if (per_sm < 1) return CWB_OK;
    // tensor map of the index matrix [B][n_pad]: {E rows, B binnings, n_pad / E}, box of a group's binnings
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return CWB_OK;
    }
    const int E = 128 / elem;
    cuuint64_t dims[3] = {(cuuint64_t)E, (cuuint64_t)m->B, (cuuint64_t)(m->n_pad / E)};
    cuuint64_t strides[2] = {(cuuint64_t)m->n_pad * elem, 128};
    cuuint32_t boxd[3] = {(cuuint32_t)E, (cuuint32_t)P.FE, (cuuint32_t)(kPStageRows / E)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = reinterpret_cast<EncodeTiledFnP>(fn)(
        &m->pmap, elem == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, m->ind, dims, strides, boxd,
        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return CWB_OK;
    // buffers
    cudaStream_t s = m->stream;
    const size_t sync_words = kPSyncHead + (size_t)sms;
    CWB_TRY(dev_alloc((void**)&m->f2, sizeof(float) * 2 * m->n_pad, s));
    CWB_TRY(dev_alloc((void**)&m->uacc, sizeof(long long) * 2 * (size_t)P.nb * m->B, s));
    CWB_TRY(dev_alloc((void**)&m->gbar, sizeof(unsigned) * sync_words, s));
    CWB_TRY(dev_alloc((void**)&m->ptime, sizeof(long long) * 4, s));
    CWB_CUDA_TRY(cudaMemsetAsync(m->uacc, 0, sizeof(long long) * 2 * (size_t)P.nb * m->B, s));
    CWB_CUDA_TRY(cudaMemsetAsync(m->ptime, 0, sizeof(long long) * 4, s));
    m->uacc_clean = true;
    // counting pass: the largest per-CTA bin count bounds the fixed-point scale
    CWB_CUDA_TRY(cudaMemsetAsync(&m->state->cnt_max[1], 0, sizeof(int), s));
    const size_t csm = sizeof(int) * (size_t)P.nb * 32;
    const void* kc = m->ind_bytes == 1 ? (const void*)k_pcount<uint8_t> : (const void*)k_pcount<uint16_t>;
    CWB_CUDA_TRY(allow_max_dynamic_smem(kc, m->device));
    if (m->ind_bytes == 1)
        k_pcount<uint8_t><<<sms, 512, csm, s>>>((const uint8_t*)m->ind, m->n, m->n_pad, m->B, P.FE, P.G, P.per_group, P.tiles,
                                               P.nb, m->state);
    else
        k_pcount<uint16_t><<<sms, 512, csm, s>>>((const uint16_t*)m->ind, m->n, m->n_pad, m->B, P.FE, P.G, P.per_group,
                                                P.tiles, P.nb, m->state);
    k_pcount_log2<<<1, 32, 0, s>>>(m->state);
    CWB_TRY(init_residual_bound(m));
    DevState st;
    CWB_CUDA_TRY(cudaMemcpyAsync(&st, m->state, sizeof(st), cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    if (st.cnt_log2p > 13) return CWB_OK;   // heavily skewed bins: the kernel path (FP32 fallback) handles them
    m->pplan = P;
    m->persist_ok = true;
    return CWB_OK;
}

cwb_status launch_persistent(cwb_model* m, int32_t iters)
{
    const PersistPlan& P = m->pplan;
    if (!m->uacc_clean) {
        // iterations of the kernel path ran since: the exact sums of both parities start from zero
        CWB_CUDA_TRY(cudaMemsetAsync(m->uacc, 0, sizeof(long long) * 2 * (size_t)P.nb * m->B, m->stream));
        m->uacc_clean = true;
    }
    PArgs a{};
    a.state = m->state;
    a.sync = m->gbar;
    a.ptime = m->prof_on ? m->ptime : nullptr;
    a.iters = iters;
    a.n = m->n;
    a.n_pad = m->n_pad;
    a.ind = m->ind;
    a.y = m->y;
    a.y_lo = m->y_lo;
    a.w = m->w;
    a.fa = m->f;
    a.fb = m->f2;
    a.loss = m->cfg.loss;
    a.nu_hi = (float)m->cfg.nu;
    a.nu_lo = (float)(m->cfg.nu - (double)a.nu_hi);
    a.wmax = (float)m->wmax;
    a.K = m->K;
    a.D = m->d_max;
    a.S = m->nstar_max;
    a.B = m->B;
    a.l_bin = m->l_bin;
    a.l_d = m->l_d;
    a.l_nstar = m->l_nstar;
    a.v = m->v;
    a.vmax = m->vmax;
    a.FE = P.FE;
    a.G = P.G;
    a.per_group = P.per_group;
    a.stages = P.stages;
    a.nb = P.nb;
    a.tiles = P.tiles;
    a.ring_off = P.ring_off;
    a.stage_stride = P.stage_stride;
    a.f_off = P.f_off;
    a.y_off = P.y_off;
    a.sel_off = P.sel_off;
    a.w_off = P.w_off;
    a.ylo_off = P.ylo_off;
    a.q_off = P.q_off;
    a.hist_off = P.hist_off;
    a.vtab_off = P.vtab_off;
    a.uacc = m->uacc;
    a.zb = m->zb;
    a.zcol = m->zcol;
    a.crange = m->crange;
    a.toff = m->toff;
    a.ztab = m->ztab;
    a.ztab_lo = m->ztab_lo;
    a.Pdf = m->Pdf;
    a.Adf = m->Adf;
    a.theta_it = m->theta_it;
    a.q_it = m->q_it;
    a.tr_k = m->tr_k;
    a.tr_mode = m->tr_mode;
    a.tr_q = m->tr_q;
    a.tr_theta = m->tr_theta;
    a.forced = m->forced;
    a.trace_cap = m->trace_cap;
    a.wait_cycles = m->wait_cycles;
    // barrier words, arrival flags and the two residual maxima start from zero
    CWB_CUDA_TRY(cudaMemsetAsync(m->gbar, 0, sizeof(unsigned) * (kPSyncHead + (size_t)P.ctas), m->stream));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.ctas, 1, 1);
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = m->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = m->ind_bytes == 1 ? cudaLaunchKernelEx(&cfg, k_iter<uint8_t>, m->pmap, a)
                                      : cudaLaunchKernelEx(&cfg, k_iter<uint16_t>, m->pmap, a);
    if (e != cudaSuccess) return cuda_status(e, "persistent iteration kernel");
    if (iters & 1) {
        // the last iteration wrote the other f buffer: it becomes the model's f (graphs of the kernel
        // path hold the old pointer and are captured again)
        std::swap(m->f, m->f2);
        release_graphs(m);
    }
    return CWB_OK;
}

// Phase times of the persistent kernel since the last reset (ms): 0 (the row pass runs inside the
// scatter phase), scatter with the row pass, solve with its barrier and the argmin.
cwb_status persistent_profile(cwb_model* m, double ms[3], int64_t* iters, bool reset)
{
    long long t[4] = {0, 0, 0, 0};
    CWB_CUDA_TRY(cudaMemcpyAsync(t, m->ptime, sizeof(t), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < 3; ++i) ms[i] = t[i] * 1e-6;
    *iters = t[3];
    if (reset) CWB_CUDA_TRY(cudaMemsetAsync(m->ptime, 0, sizeof(t), m->stream));
    return CWB_OK;
}

// w r at the current model (the scatter input of the latest persistent iteration, unrounded) into out.
cwb_status persistent_residuals(cwb_model* m, float* out_dev)
{
    const int sms = num_sms_p(m->device);
    k_resid_now<<<std::max(1, std::min(4 * sms, (int)((m->n + 255) / 256))), 256, 0, m->stream>>>(
        m->n, m->cfg.loss, m->y, m->y_lo, m->w, m->f, out_dev);
    CWB_CUDA_TRY(cudaGetLastError());
    return CWB_OK;
}

}  // namespace cwb
