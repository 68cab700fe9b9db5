// cwb_iter.cu -- one boosting iteration on the device, no host round trip.
//
//   k_rows     apply the previous iteration's update (Algorithm 1: f += nu b_k;
//              Algorithm 3: f = g + nu b_k, h += eta_m b_cor) and compute the
//              pseudo residuals of the next iteration (and the error-corrected
//              residuals c for ACWB), scaled by the observation weights.  For
//              HCWB the update pass also reduces the validation risk and
//              decides the next mode (Algorithm 4).
//   k_scatter  binMatVec (Algorithm 2): u_k[l] = sum_{i: ind_k,i = l} w_i r_i for
//              every binning, shared-memory histograms, one lane per binning.
//   k_solve    per learner: u -> s = Z^b^T u -> theta = P s -> criterion
//              Q_k = theta^T G theta - 2 theta^T s = SSE_k - r^T W r (float-float
//              from the cached FP64 matrices) and the update table v_k = Z^b theta;
//              the last CTA takes the argmin (ties: lowest k) and writes the trace.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <string>
#include <type_traits>

#include <cooperative_groups.h>
#include <cuda.h>

#include "cwb_internal.cuh"
#include "cwb_device.cuh"

namespace cwb {

namespace {

constexpr int kRowThreads = 256;
constexpr int kScatterWarps = 16;      // consumer warps of a scatter CTA
constexpr int kScatterThreads = (kScatterWarps + 2) * 32;   // + 1 loader warp + 1 converter warp
constexpr int kStageRows = 256;        // rows per pipeline stage (tile)
constexpr int kGraphIters = 32;

enum { kRowsFused = 0, kRowsUpdate = 1, kRowsResid = 2 };


struct RowArgs {
    DevState* state;
    const void* ind;
    int64_t n, n_tr, n_pad;
    const float* y;
    const float* y_lo;    // low part of FP64 targets (NULL for FP32 targets)
    const float* w;
    float* f;             // [n_pad][2] hi, lo
    float* h;             // [n_pad][2] hi, lo (ACWB/HCWB)
    float* c;
    float* rw;
    const float* v;       // [2][K][S] fitted values Z^b theta of every learner per bin
    const int32_t* l_bin;
    int S, K, D;
    const double* theta_it;   // [2][K][D] coefficients of the last solve
    double* tr_theta;         // [cap][2][D] trace of the selected coefficients
    int trace_cap;
    int loss;
    double nu, gamma;
    float nu_hi, nu_lo;       // nu as a float-float pair (rounded on the host)
    int hybrid;
    int patience;
    double* risk_part;
    int direct;               // plain CWB: write w r as int32 fixed point (scale from residual_bound)
    float wmax;               // largest observation weight (1 without weights)
    const float* vmax;        // [K] max |v_k| of the last solve
};

__device__ __forceinline__ float get4(const float4& v, int t)
{
    return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

__device__ __forceinline__ void set4(float4& v, int t, float x)
{
    if (t == 0) v.x = x; else if (t == 1) v.y = x; else if (t == 2) v.z = x; else v.w = x;
}

__device__ __forceinline__ void store_df4(float* p, int64_t i4, const DF v[4])
{
    *reinterpret_cast<float4*>(p + 2 * i4) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    *reinterpret_cast<float4*>(p + 2 * i4 + 4) = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
}

// Inputs of one group of 4 rows that do not depend on the iteration state (the low parts of
// FP64 targets and the weights, absent in the common case, are loaded with the selected bins).
struct RowIn {
    DF f[4], h[4];
    float4 y;
};

// need_y: targets (residual passes and the validation risk)
// Loads through L2 (ld.global.cg): the first pass's loads may be issued before the kernel waits
// for its predecessor, and only L2 is coherent with what earlier kernels wrote.
__device__ __forceinline__ void load_df4_cg(const float* p, int64_t i4, DF out[4])
{
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p + 2 * i4));
    const float4 b = __ldcg(reinterpret_cast<const float4*>(p + 2 * i4 + 4));
    out[0] = {a.x, a.y};
    out[1] = {a.z, a.w};
    out[2] = {b.x, b.y};
    out[3] = {b.z, b.w};
}

template <bool ACC>
__device__ __forceinline__ void load_row_in(const RowArgs& a, int64_t i4, RowIn& in, bool need_y)
{
    load_df4_cg(a.f, i4, in.f);
    if (ACC && a.h) load_df4_cg(a.h, i4, in.h);
    else for (int t = 0; t < 4; ++t) in.h[t] = {0.0f, 0.0f};
    in.y = need_y ? __ldcg(reinterpret_cast<const float4*>(a.y + i4)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// A thread handles row_groups(ACC) groups of 4 rows per pass (blockDim.x * 4 rows apart); the
// loads of a pass are all issued before any of its arithmetic, and those of the first pass
// before the iteration state is read, so a pass costs about one memory round trip.  One group
// for every model: plain CWB models with two groups per thread (half the threads) ran 4 % slower
// per iteration at n = 1M, with four 20 % slower.
__host__ __device__ constexpr int row_groups(bool) { return 1; }

// ACC: the model runs accelerated iterations (ACWB / HCWB); plain CWB models compile without
// the momentum sequence, the error-corrected residual and their loads.
template <int KIND, typename IndT, bool ACC>
__global__ void __launch_bounds__(kRowThreads, 4) k_rows(RowArgs a)
{
    constexpr int kRowGroups = row_groups(ACC);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4 * kRowGroups;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x * 4 * kRowGroups + threadIdx.x * 4;
    const bool need_y = KIND != kRowsUpdate || a.hybrid, need_w = KIND != kRowsUpdate;
    const bool need_ylo = need_y && a.y_lo != nullptr, load_w = need_w && a.w != nullptr;
    RowIn in[kRowGroups];
    auto first_pass_loads = [&]() {
#pragma unroll
        for (int u = 0; u < kRowGroups; ++u) {
            const int64_t i4 = first + (int64_t)u * blockDim.x * 4;
            if (i4 < a.n_pad) load_row_in<ACC>(a, i4, in[u], need_y);
        }
    };
    // Without HCWB the kernel this one depends on is the solve (or nothing), which writes none of
    // these inputs: f, h were last written by the previous row pass, which finished before the
    // previous scatter began.  So the first pass's loads go out before the wait and overlap the
    // solve's tail, on SMs the solve leaves idle.  (With HCWB a row pass follows another row pass.)
    if (!a.hybrid) first_pass_loads();
    grid_dep_wait();
    grid_dep_launch();
    if (a.hybrid) first_pass_loads();
    const DevState st = *a.state;
    // HCWB runs the fused pass (update, validation risk, residuals of the current mode) and then this
    // residual pass, which has work only in the iteration where the fused pass switched to CWB
    if (KIND == kRowsResid && ACC && a.hybrid && !st.resid_stale) return;
    const bool pend = (KIND != kRowsResid) && (st.m > st.m_applied);
    const int pm = st.pend_mode;
    const bool pm_acwb = ACC && pm == kModeACWB;
    const IndT* ind = static_cast<const IndT*>(a.ind);
    const IndT* ind_sel = (st.k_sel >= 0) ? ind + (int64_t)a.l_bin[st.k_sel] * a.n_pad : nullptr;
    const IndT* ind_cor = (st.k_cor >= 0) ? ind + (int64_t)a.l_bin[st.k_cor] * a.n_pad : nullptr;
    const float* v0 = a.v + (int64_t)max(st.k_sel, 0) * a.S;
    const float* v1 = a.v + ((int64_t)a.K + max(st.k_cor, 0)) * a.S;
    // the pending iteration's selected coefficients go to the trace (the next solve overwrites theta_it)
    if (pend && blockIdx.x == 0 && st.m >= 1 && st.m - 1 < a.trace_cap) {
        for (int e = threadIdx.x; e < 2 * a.D; e += blockDim.x) {
            const int ch = e / a.D, i = e % a.D;
            const int kk = ch ? st.k_cor : st.k_sel;
            if (kk >= 0)
                a.tr_theta[((int64_t)2 * (st.m - 1) + ch) * a.D + i] = a.theta_it[((int64_t)ch * a.K + kk) * a.D + i];
        }
    }

    // Per-iteration scalars, one thread per block (FP64 is slow on this part and every value
    // is uniform): pending update of iteration st.m (Algorithm 1: f = f + nu b; Algorithm 3:
    // f = g + nu b, h += eta b_cor) and the momentum weights of iteration st.m + 1.
    __shared__ DF sc_df[7];
    const int mode_n = st.mode;
    const int m_n = st.m + 1;
    const bool acwb_n = ACC && (mode_n == kModeACWB);
    if (ACC && threadIdx.x == 0) {     // plain CWB needs none of these (and no FP64 divisions)
        DF om_p = {1.0f, 0.0f}, th_p = {0.0f, 0.0f}, eta_p = {0.0f, 0.0f};
        if (pend && pm_acwb) {
            const double thm = 2.0 / ((double)st.m + 1.0);
            om_p = df_of(1.0 - thm);
            th_p = df_of(thm);
            eta_p = df_of(a.gamma * a.nu / thm);
        }
        const double thn_d = 2.0 / ((double)m_n + 1.0);
        sc_df[0] = om_p;
        sc_df[1] = th_p;
        sc_df[2] = eta_p;
        sc_df[3] = df_of(1.0 - thn_d);
        sc_df[4] = df_of(thn_d);
        sc_df[5] = df_of((double)m_n / ((double)m_n + 1.0));
    }
    if (ACC) __syncthreads();
    const DF one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
    const DF om_p = ACC ? sc_df[0] : one, th_p = ACC ? sc_df[1] : zero, eta_p = ACC ? sc_df[2] : zero;
    const DF om_n = ACC ? sc_df[3] : one, th_n = ACC ? sc_df[4] : zero, cmul = ACC ? sc_df[5] : zero;
    const int64_t n_act = (acwb_n && a.hybrid) ? a.n_tr : a.n;
    const bool first_acwb = (m_n == 1);
    const DF nu = {a.nu_hi, a.nu_lo};
    const bool need_bc = pend && pm_acwb;
    const bool need_bc_resid = (KIND != kRowsUpdate) && acwb_n && !first_acwb;
    const bool eval_risk = (KIND != kRowsResid) && ACC && a.hybrid && (!st.risk_valid || (pend && pm_acwb));
    // plain CWB: the residuals go out as int32 fixed point at the scale of a bound on max |w r| known
    // before the pass, so the scatter needs no conversion step (the histograms keep their overflow
    // guarantee as long as the bound holds, which is checked)
    constexpr bool kDirect = !ACC && KIND == kRowsFused;
    int q_exp = 0;
    float q_scale = 1.0f, q_bound = 0.0f;
    if (kDirect && a.direct) {
        const float vsel = (pend && st.k_sel >= 0) ? __ldcg(a.vmax + st.k_sel) : 0.0f;
        const uint32_t bb = residual_bound(a.loss, pend, st.rprev_bits, vsel, a.nu_hi, a.wmax);
        q_exp = fixed_scale(bb, st.cnt_log2[0]);
        q_scale = pow2f(q_exp);
        q_bound = __uint_as_float(bb);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.state->fix_exp = q_exp;
            a.state->resid_path = 2;
        }
    }
    bool over_bound = false;

    double risk_acc = 0.0;
    float rmax0 = 0.0f, rmax1 = 0.0f;
    bool nonfinite = false;
    for (int64_t p0 = first; p0 < a.n_pad; p0 += stride) {
        if (p0 != first) {
#pragma unroll
            for (int u = 0; u < kRowGroups; ++u) {
                const int64_t i4 = p0 + (int64_t)u * blockDim.x * 4;
                if (i4 < a.n_pad) load_row_in<ACC>(a, i4, in[u], need_y);
            }
        }
        // state-dependent loads of the pass: selected bins, then their fitted values
        int ks[kRowGroups][4], kc[kRowGroups][4];
        float4 c4in[kRowGroups], yl4in[kRowGroups], w4in[kRowGroups];
#pragma unroll
        for (int u = 0; u < kRowGroups; ++u) {
            const int64_t i4 = p0 + (int64_t)u * blockDim.x * 4;
            yl4in[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            w4in[u] = make_float4(1.f, 1.f, 1.f, 1.f);
            if (i4 >= a.n_pad) continue;
            if ((need_bc || need_bc_resid) && ind_cor) load_ind4<IndT>(ind_cor, i4, kc[u]);
            if (pend && ind_sel) load_ind4<IndT>(ind_sel, i4, ks[u]);
            if (KIND != kRowsUpdate && acwb_n) c4in[u] = *reinterpret_cast<const float4*>(a.c + i4);
            if (need_ylo) yl4in[u] = *reinterpret_cast<const float4*>(a.y_lo + i4);
            if (load_w) w4in[u] = *reinterpret_cast<const float4*>(a.w + i4);
        }
#pragma unroll
        for (int u = 0; u < kRowGroups; ++u) {
            const int64_t i4 = p0 + (int64_t)u * blockDim.x * 4;
            if (i4 >= a.n_pad) continue;
            DF* fv = in[u].f;
            DF* hv = in[u].h;
            float bc[4] = {0.f, 0.f, 0.f, 0.f};
            if ((need_bc || need_bc_resid) && ind_cor) {
#pragma unroll
                for (int t = 0; t < 4; ++t) bc[t] = __ldg(v1 + kc[u][t]);
            }
            if (pend && ind_sel) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float b0 = __ldg(v0 + ks[u][t]);
                    if (!pm_acwb) {
                        fv[t] = df_add(fv[t], df_mul_f(nu, b0));
                    } else {
                        DF g = df_add(df_mul(fv[t], om_p), df_mul(hv[t], th_p));
                        fv[t] = df_add(g, df_mul_f(nu, b0));
                        hv[t] = df_add(hv[t], df_mul_f(eta_p, bc[t]));
                    }
                }
                store_df4(a.f, i4, fv);
                if (pm_acwb && a.h) store_df4(a.h, i4, hv);
            }
            const float4 y4 = in[u].y, yl4 = yl4in[u], w4 = w4in[u];
            if (eval_risk) {
                if (i4 + 4 > a.n_tr && i4 < a.n) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        int64_t i = i4 + t;
                        if (i >= a.n_tr && i < a.n)
                            risk_acc += (double)loss_value(a.loss, get4(y4, t), get4(yl4, t), fv[t]);
                    }
                }
            }
            if (KIND != kRowsUpdate) {
                float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
                float4 c4 = r0;
                if (acwb_n) c4 = c4in[u];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    int64_t i = i4 + t;
                    if (i >= n_act) continue;
                    float yv = get4(y4, t), ylo = get4(yl4, t), wv = get4(w4, t);
                    if (!acwb_n) {
                        set4(r0, t, wv * neg_gradient(a.loss, yv, ylo, fv[t]));
                    } else {
                        DF g = df_add(df_mul(fv[t], om_n), df_mul(hv[t], th_n));
                        float r = neg_gradient(a.loss, yv, ylo, g);
                        float cv = r;
                        if (!first_acwb) {
                            DF ct = df_mul_f(cmul, get4(c4, t) - bc[t]);
                            DF cs = df_add(ct, DF{r, 0.0f});
                            cv = cs.hi + cs.lo;
                        }
                        set4(c4, t, cv);
                        set4(r0, t, wv * r);
                        set4(r1, t, wv * cv);
                    }
                }
                const float m0 = fmaxf(fmaxf(fabsf(r0.x), fabsf(r0.y)), fmaxf(fabsf(r0.z), fabsf(r0.w)));
                const float m1 = fmaxf(fmaxf(fabsf(r1.x), fabsf(r1.y)), fmaxf(fabsf(r1.z), fabsf(r1.w)));
                if (!(fabsf(r0.x) + fabsf(r0.y) + fabsf(r0.z) + fabsf(r0.w) + fabsf(r1.x) + fabsf(r1.y) + fabsf(r1.z) +
                      fabsf(r1.w) <= 3.0e38f))
                    nonfinite = true;
                rmax0 = fmaxf(rmax0, m0);
                rmax1 = fmaxf(rmax1, m1);
                if (kDirect && a.direct) {
                    if (m0 > q_bound) over_bound = true;
                    *reinterpret_cast<int4*>(a.rw + i4) =
                        make_int4(__float2int_rn(r0.x * q_scale), __float2int_rn(r0.y * q_scale),
                                  __float2int_rn(r0.z * q_scale), __float2int_rn(r0.w * q_scale));
                } else {
                    *reinterpret_cast<float4*>(a.rw + i4) = r0;
                }
                if (acwb_n) {
                    *reinterpret_cast<float4*>(a.rw + a.n_pad + i4) = r1;
                    *reinterpret_cast<float4*>(a.c + i4) = c4;
                }
            }
        }
    }

    // block partial of the validation risk, then the last block finishes the iteration bookkeeping
    __shared__ double red[kRowThreads];
    __shared__ bool is_last;
    __shared__ float wmax[2][kRowThreads / 32];
    __shared__ bool bad_blk;
    if (threadIdx.x == 0) bad_blk = false;
    if (KIND != kRowsUpdate) {
        // largest |scatter input| per channel: sets the fixed-point scale of the histograms
        for (int o = 16; o > 0; o >>= 1) {
            rmax0 = fmaxf(rmax0, __shfl_xor_sync(0xffffffffu, rmax0, o));
            rmax1 = fmaxf(rmax1, __shfl_xor_sync(0xffffffffu, rmax1, o));
        }
        const bool anybad = __any_sync(0xffffffffu, nonfinite);
        if (kDirect && __any_sync(0xffffffffu, over_bound) && (threadIdx.x & 31) == 0) atomicOr(&a.state->err, kErrBound);
        __shared__ bool wbad[kRowThreads / 32];
        if ((threadIdx.x & 31) == 0) {
            wmax[0][threadIdx.x >> 5] = rmax0;
            wmax[1][threadIdx.x >> 5] = rmax1;
            wbad[threadIdx.x >> 5] = anybad;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b0 = 0.0f, b1 = 0.0f;
            for (int w = 0; w < kRowThreads / 32; ++w) {
                b0 = fmaxf(b0, wmax[0][w]);
                b1 = fmaxf(b1, wmax[1][w]);
                if (wbad[w]) bad_blk = true;
            }
            // non-negative FP32 values order like their bit patterns; the solve of the
            // previous iteration reset both maxima to 0
            atomicMax(&a.state->rmax_bits[0], __float_as_uint(b0));
            if (acwb_n) atomicMax(&a.state->rmax_bits[1], __float_as_uint(b1));
            if (bad_blk) atomicOr(&a.state->err, kErrNonFinite);
        }
        // the residual passes end here (the fused pass too, outside HCWB): the next iteration's row
        // pass sees m > m_applied for the pending update, and only an update pass records what it applied
        if (KIND == kRowsResid || !(ACC && a.hybrid)) return;   // (HCWB models are accelerated)
    }
    if (eval_risk) {
        red[threadIdx.x] = risk_acc;
        __syncthreads();
        for (int s = kRowThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
    } else {
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (bad_blk) atomicOr(&a.state->err, kErrNonFinite);
        if (eval_risk && a.risk_part) a.risk_part[blockIdx.x] = red[0];
        fence_acq_rel_gpu();
        unsigned t = atomicAdd(&a.state->ticket_rows, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    fence_acq_rel_gpu();
    // last block (update pass): block-parallel, fixed-order reduction of the validation risk partials
    {
        double rs = 0.0;
        if (eval_risk)
            for (int b = threadIdx.x; b < (int)gridDim.x; b += kRowThreads) rs += __ldcg(a.risk_part + b);
        red[threadIdx.x] = rs;
    }
    __syncthreads();
    for (int s = kRowThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        DevState* S = a.state;
        if (eval_risk) {
            double risk = red[0] / (double)(a.n - a.n_tr);
            if (!S->risk_valid) {
                S->risk_prev = risk;
                S->risk_valid = 1;
            } else {
                S->counter = (risk > S->risk_prev) ? S->counter + 1 : 0;
                S->risk_prev = risk;
            }
        }
        bool switched = false;
        if (KIND != kRowsResid && ACC && a.hybrid && S->mode == kModeACWB && S->counter >= a.patience) {
            S->mode = kModeCWB;
            S->phase = 1;
            S->switch_iter = S->m + 1;
            switched = true;
        }
        if (KIND == kRowsFused) {
            // the residuals this pass wrote are those of the mode it started in; after a switch the
            // residual pass recomputes them (CWB on all rows) and takes the maxima afresh
            S->resid_stale = switched ? 1 : 0;
            if (switched) {
                S->rmax_bits[0] = 0u;
                S->rmax_bits[1] = 0u;
            }
        }
        if (pend) S->m_applied = st.m;
        if (KIND == kRowsUpdate && pend && st.k_sel >= 0) {
            // this pass moved f without forming residuals: widen the bound on max |w r| by the update,
            // so that the next row pass's fixed-point scale stays valid
            S->rprev_bits = residual_bound(a.loss, true, S->rprev_bits, __ldcg(a.vmax + st.k_sel), a.nu_hi, a.wmax);
        }
        S->ticket_rows = 0;
    }
}

// ---------------------------------------------------------------------------
// binMatVec scatter (Algorithm 2): u_b[l] = sum_{i: ind_b,i = l} w_i r_i.
//
// A thread-block cluster of `cs` CTAs owns one slot (F binnings x one bin range)
// and a contiguous run of 256-row tiles.  Inside a CTA one producer warp streams
// tiles with TMA: a 3D tiled copy of the uint8/uint16 index matrix (box = the
// tile's 256 rows x FE binnings, landing as 128-byte rows [chunk][binning] with
// the 128-byte swizzle) and a 1D bulk copy of the matching residual rows, into a
// ring of `stages` shared-memory buffers guarded by mbarriers; a converter warp
// turns the residual tile into fixed point (see fixed_scale).  Consumer warps give
// every lane its own binning (lane % F), channel and row subset; the lanes of a
// row subset read the same 16-byte unit of rows of their binnings, so the residual
// read is a broadcast and the swizzle spreads the index reads over all banks.
// Lanes add into hist[channel][bin][lane's binning] with int32 shared-memory
// atomics: lanes of a warp never share an address and, for F = 32 (or F = 16
// with two channels), never share a bank.  At the end the cluster's histograms
// are summed through distributed shared memory, each CTA reducing a slice of the
// bins, and written once per cluster.

namespace cg = cooperative_groups;

struct ScatterArgs {
    const DevState* state;
    const float* rw;
    int64_t n, n_tr, n_pad;
    int B, F, FE, bin_ranges, nb_cta, ch_stride;
    int stage_rows, stages, nb_box, box_bytes, unit_rows;
    int cs;
    const int32_t* cluster_slot;   // [2][clusters]: slot of each cluster, then its index within the slot
    const int32_t* slot_c0;        // [slots + 1]: first cluster of each slot
    int hybrid;
    uint32_t ind_off, r_off, q_off, hist_off, bar_off, stage_ind_bytes, stage_r_bytes;
    float* part;                   // [clusters][cmax][F][nb_cta] (int32 fixed point or FP32)
    int stage_cb;                  // bins per chunk of the epilogue's transposing stage
    uint32_t* err;
    int64_t count_rows;            // >= 0: counting pass over this many rows (every row adds 1)
    long long wait_cycles;         // limit of each ring wait (SM clocks); copies in flight are drained with kWaitCycles
    int withhold;                  // test hook: >= 0 makes CTA 0 arm, but never fill, its tile min(withhold, ntiles - 1)
    int direct;                    // 1: the residual rows are already int32 fixed point (no conversion step)
    int sleep_waits;               // 1: ring waits sleep with a suspend-time hint (deep rings)
};

constexpr int kEpiVec = 4;                         // 16-byte vectors per thread and pass of the cluster epilogue

// FL2 >= 0: the lanes per channel F = 2^FL2 is a compile-time constant (the common plans), -1: read at run time.
template <typename IndT, int CMAX, bool INT_ACC, bool RANGED, int FL2>
__global__ void __launch_bounds__(kScatterThreads, 1) k_scatter(const __grid_constant__ CUtensorMap tmap, ScatterArgs a)
{
    constexpr int U = 16 / sizeof(IndT);                   // rows per 16-byte unit
    constexpr int UN = sizeof(IndT) == 2 ? 2 : 1;          // units in flight per lane (16 consumer warps)
    using Acc = typename std::conditional<INT_ACC, int, float>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the ring; offsetting the shared array itself keeps every
    // access below in the shared state space (no generic addressing)
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int cl = blockIdx.x / a.cs;
    const int slot = a.cluster_slot[cl];
    const int cin = a.cluster_slot[gridDim.x / a.cs + cl];
    const int g = slot / a.bin_ranges, br = slot % a.bin_ranges;
    const int ncl = a.slot_c0[slot + 1] - a.slot_c0[slot];
    const int pcl = a.slot_c0[slot] + cin;        // this cluster's row of partial histograms

    const bool counting = a.count_rows >= 0;
    const int F = FL2 >= 0 ? (1 << FL2) : a.F;   // lanes per channel and row set (power of two)
    const int FE = a.FE;                // binnings of this group held in the ring (<= F)
    const int b_lo = br * a.nb_cta;
    constexpr int row_bytes = kStageRows * (int)sizeof(IndT);
    Acc* hist = reinterpret_cast<Acc*>(smem + a.hist_off);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.bar_off);
    uint64_t* ready = full + a.stages;
    uint64_t* empty = ready + a.stages;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int W = kScatterWarps;                          // consumer warps; warp W loads, warp W+1 converts

    for (int i = tid; i < CMAX * a.ch_stride; i += blockDim.x) hist[i] = Acc(0);
    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], 1);
            mbar_init(&empty[s], W);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // Without HCWB the iteration mode never changes (ACWB models use two channels, CWB models one),
    // so the tiles can be planned without the iteration state and the loader can start on the index
    // matrix, which no kernel writes, before the row pass has finished; every other read of what
    // the row pass wrote waits for it.
    const bool fixed_mode = !a.hybrid;
    int mode = CMAX == 2 ? kModeACWB : kModeCWB;
    if (!fixed_mode) {
        grid_dep_wait();
        mode = a.state->mode;
    }
    const int C = (!counting && CMAX == 2 && mode == kModeACWB) ? 2 : 1;
    const bool train_rows = a.hybrid && mode == kModeACWB;
    const int64_t n_act = counting ? a.count_rows : (train_rows ? a.n_tr : a.n);
    const int64_t tiles = (n_act + kStageRows - 1) / kStageRows;
    const int64_t pieces = (int64_t)ncl * a.cs, piece = (int64_t)cin * a.cs + rank;
    const int64_t t_lo = tiles * piece / pieces, t_hi = tiles * (piece + 1) / pieces;
    const int ntiles = (int)(t_hi - t_lo);
    const long long deadline = clock64() + a.wait_cycles;

    if (warp == W) {
        // loader: one 3D TMA box (the tile's rows x FE binnings) and C residual rows per tile
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(FE * row_bytes + C * kStageRows * 4);   // box bytes + residual rows
            int issued = 0;
            bool ok = true;
            // a withheld tile's stage is armed but no copy is issued, so its barrier never completes and
            // the waits on it run out (the failure-path test); the drain below skips it
            const int wh = (a.withhold >= 0 && blockIdx.x == 0 && ntiles > 0) ? min(a.withhold, ntiles - 1) : -1;
            // the first ring's index boxes before the wait (their barriers expect the residual
            // bytes too, which follow once the row pass is complete)
            const int early = fixed_mode ? min(a.stages, ntiles) : 0;
            auto load_ind = [&](int st, int64_t row0) {
                tma_load_3d(smem + a.ind_off + (size_t)st * a.stage_ind_bytes, &tmap, 0, g * FE,
                            (int)(row0 / (128 / (int)sizeof(IndT))), &full[st]);
            };
            auto load_r = [&](float* dst, const float* src, uint64_t* bar) {
                bulk_load(dst, src, (uint32_t)kStageRows * 4, bar);
            };
            for (int it = 0; it < early; ++it) {
                const int64_t row0 = (t_lo + it) * kStageRows;
                mbar_arrive_expect_tx(&full[it], bytes);
                if (it == wh) continue;
                load_ind(it, row0);
            }
            if (fixed_mode) grid_dep_wait();
            for (int it = 0; it < early; ++it) {
                const int64_t row0 = (t_lo + it) * kStageRows;
                float* r_dst = reinterpret_cast<float*>(smem + a.r_off + (size_t)it * a.stage_r_bytes);
                if (it == wh) {
                    ++issued;
                    continue;
                }
                for (int ch = 0; ch < C; ++ch) load_r(r_dst + ch * kStageRows, a.rw + ch * a.n_pad + row0, &full[it]);
                ++issued;
            }
            // ring position kept incrementally (no division by the run-time stage count per tile)
            int s = early;
            uint32_t ph = 0;
            for (int it = early; it < ntiles; ++it, ++s) {
                if (s == a.stages) {
                    s = 0;
                    ph ^= 1u;
                }
                if (it >= a.stages && !mbar_wait(&empty[s], ph ^ 1u, deadline, a.sleep_waits)) {
                    ok = false;
                    break;
                }
                const int64_t row0 = (t_lo + it) * kStageRows;
                mbar_arrive_expect_tx(&full[s], bytes);
                if (it == wh) {
                    ++issued;
                    continue;
                }
                load_ind(s, row0);
                float* r_dst = reinterpret_cast<float*>(smem + a.r_off + (size_t)s * a.stage_r_bytes);
                for (int ch = 0; ch < C; ++ch) load_r(r_dst + ch * kStageRows, a.rw + ch * a.n_pad + row0, &full[s]);
                ++issued;
            }
            if (!ok || wh >= 0) {
                if (!ok) atomicOr(a.err, kErrTimeout);
                // let copies already in flight land before the CTA retires (a withheld tile has none)
                const long long d2 = clock64() + kWaitCycles;
                for (int it = (issued > a.stages ? issued - a.stages : 0); it < issued; ++it)
                    if (it != wh) mbar_wait(&full[it % a.stages], (it / a.stages) & 1, d2);
            }
        }
    } else if (warp == W + 1 && !a.direct) {
        // converter: residual tile -> fixed point (or a plain hand-over for FP32 accumulation)
        if (fixed_mode) grid_dep_wait();
        float scale[2] = {1.0f, 1.0f};
        if (INT_ACC && !counting) {
            const int cidx = train_rows ? 1 : 0;
            scale[0] = pow2f(fixed_scale(a.state->rmax_bits[0], a.state->cnt_log2[cidx]));
            if (C == 2) scale[1] = pow2f(fixed_scale(a.state->rmax_bits[1], a.state->cnt_log2[cidx]));
        }
        int s = 0;
        uint32_t ph = 0;
        for (int jt = 0; jt < ntiles; ++jt, ++s) {
            if (s == a.stages) {
                s = 0;
                ph ^= 1u;
            }
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, deadline, a.sleep_waits))) {
                if (lane == 0) atomicOr(a.err, kErrTimeout);
                break;
            }
            if (INT_ACC) {
                // fixed point in place of the residuals (every lane rewrites the values it read):
                // the stage holds one copy, which leaves room for one more ring stage; a proxy fence
                // orders these generic writes before the stage's next bulk copy
                const float* rt = reinterpret_cast<const float*>(smem + a.r_off + (size_t)s * a.stage_r_bytes);
                int* qt = reinterpret_cast<int*>(smem + a.q_off + (size_t)s * a.stage_r_bytes);
                const int64_t row0 = (t_lo + jt) * kStageRows;
                // 16-byte vectors, the loads of a lane issued together: the conversion sits on
                // the pipeline's critical path and its shared-memory accesses queue behind the
                // consumers' atomics, so it pays that queue once per batch, not once per value
                const int total = C * kStageRows;          // multiple of 128
#pragma unroll 4
                for (int i0 = lane * 4; i0 < total; i0 += 128) {
                    const int ch = i0 >= kStageRows ? 1 : 0;
                    int4 q;
                    if (counting) {
                        const int64_t r = row0 + i0;
                        q = make_int4(r < n_act, r + 1 < n_act, r + 2 < n_act, r + 3 < n_act);
                    } else {
                        const float sc = ch ? scale[1] : scale[0];
                        const float4 x = *reinterpret_cast<const float4*>(rt + i0);
                        q = make_int4(__float2int_rn(x.x * sc), __float2int_rn(x.y * sc), __float2int_rn(x.z * sc),
                                      __float2int_rn(x.w * sc));
                    }
                    *reinterpret_cast<int4*>(qt + i0) = q;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[s]);
        }
    } else if (warp < W) {
        const int q = lane / F;
        const int f = lane % F;
        const int ch = q % C, rs = q / C;
        const int RS = 32 / (F * C);                      // compile-time for the common plans
        const bool active = f < FE && g * FE + f < a.B;
        Acc* hf = hist + ch * a.ch_stride + f;
        const int fsh = FL2 >= 0 ? FL2 : __ffs(F) - 1;    // F is a power of two
        constexpr int nunits = row_bytes / 16;
        const int step = UN * RS;
        int s = 0;
        uint32_t ph = 0;
        for (int it = 0; it < ntiles; ++it, ++s) {
            if (s == a.stages) {
                s = 0;
                ph ^= 1u;
            }
            // (without a conversion step the stage is ready as soon as its copies have landed)
            if (!__all_sync(0xffffffffu, mbar_wait(a.direct ? &full[s] : &ready[s], ph, deadline, a.sleep_waits))) {
                if (lane == 0) atomicOr(a.err, kErrTimeout);
                break;
            }
            const unsigned char* ind_st = smem + a.ind_off + (size_t)s * a.stage_ind_bytes;
            const Acc* r_st =
                reinterpret_cast<const Acc*>(smem + (INT_ACC ? a.q_off : a.r_off) + (size_t)s * a.stage_r_bytes) +
                ch * kStageRows;
            bool released = false;
#pragma unroll 1
            for (int u0 = warp * step; u0 < nunits; u0 += W * step) {      // warp-uniform bounds
                uint4 raw[UN];
                Acc rv[UN][U];
                bool live[UN];
#pragma unroll
                for (int k = 0; k < UN; ++k) {
                    // the lanes of a row set read the same logical 16-byte unit (8 or 16 rows) of
                    // their binnings: the residuals are one broadcast, and the 128-byte swizzle
                    // of the TMA box spreads the index reads over all banks.  Unit u of binning
                    // f sits in 128-byte row R = (u / 8) FE + f at 16-byte slot (u % 8) ^ (R % 8).
                    const int pos = u0 + k * RS + rs;
                    live[k] = active && pos < nunits;
                    if (!active) continue;
                    const int R = (pos >> 3) * FE + f;
                    raw[k] = *reinterpret_cast<const uint4*>(ind_st + R * 128 + (((pos & 7) ^ (R & 7)) << 4));
#pragma unroll
                    for (int t4 = 0; t4 < U / 4; ++t4) {
                        if (INT_ACC) {
                            const int4 r4 = reinterpret_cast<const int4*>(r_st + pos * U)[t4];
                            rv[k][4 * t4] = r4.x; rv[k][4 * t4 + 1] = r4.y; rv[k][4 * t4 + 2] = r4.z; rv[k][4 * t4 + 3] = r4.w;
                        } else {
                            const float4 r4 = reinterpret_cast<const float4*>(r_st + pos * U)[t4];
                            rv[k][4 * t4] = r4.x; rv[k][4 * t4 + 1] = r4.y; rv[k][4 * t4 + 2] = r4.z; rv[k][4 * t4 + 3] = r4.w;
                        }
                    }
                }
                if (u0 + W * step >= nunits) {
                    // the stage is free once the warp's last values of it are in registers: hand it
                    // back to the loader before the atomics (the arrive orders the loads before it)
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                    released = true;
                }
#pragma unroll
                for (int k = 0; k < UN; ++k) {
                    if (!live[k]) continue;
                    int idx[U];
                    unpack16<IndT>(raw[k], idx);
#pragma unroll
                    for (int t = 0; t < U; ++t) {
                        if (RANGED) {
                            const unsigned bl = (unsigned)(idx[t] - b_lo);
                            if (bl < (unsigned)a.nb_cta) atomicAdd(hf + (bl << fsh), rv[k][t]);
                        } else {
                            atomicAdd(hf + (idx[t] << fsh), rv[k][t]);
                        }
                    }
                }
            }
            if (!released) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
        }
    }
    grid_dep_launch();                 // the solve may be scheduled as SMs free up
    __syncthreads();
    cluster.sync();
    // Sum the cluster's histograms (fixed rank order), each CTA one slice of the bins,
    // and store them binning-major, part[cluster][ch][f][bin], so that a learner's
    // partial histogram is one contiguous row.  The slice goes through the idle ring
    // as [f][cb + 1] (odd row pitch): the 16-byte DSMEM reads in [bin][f] order and
    // the transposed stores are both free of bank conflicts, the global stores coalesced.
    const int nb = a.nb_cta;
    const int bpr = ((nb + a.cs - 1) / a.cs + 3) & ~3;          // bins per rank, multiple of 4
    const int bl0 = min(nb, rank * bpr), bl1 = min(nb, bl0 + bpr);
    const int cb = a.stage_cb;                                  // bins per staged chunk, multiple of 4
    const int fsh_e = __ffs(F) - 1;
    Acc* stg = reinterpret_cast<Acc*>(smem);
    for (int ch = 0; ch < C; ++ch) {
        Acc* dst = reinterpret_cast<Acc*>(a.part) + ((int64_t)pcl * CMAX + ch) * (int64_t)F * nb;
        for (int c0 = bl0; c0 < bl1; c0 += cb) {
            const int c1 = min(bl1, c0 + cb);
            const int nvec = ((c1 - c0) * F) >> 2;
            // kEpiVec vectors per thread and pass, the loads from one rank issued together (a
            // remote rank's distributed shared memory is a long round trip)
            for (int v0 = tid; v0 < nvec; v0 += kEpiVec * blockDim.x) {
                Acc acc[kEpiVec][4];
#pragma unroll
                for (int k = 0; k < kEpiVec; ++k)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[k][t] = Acc(0);
                for (int r = 0; r < a.cs; ++r) {
                    const Acc* h = cluster.map_shared_rank(hist, r) + ch * a.ch_stride + c0 * F;
                    int4 x[kEpiVec];
#pragma unroll
                    for (int k = 0; k < kEpiVec; ++k) {
                        const int v = v0 + k * blockDim.x;
                        x[k] = v < nvec ? reinterpret_cast<const int4*>(h)[v] : make_int4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int k = 0; k < kEpiVec; ++k) {
                        if (INT_ACC) {
                            acc[k][0] += x[k].x; acc[k][1] += x[k].y; acc[k][2] += x[k].z; acc[k][3] += x[k].w;
                        } else {
                            acc[k][0] += __int_as_float(x[k].x); acc[k][1] += __int_as_float(x[k].y);
                            acc[k][2] += __int_as_float(x[k].z); acc[k][3] += __int_as_float(x[k].w);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < kEpiVec; ++k) {
                    const int v = v0 + k * blockDim.x;
                    if (v < nvec) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int e = 4 * v + t;
                            stg[(e & (F - 1)) * (cb + 1) + (e >> fsh_e)] = acc[k][t];
                        }
                    }
                }
            }
            __syncthreads();
            const int nbc = c1 - c0;
            // the rows of lanes beyond the group's binnings are never read (the counting pass's
            // maximum reads every row, so it writes them all)
            const int f_end = counting ? F : FE;
            for (int f = warp; f < f_end; f += (int)(blockDim.x >> 5))      // a warp per binning row
                for (int lb = lane; lb < nbc; lb += 32) dst[(int64_t)f * nb + c0 + lb] = stg[f * (cb + 1) + lb];
            __syncthreads();
        }
    }
    cluster.sync();
}

// ceil(log2(largest bin count of any cluster)) from a counting pass of the scatter.
__global__ void k_count_max(const int* __restrict__ part, int clusters, int cmax, int nbf, DevState* state, int idx)
{
    __shared__ int red[256];
    const int64_t total = (int64_t)clusters * nbf;
    int mx = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / nbf, i = e - c * nbf;
        mx = max(mx, part[(c * cmax) * (int64_t)nbf + i]);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(&state->cnt_max[idx], red[0]);
}

__global__ void k_count_log2(DevState* state, int idx)
{
    if (threadIdx.x != 0) return;
    const int c = state->cnt_max[idx];
    int l = 0;
    while ((1 << l) < c && l < 30) ++l;
    state->cnt_log2[idx] = l;
}

// Exact int64 sums of the per-cluster fixed-point partials of channel 0, u[b][l] (row shards
// exchange these).  One thread per (binning, bin); the clusters of a bin are those of its slot.
__global__ void k_partials_to_u(const int* __restrict__ part, const int32_t* __restrict__ slot_c0, int B, int S, int FE,
                                int F, int nb_cta, int bin_ranges, int cmax, long long* __restrict__ u)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * S; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / S), l = (int)(e - (int64_t)b * S);
        const int g = b / FE, f = b - g * FE;
        const int br = l / nb_cta, lb = l - br * nb_cta;
        const int slot = g * bin_ranges + br;
        long long acc = 0;
        for (int c = slot_c0[slot]; c < slot_c0[slot + 1]; ++c)
            acc += __ldcg(part + (((int64_t)c * cmax) * F + f) * nb_cta + lb);
        u[e] = acc;
    }
}

// ---------------------------------------------------------------------------
// Per-learner fit, criterion and argmin.
//
// One CTA per learner k on binning b: u_b[l] = sum over the clusters of b's slot
// of the partial histograms (exact int64 sum of the fixed-point partials, or a
// compensated FP32 sum), s = Z^b^T u (FP32, column-major design staged in shared
// memory), theta = P s and Q = theta^T G theta - 2 theta^T s = s^T A s with the
// cached A = P G P - 2 P (float-float arithmetic, about 44 bits), and the learner's
// update table v_k = Z^b theta (FP32).  The last CTA to take the ticket finds the
// argmin of Q per channel (ties: lowest k), writes the trace and advances the
// iteration state.

// Solve block sizes: 512 threads for models with more than 512 design points (a pass over the
// partial histograms covers 1024 bins, two halves of 256 threads x 4 bins), 256 threads otherwise,
// so that two solve CTAs share an SM: fits that run side by side (batches, the server) are bound by
// the solve's SM occupancy, not its latency.  A pass covers 2 x threads bins (kSolveChunk).
__host__ __device__ constexpr int solve_chunk(int threads) { return 2 * threads; }
// partial-histogram rows per thread and batch (per channel): 20 for the 512-thread solve of large
// models (many clusters per slot); the 256-thread solve of small models (few clusters) takes 8, which
// keeps it within its 128 registers (20 spilled there)
__host__ __device__ constexpr int solve_batch(int threads) { return threads >= 512 ? 20 : 8; }

struct SolveArgs {
    DevState* state;
    int K, D, S;
    const float* part;        // [clusters][cmax][F][nb_cta]
    const int32_t* slot_c0;   // [slots + 1]
    int F, FE, cmax, nb_cta, bin_ranges, hybrid;   // binning b lives in lane b % FE of group b / FE
    int stage_v;              // the learner's design rows (float4 + first column per bin) are staged
    int stage_z;              // the learner's column-major design is staged
    const float* zb;          // [K][S][4]
    const int32_t* zcol;      // [K][S]
    const int32_t* crange;    // [K][D][2]
    const int32_t* toff;      // [K][D]
    const float* ztab;        // [K][4 S]
    const float* ztab_lo;     // [K][4 S] low parts (float-float design)
    const int32_t* l_bin;
    const int32_t* l_d;
    const int32_t* l_nstar;
    const float2* A;          // [2][K][D][D] criterion matrix P G P - 2 P, float-float pairs
    const float2* P;          // [2][K][D][D] cached inverse, float-float pairs
    double* theta_it;         // [2][K][D]
    double* q_it;             // [2][K]
    float* v;                 // [2][K][S]
    int32_t* tr_k;            // [cap][2]
    int32_t* tr_mode;         // [cap]
    double* tr_q;             // [cap][2]
    const int32_t* forced;    // [cap]
    int trace_cap;
    float* vmax;              // [K] max |v_k| of channel 0 (input of the residual bound of the next row pass)
    const long long* u64;     // row shards: exact histogram sums [B][S] of all shards (replaces the partials)
    int direct;               // the row pass wrote the fixed point itself, at the state's fix_exp
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <bool INT_ACC, int kSolveThreads>
__global__ void __launch_bounds__(kSolveThreads, 512 / kSolveThreads) k_solve(SolveArgs a)
{
    constexpr int kSolveChunk = solve_chunk(kSolveThreads);
    constexpr int kSolveBatch = solve_batch(kSolveThreads);
    constexpr int NW = kSolveThreads / 32;
    constexpr int kColsPerWarp = (kMaxD + NW - 1) / NW;
    const int k = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = a.l_bin[k], d = a.l_d[k], nst = a.l_nstar[k];
    const int D = a.D, S = a.S;
    // dynamic shared memory: P, A (D x D float-float pairs), the learner's design rows (float4 + first
    // column per bin), u for one chunk of bins, the second cluster half's partial sums and,
    // when it fits, the column-major design
    extern __shared__ __align__(16) double dsm[];
    float2* Ps = reinterpret_cast<float2*>(dsm);            // float-float pairs (hi, lo)
    float2* As = Ps + (size_t)D * D;
    DF* u_s = reinterpret_cast<DF*>(As + (size_t)D * D);                          // [2][kSolveChunk] float-float
    long long* pb = reinterpret_cast<long long*>(u_s + 2 * kSolveChunk);          // [2][kSolveChunk]
    float4* zb_s = reinterpret_cast<float4*>(pb + 2 * kSolveChunk);              // [nst] when staged
    int* zc_s = reinterpret_cast<int*>(zb_s + (a.stage_v ? S : 0));
    float* zt_s = reinterpret_cast<float*>(zc_s + (a.stage_v ? ((S + 3) & ~3) : 0));   // [4 nst] when staged
    float* zl_s = zt_s + (a.stage_z ? kMaxNnz * S : 0);                                 // low parts, [4 nst]
    __shared__ DF s_s[2][kMaxD];
    __shared__ double th_s[2][kMaxD];
    __shared__ DF term[2][kMaxD];
    __shared__ bool is_last;

    // ---- static per-learner data (independent of this iteration), fetched before waiting for
    // the scatter so that it overlaps the scatter's tail: the design (asynchronous copies), its
    // column ranges, the first chunk's cluster range and, when the model never switches caches
    // (no HCWB), P and A of phase 0
    {
        if (a.stage_v) {
            const float4* zb_g = reinterpret_cast<const float4*>(a.zb) + (int64_t)k * S;
            const int* zc_g = a.zcol + (int64_t)k * S;
            for (int e = tid; e < nst; e += blockDim.x) {
                cp_async16(zb_s + e, zb_g + e);
                cp_async4(zc_s + e, zc_g + e);
            }
        }
        if (a.stage_z) {
            const float4* zt4 = reinterpret_cast<const float4*>(a.ztab + (int64_t)k * kMaxNnz * S);
            const float4* zl4 = reinterpret_cast<const float4*>(a.ztab_lo + (int64_t)k * kMaxNnz * S);
            for (int e = tid; e < nst; e += blockDim.x) {
                cp_async16(reinterpret_cast<float4*>(zt_s) + e, zt4 + e);
                cp_async16(reinterpret_cast<float4*>(zl_s) + e, zl4 + e);
            }
        }
    }
    auto stage_pa = [&](int ph) {          // P and A of the cache `ph`
        const float2* Pk = a.P + ((int64_t)ph * a.K + k) * D * D;
        const float2* Ak = a.A + ((int64_t)ph * a.K + k) * D * D;
        for (int e = tid; e < D * D; e += blockDim.x) {
            cp_async8(Ps + e, Pk + e);
            cp_async8(As + e, Ak + e);
        }
    };
    if (!a.hybrid) stage_pa(0);
    const float* zt = a.stage_z ? zt_s : a.ztab + (int64_t)k * kMaxNnz * S;
    const float* ztl = a.stage_z ? zl_s : a.ztab_lo + (int64_t)k * kMaxNnz * S;
    const float4* zbp = a.stage_v ? zb_s : reinterpret_cast<const float4*>(a.zb) + (int64_t)k * S;
    const int* zcp = a.stage_v ? zc_s : a.zcol + (int64_t)k * S;
    int c_lo[kColsPerWarp], c_len[kColsPerWarp], c_off[kColsPerWarp];
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c) {
        const int j = warp + c * NW;
        c_lo[c] = 0;
        c_len[c] = 0;
        c_off[c] = 0;
        if (j < d) {
            c_lo[c] = __ldg(a.crange + ((int64_t)k * D + j) * 2);
            c_len[c] = __ldg(a.crange + ((int64_t)k * D + j) * 2 + 1) - c_lo[c];
            c_off[c] = __ldg(a.toff + (int64_t)k * D + j);
        }
    }
    if (tid < 2 * kMaxD) {
        th_s[tid / kMaxD][tid % kMaxD] = 0.0;
        s_s[tid / kMaxD][tid % kMaxD] = DF{0.0f, 0.0f};
    }
    // Thread (i, half) sums bins 4i..4i+3 of a chunk over the clusters of parity `half`; the
    // clusters holding a bin are those of its slot (binning group x bin range)
    const int g = b / a.FE, f = b - g * a.FE;
    const int gi = tid & (kSolveThreads / 2 - 1), half = tid / (kSolveThreads / 2);
    auto chunk_clusters = [&](int L0, int L1, int& c0, int& c1, int& lb) {
        c0 = c1 = lb = 0;
        if (4 * gi < L1 - L0) {
            const int l0 = L0 + 4 * gi;
            const int br = l0 / a.nb_cta;
            lb = l0 - br * a.nb_cta;
            const int slot = g * a.bin_ranges + br;
            c0 = __ldg(a.slot_c0 + slot);
            c1 = __ldg(a.slot_c0 + slot + 1);
        }
    };
    int c0n, c1n, lbn;
    chunk_clusters(0, min(nst, kSolveChunk), c0n, c1n, lbn);

    grid_dep_wait();                   // histograms and iteration state from here on
    grid_dep_launch();                 // the next row pass may be scheduled on idle SMs
    const DevState st = *a.state;      // first used once the first chunk's loads are in flight
    const int mode = st.mode;
    // without HCWB the channel count never changes (CWB one, ACWB two) and needs no state
    const int C = a.hybrid ? ((mode == kModeACWB) ? 2 : 1) : a.cmax;
    if (a.hybrid) stage_pa((mode == kModeACWB) ? 0 : st.phase);

    // ---- u = sum of the slot's partial histograms, then s = Z^b^T u, in chunks of bins
    const int64_t cl_stride = (int64_t)a.cmax * a.F * a.nb_cta;
    DF acc0[kColsPerWarp], acc1[kColsPerWarp];
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c) acc0[c] = acc1[c] = DF{0.0f, 0.0f};
    for (int L0 = 0; L0 < nst; L0 += kSolveChunk) {
        const int L1 = min(nst, L0 + kSolveChunk);
        const bool mine = 4 * gi < L1 - L0;
        int c0 = c0n, c1 = c1n, lb = lbn;
        if (L0 > 0) {
            if (a.bin_ranges == 1) {
                // one bin range: every chunk's bins lie in the slot of chunk 0 (no table lookup)
                c0 = mine ? c0n : 0;
                c1 = mine ? c1n : 0;
                lb = mine ? L0 + 4 * gi : 0;
            } else {
                chunk_clusters(L0, L1, c0, c1, lb);
            }
        }
        long long it0[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        if (a.u64) {
            // row shards: the exchanged exact sums of every shard's histograms stand for the partials
            c0 = c1 = 0;
            if (half == 0 && mine)
                for (int t = 0; t < 4; ++t) {
                    const int l = L0 + 4 * gi + t;
                    it0[0][t] = l < nst ? __ldcg(a.u64 + (int64_t)b * S + l) : 0;
                }
        }
        float ft[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        float fc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        for (int cc = c0 + half; cc < c1; cc += 2 * kSolveBatch) {
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                if (ch < C) {           // a guard, not a break: the loop stays unrolled, the sums in registers
                const float* base = a.part + ((int64_t)ch * a.F + f) * a.nb_cta + lb;
                int4 x[kSolveBatch];
#pragma unroll
                for (int q = 0; q < kSolveBatch; ++q) {
                    const int c = cc + 2 * q;
                    x[q] = c < c1 ? __ldcg(reinterpret_cast<const int4*>(base + c * cl_stride)) : make_int4(0, 0, 0, 0);
                }
#pragma unroll
                for (int q = 0; q < kSolveBatch; ++q) {
                    if (INT_ACC) {
                        it0[ch][0] += x[q].x; it0[ch][1] += x[q].y; it0[ch][2] += x[q].z; it0[ch][3] += x[q].w;
                    } else {
                        const float xv[4] = {__int_as_float(x[q].x), __int_as_float(x[q].y), __int_as_float(x[q].z),
                                             __int_as_float(x[q].w)};
#pragma unroll
                        for (int t = 0; t < 4; ++t) {       // compensated sum
                            const float y = xv[t] - fc[ch][t];
                            const float tt = ft[ch][t] + y;
                            fc[ch][t] = (tt - ft[ch][t]) - y;
                            ft[ch][t] = tt;
                        }
                    }
                }
                }
            }
        }
        // the odd-cluster half hands its sums to the even half
        if (half == 1 && mine) {
#pragma unroll
            for (int ch = 0; ch < 2; ++ch)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (ch >= C) continue;
                    if (INT_ACC) pb[ch * kSolveChunk + 4 * gi + t] = it0[ch][t];
                    else reinterpret_cast<float*>(pb)[ch * kSolveChunk + 4 * gi + t] = ft[ch][t] - fc[ch][t];
                }
        }
        __syncthreads();
        if (half == 0 && mine) {
            float scl0 = 1.0f, scl1 = 1.0f;
            if (INT_ACC) {
                // (selects, not an index: a run-time index into the state copy would put it in local memory)
                const int cl2 = (a.hybrid && mode == kModeACWB) ? st.cnt_log2[1] : st.cnt_log2[0];
                scl0 = a.direct ? pow2f(-st.fix_exp) : pow2f(-fixed_scale(st.rmax_bits[0], cl2));
                scl1 = pow2f(-fixed_scale(st.rmax_bits[1], cl2));
            }
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                if (ch >= C) continue;
                DF o[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (INT_ACC) {
                        // the exact integer sum as a float-float pair (48 bits), power-of-two scale
                        const long long tot = it0[ch][t] + pb[ch * kSolveChunk + 4 * gi + t];
                        o[t] = df_scale(df_of_ll(tot), ch ? scl1 : scl0);
                    } else {
                        o[t] = df_add(DF{ft[ch][t], -fc[ch][t]},
                                      DF{reinterpret_cast<float*>(pb)[ch * kSolveChunk + 4 * gi + t], 0.0f});
                    }
                }
                *reinterpret_cast<float4*>(u_s + ch * kSolveChunk + 4 * gi) = make_float4(o[0].hi, o[0].lo, o[1].hi, o[1].lo);
                *reinterpret_cast<float4*>(u_s + ch * kSolveChunk + 4 * gi + 2) = make_float4(o[2].hi, o[2].lo, o[3].hi, o[3].lo);
            }
        }
        if (L0 == 0) cp_async_wait_all();              // the design must be in shared memory before s
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kColsPerWarp; ++c) {
            const int from = max(c_lo[c], L0), to = min(c_lo[c] + c_len[c], L1);
            const float* zc = zt + c_off[c] - c_lo[c];
            const float* zcl = ztl + c_off[c] - c_lo[c];
            for (int t = from + lane; t < to; t += 32) {
                // s in float-float: the design as (hi, lo) pairs times the float-float sums
                const DF z = {zc[t], zcl[t]};
                acc0[c] = df_add(acc0[c], df_mul(z, u_s[t - L0]));
                if (C == 2) acc1[c] = df_add(acc1[c], df_mul(z, u_s[kSolveChunk + t - L0]));
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c) {
        const int j = warp + c * NW;
        if (j >= d) break;                    // warp-uniform
        for (int o = 16; o > 0; o >>= 1) acc0[c] = df_add(acc0[c], df_shfl_xor(acc0[c], o));
        if (C == 2)
            for (int o = 16; o > 0; o >>= 1) acc1[c] = df_add(acc1[c], df_shfl_xor(acc1[c], o));
        if (lane == 0) {
            s_s[0][j] = acc0[c];
            s_s[1][j] = acc1[c];
        }
    }
    __syncthreads();

    // ---- theta = P s and t = A s together in float-float arithmetic (s is an FP32 vector; P and A
    // are float-float pairs, so every product and sum carries about 44 bits and the FP64 pipe,
    // a small fraction of the FP32 rate here, stays out of the loop): eight lanes per row,
    // partial sums over j = q mod 8.  The criterion Q = theta^T G theta - 2 theta^T s = s^T A s = s . t
    const int rows8 = C * d * 8;
    for (int base = 0; base < 2 * rows8; base += blockDim.x) {
        const int e = base + tid;
        const bool valid = e < 2 * rows8;
        const int mat = valid && e >= rows8 ? 1 : 0;
        const int r = e - mat * rows8;
        const int ch = valid ? r / (8 * d) : 0;
        const int rem = r - ch * 8 * d;
        const int i = rem >> 3, q = rem & 7;
        const float2* Mx = mat ? As : Ps;
        DF p = {0.0f, 0.0f};
        if (valid)
            for (int j = q; j < d; j += 8) {
                const float2 mij = Mx[i * D + j];
                p = df_add(p, df_mul(DF{mij.x, mij.y}, s_s[ch][j]));
            }
#pragma unroll 1
        for (int o = 1; o < 8; o <<= 1) {
            const DF other = {__shfl_xor_sync(0xffffffffu, p.hi, o), __shfl_xor_sync(0xffffffffu, p.lo, o)};
            p = df_add(p, other);
        }
        if (valid && q == 0) {
            if (mat) term[ch][i] = df_mul(p, s_s[ch][i]);
            else th_s[ch][i] = (double)p.hi + (double)p.lo;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // Q = sum_i s_i t_i per channel: fixed-order tree over the warp.  The criteria are all
        // the argmin needs, so the ticket is taken right after they are stored and its round
        // trip overlaps the update table below.
        double qv[2] = {0.0, 0.0};
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            if (ch >= C) continue;
            DF x = {0.0f, 0.0f};
#pragma unroll 1
            for (int i = lane; i < d; i += 32) x = df_add(x, term[ch][i]);
#pragma unroll 1
            for (int o = 16; o > 0; o >>= 1) {
                const DF other = {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
                x = df_add(x, other);
            }
            qv[ch] = (double)x.hi + (double)x.lo;
        }
        if (lane == 0) {
            a.q_it[k] = qv[0];
            if (C == 2) a.q_it[(int64_t)a.K + k] = qv[1];
            fence_acq_rel_gpu();
            const unsigned t = atomicAdd(&a.state->ticket_solve, 1u);
            is_last = (t == gridDim.x - 1);
        }
    }
    for (int e = tid; e < C * D; e += blockDim.x) {
        const int ch = e / D, i = e - (e / D) * D;
        a.theta_it[((int64_t)ch * a.K + k) * D + i] = th_s[ch][i];
    }
    // ---- update table of this learner, v_k = Z^b theta (FP32), and max |v_k| of channel 0
    float vm = 0.0f;
    for (int e = tid; e < C * nst; e += blockDim.x) {
        const int ch = e >= nst ? 1 : 0, l = e - ch * nst;
        const int c0 = zcp[l];
        const float4 z = zbp[l];
        float acc = 0.0f;
        if (c0 < D) acc = fmaf(z.x, (float)th_s[ch][c0], acc);
        if (c0 + 1 < D) acc = fmaf(z.y, (float)th_s[ch][c0 + 1], acc);
        if (c0 + 2 < D) acc = fmaf(z.z, (float)th_s[ch][c0 + 2], acc);
        if (c0 + 3 < D) acc = fmaf(z.w, (float)th_s[ch][c0 + 3], acc);
        a.v[((int64_t)ch * a.K + k) * S + l] = acc;
        if (ch == 0) vm = fmaxf(vm, fabsf(acc));
    }
    for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    __shared__ float vm_w[NW];
    if (lane == 0) vm_w[warp] = vm;
    __syncthreads();
    if (tid == 0) {
        float mx = 0.0f;
        for (int w2 = 0; w2 < NW; ++w2) mx = fmaxf(mx, vm_w[w2]);
        a.vmax[k] = mx;
    }
    // ---- last CTA: argmin per channel, trace, state -- one warp (no block barriers on the
    // iteration's critical path)
    if (warp != 0) return;
    __syncwarp();
    if (!is_last) return;
    fence_acq_rel_gpu();
    const long long kInf = order_key(INFINITY);
    Best2 cand[2] = {{kInf, kInf, -1}, {kInf, kInf, -1}};
    bool bad = false;
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
        if (ch >= C) continue;
        Best2 x = {kInf, kInf, -1};
#pragma unroll 1
        for (int k0 = 0; k0 < a.K; k0 += 4 * 32) {
            long long qb[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {       // the loads of a pass issued together
                const int kk = k0 + 32 * t + lane;
                qb[t] = kk < a.K ? __ldcg(reinterpret_cast<const long long*>(a.q_it) + (int64_t)ch * a.K + kk) : 0LL;
            }
            // a rolled loop: this code runs once per iteration on one SM, where every line of it
            // is an instruction-cache miss, so it is kept short
#pragma unroll 1
            for (int t = 0; t < 4; ++t) {
                const int kk = k0 + 32 * t + lane;
                if (kk >= a.K) continue;
                const long long qt = t == 0 ? qb[0] : (t == 1 ? qb[1] : (t == 2 ? qb[2] : qb[3]));
                // integer tests only: -0 ties with +0, inf and NaN are flagged
                long long key = (qt & 0x7fffffffffffffffLL) == 0 ? 0LL : order_key(__longlong_as_double(qt));
                if ((qt & 0x7ff0000000000000LL) == 0x7ff0000000000000LL) {
                    bad = true;
                    key = kInf;
                }
                x = best2_merge(x, Best2{key, kInf, kk});
            }
        }
#pragma unroll 1
        for (int o = 16; o > 0; o >>= 1) x = best2_merge(x, best2_shfl(x, o));
        cand[ch] = x;
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        const int it = st.m;
        const bool trace_ok = it < a.trace_cap;
        DevState* S_ = a.state;
        int best_k[2] = {-1, -1};
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
            if (ch >= C) continue;
            const Best2 x = cand[ch];
            int i1 = x.k1 < 0 ? 0 : x.k1;
            if (ch == 0 && trace_ok && a.forced) {
                const int fk = a.forced[it];
                if (fk >= 0 && fk < a.K) i1 = fk;
            }
            best_k[ch] = i1;
            if (trace_ok) {
                a.tr_k[2 * it + ch] = i1;
                if (ch == 0) {
                    a.tr_q[2 * it] = key_value(x.q1);
                    a.tr_q[2 * it + 1] = key_value(x.q2);
                }
            }
        }
        if (trace_ok) {
            a.tr_mode[it] = mode;
            if (C == 1) a.tr_k[2 * it + 1] = -1;
        } else {
            atomicOr(&S_->err, kErrIndex);
        }
        if (bad) atomicOr(&S_->err, kErrNonFinite);
        S_->k_sel = best_k[0];
        S_->k_cor = (C == 2) ? best_k[1] : -1;
        S_->pend_mode = mode;
        S_->m = st.m + 1;
        S_->rprev_bits = S_->rmax_bits[0];   // max |w r| of this iteration (input of the persistent path's bound)
        S_->resid_path = a.direct ? 2 : 0;
        S_->rmax_bits[0] = 0u;           // the next row pass takes its maxima with atomicMax
        S_->rmax_bits[1] = 0u;
        S_->ticket_solve = 0;
    }
}

// Aggregated parameters from the trace (eq. (1); Sec. 3.2.1 for ACWB iterations).
__global__ void k_aggregate(int K, int D, int done, const int32_t* __restrict__ l_d, const int32_t* __restrict__ tr_k,
                            const int32_t* __restrict__ tr_mode, const double* __restrict__ tr_theta, double nu,
                            double gamma, double* __restrict__ coef)
{
    const int k = blockIdx.x, j = threadIdx.x;
    if (j >= D) return;
    double tf = 0.0, th = 0.0;
    for (int t = 0; t < done; ++t) {
        const int md = tr_mode[t], ks = tr_k[2 * t], kc = tr_k[2 * t + 1];
        if (md == kModeCWB) {
            if (ks == k) tf += nu * tr_theta[((int64_t)2 * t) * D + j];
        } else {
            const double thm = 2.0 / ((double)t + 2.0);
            tf = (1.0 - thm) * tf + thm * th;
            if (ks == k) tf += nu * tr_theta[((int64_t)2 * t) * D + j];
            if (kc == k) th += (gamma * nu / thm) * tr_theta[((int64_t)2 * t + 1) * D + j];
        }
    }
    coef[(int64_t)k * D + j] = tf;
    coef[((int64_t)K + k) * D + j] = th;
}

int num_sms(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

int rows_grid(const cwb_model* m)
{
    int64_t g = (m->n_pad / (4 * row_groups(m->accel)) + kRowThreads - 1) / kRowThreads;
    int64_t cap = (int64_t)num_sms(m->device) * 4;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

RowArgs row_args(cwb_model* m)
{
    RowArgs a;
    a.state = m->state;
    a.ind = m->ind;
    a.n = m->n;
    a.n_tr = m->n_tr;
    a.n_pad = m->n_pad;
    a.y = m->y;
    a.y_lo = m->y_lo;
    a.w = m->w;
    a.f = m->f;
    a.h = m->h;
    a.c = m->c;
    a.rw = m->rw;
    a.v = m->v;
    a.l_bin = m->l_bin;
    a.S = m->nstar_max;
    a.K = m->K;
    a.D = m->d_max;
    a.theta_it = m->theta_it;
    a.tr_theta = m->tr_theta;
    a.trace_cap = m->trace_cap;
    a.loss = m->cfg.loss;
    a.nu = m->cfg.nu;
    a.gamma = m->cfg.gamma;
    a.nu_hi = (float)m->cfg.nu;
    a.nu_lo = (float)(m->cfg.nu - (double)a.nu_hi);
    a.hybrid = m->hybrid ? 1 : 0;
    a.patience = m->cfg.patience;
    a.risk_part = m->risk_part;
    a.direct = direct_q(m) ? 1 : 0;
    a.wmax = (float)m->wmax;
    a.vmax = m->vmax;
    return a;
}

template <int KIND>
void launch_rows(cwb_model* m, cudaStream_t s)
{
    RowArgs a = row_args(m);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(rows_grid(m), 1, 1);
    cfg.blockDim = dim3(kRowThreads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = m->use_pdl ? 1 : 0;
    if (m->accel) {
        if (m->ind_bytes == 1) cudaLaunchKernelEx(&cfg, k_rows<KIND, uint8_t, true>, a);
        else cudaLaunchKernelEx(&cfg, k_rows<KIND, uint16_t, true>, a);
    } else {
        if (m->ind_bytes == 1) cudaLaunchKernelEx(&cfg, k_rows<KIND, uint8_t, false>, a);
        else cudaLaunchKernelEx(&cfg, k_rows<KIND, uint16_t, false>, a);
    }
}

template <typename IndT, int CMAX, bool INT_ACC>
cudaError_t launch_scatter_t(cwb_model* m, cudaStream_t s, const ScatterArgs& a)
{
    const ScatterPlan& P = m->plan;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.clusters * P.cs, 1, 1);
    cfg.blockDim = dim3(P.threads, 1, 1);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = m->use_pdl ? 2 : 1;
    if (P.bin_ranges > 1) return cudaLaunchKernelEx(&cfg, k_scatter<IndT, CMAX, INT_ACC, true, -1>, m->tmap, a);
    if (P.f_lane == 32) return cudaLaunchKernelEx(&cfg, k_scatter<IndT, CMAX, INT_ACC, false, 5>, m->tmap, a);
    if (P.f_lane == 16) return cudaLaunchKernelEx(&cfg, k_scatter<IndT, CMAX, INT_ACC, false, 4>, m->tmap, a);
    if (P.f_lane == 8) return cudaLaunchKernelEx(&cfg, k_scatter<IndT, CMAX, INT_ACC, false, 3>, m->tmap, a);
    return cudaLaunchKernelEx(&cfg, k_scatter<IndT, CMAX, INT_ACC, false, -1>, m->tmap, a);
}

constexpr int kSleepStages = 6;                    // rings at least this deep wait with a suspend-time hint

ScatterArgs scatter_args(cwb_model* m)
{
    const ScatterPlan& P = m->plan;
    ScatterArgs a;
    a.state = m->state;
    a.rw = m->rw;
    a.n = m->n;
    a.n_tr = m->n_tr;
    a.n_pad = m->n_pad;
    a.B = m->B;
    a.F = P.f_lane;
    a.FE = P.fe;
    a.bin_ranges = P.bin_ranges;
    a.nb_cta = P.nb_cta;
    a.ch_stride = P.ch_stride;
    a.stage_rows = P.stage_rows;
    a.stages = P.stages;
    a.nb_box = P.nb_box;
    a.box_bytes = P.box_bytes;
    a.unit_rows = 16 / m->ind_bytes;
    a.cs = P.cs;
    a.cluster_slot = m->cluster_slot;
    a.slot_c0 = m->slot_c0;
    a.hybrid = m->hybrid ? 1 : 0;
    a.ind_off = P.ind_off;
    a.r_off = P.r_off;
    a.q_off = P.q_off;
    a.hist_off = P.hist_off;
    a.bar_off = P.bar_off;
    a.stage_ind_bytes = P.stage_ind_bytes;
    a.stage_r_bytes = P.stage_r_bytes;
    a.part = m->part;
    a.stage_cb = P.stage_cb;
    a.err = &m->state->err;
    a.count_rows = -1;
    a.wait_cycles = m->wait_cycles;
    a.withhold = m->withhold_tile;
    a.direct = direct_q(m) ? 1 : 0;
    a.sleep_waits = m->sleep_waits >= 0 ? m->sleep_waits : (P.stages >= kSleepStages ? 1 : 0);
    return a;
}

cudaError_t launch_scatter_args(cwb_model* m, cudaStream_t s, const ScatterArgs& a, bool int_acc)
{
    const bool two = m->plan.cmax == 2;
    if (m->ind_bytes == 1) {
        if (two) return int_acc ? launch_scatter_t<uint8_t, 2, true>(m, s, a) : launch_scatter_t<uint8_t, 2, false>(m, s, a);
        return int_acc ? launch_scatter_t<uint8_t, 1, true>(m, s, a) : launch_scatter_t<uint8_t, 1, false>(m, s, a);
    }
    if (two) return int_acc ? launch_scatter_t<uint16_t, 2, true>(m, s, a) : launch_scatter_t<uint16_t, 2, false>(m, s, a);
    return int_acc ? launch_scatter_t<uint16_t, 1, true>(m, s, a) : launch_scatter_t<uint16_t, 1, false>(m, s, a);
}

void launch_scatter(cwb_model* m, cudaStream_t s)
{
    launch_scatter_args(m, s, scatter_args(m), m->plan.int_acc);
}

int solve_threads(const cwb_model* m) { return m->nstar_max > solve_chunk(256) ? 512 : 256; }

size_t solve_smem(const cwb_model* m, bool stage_v, bool stage_z)
{
    const size_t S = m->nstar_max;
    const size_t chunk = solve_chunk(solve_threads(m));
    size_t b = sizeof(float2) * 2 * (size_t)m->d_max * m->d_max;        // P, A (float-float pairs)
    b += sizeof(float2) * 2 * chunk + sizeof(long long) * 2 * chunk;     // u chunk (float-float), half sums
    if (stage_v) b += 16 * S + 4 * ((S + 3) & ~size_t(3));              // design rows, first columns
    if (stage_z) b += 2 * sizeof(float) * kMaxNnz * S;                   // column-major design (hi, lo)
    return b;
}

void launch_solve(cwb_model* m, cudaStream_t s)
{
    const ScatterPlan& P = m->plan;
    SolveArgs a;
    a.state = m->state;
    a.K = m->K;
    a.D = m->d_max;
    a.S = m->nstar_max;
    a.part = m->part;
    a.slot_c0 = m->slot_c0;
    a.F = P.f_lane;
    a.FE = P.fe;
    a.cmax = P.cmax;
    a.nb_cta = P.nb_cta;
    a.bin_ranges = P.bin_ranges;
    a.hybrid = m->hybrid ? 1 : 0;
    a.stage_v = P.solve_stage_v ? 1 : 0;
    a.stage_z = P.solve_stage_z ? 1 : 0;
    a.zb = m->zb;
    a.zcol = m->zcol;
    a.crange = m->crange;
    a.toff = m->toff;
    a.ztab = m->ztab;
    a.ztab_lo = m->ztab_lo;
    a.l_bin = m->l_bin;
    a.l_d = m->l_d;
    a.l_nstar = m->l_nstar;
    a.A = m->Adf;
    a.P = m->Pdf;
    a.theta_it = m->theta_it;
    a.q_it = m->q_it;
    a.v = m->v;
    a.tr_k = m->tr_k;
    a.tr_mode = m->tr_mode;
    a.tr_q = m->tr_q;
    a.forced = m->forced;
    a.trace_cap = m->trace_cap;
    a.vmax = m->vmax;
    a.u64 = m->solve_u64;
    a.direct = direct_q(m) ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(m->K, 1, 1);
    const int threads = solve_threads(m);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = solve_smem(m, P.solve_stage_v, P.solve_stage_z);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = m->use_pdl ? 1 : 0;
    if (threads == 512) {
        if (P.int_acc) cudaLaunchKernelEx(&cfg, k_solve<true, 512>, a);
        else cudaLaunchKernelEx(&cfg, k_solve<false, 512>, a);
    } else {
        if (P.int_acc) cudaLaunchKernelEx(&cfg, k_solve<true, 256>, a);
        else cudaLaunchKernelEx(&cfg, k_solve<false, 256>, a);
    }
}

template <typename IndT, int CMAX>
cwb_status prepare_scatter_kernel(cwb_model* m, int cs, int* active_clusters)
{
    const ScatterPlan& P = m->plan;
    // every instantiation a launch may pick
    const void* kernels[] = {
        (const void*)k_scatter<IndT, CMAX, true, true, -1>,  (const void*)k_scatter<IndT, CMAX, false, true, -1>,
        (const void*)k_scatter<IndT, CMAX, true, false, 5>,  (const void*)k_scatter<IndT, CMAX, false, false, 5>,
        (const void*)k_scatter<IndT, CMAX, true, false, 4>,  (const void*)k_scatter<IndT, CMAX, false, false, 4>,
        (const void*)k_scatter<IndT, CMAX, true, false, 3>,  (const void*)k_scatter<IndT, CMAX, false, false, 3>,
        (const void*)k_scatter<IndT, CMAX, true, false, -1>, (const void*)k_scatter<IndT, CMAX, false, false, -1>};
    for (const void* kf : kernels) {
        CWB_CUDA_TRY(allow_max_dynamic_smem(kf, m->device));
        if (cs > 8) CWB_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * 64, 1, 1);
    cfg.blockDim = dim3(P.threads, 1, 1);
    cfg.dynamicSmemBytes = P.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, k_scatter<IndT, CMAX, true, false, -1>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    *active_clusters = n;
    return CWB_OK;
}

cwb_status active_clusters_for(cwb_model* m, int cs, int* n)
{
    if (m->ind_bytes == 1) {
        if (m->plan.cmax == 2) return prepare_scatter_kernel<uint8_t, 2>(m, cs, n);
        return prepare_scatter_kernel<uint8_t, 1>(m, cs, n);
    }
    if (m->plan.cmax == 2) return prepare_scatter_kernel<uint16_t, 2>(m, cs, n);
    return prepare_scatter_kernel<uint16_t, 1>(m, cs, n);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn()
{
    // looked up once (a function-local static is initialised once even when models are created on
    // several host threads at the same time)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        EncodeTiledFn f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
        return f;
    }();
    return fn;
}

}  // namespace

// One iteration's launches.  With a profiling mask (only while capturing the
// profiling graph) the kernels of the selected classes are bracketed by external
// event-record nodes on placeholder events; the placeholders are replaced by fresh
// events before every launch of that graph.
void enqueue_iteration(cwb_model* m, cudaStream_t s, int mask)
{
    auto mark = [&](int cls, int edge) {
        if (mask & (1 << cls)) cudaEventRecordWithFlags(m->prof_ph[2 * cls + edge], s, cudaEventRecordExternal);
    };
    mark(0, 0);
    launch_rows<kRowsFused>(m, s);
    if (m->hybrid) launch_rows<kRowsResid>(m, s);        // work only in the iteration that switches to CWB
    mark(0, 1);
    mark(1, 0);
    launch_scatter(m, s);
    mark(1, 1);
    mark(2, 0);
    launch_solve(m, s);
    mark(2, 1);
}


// Frees the buffers a scatter plan owns (cluster tables, partial histograms) and the graphs
// that captured them.
void release_scatter_plan(cwb_model* m)
{
    if (m->stream) cudaStreamSynchronize(m->stream);
    dev_free(m->cluster_slot);
    dev_free(m->slot_c0);
    dev_free(m->part);
    m->cluster_slot = nullptr;
    m->slot_c0 = nullptr;
    m->part = nullptr;
    release_graphs(m);
}

// Scatter decomposition.  max_ctas > 0 caps the grid (the autotuner's knob); 0 sizes it by the
// work: every resident CTA for large inputs, about kTilesPerCta tile-slots per CTA for small ones,
// so that small fits leave SMs to others.  cs_req > 0 forces the cluster size when it can be resident.
constexpr int kTilesPerCta = 8;
constexpr int kMaxScatterStages = 8;               // ring stages of the scatter (shared memory permitting)

cwb_status plan_scatter(cwb_model* m, int max_ctas, int cs_req)
{
    int optin = 0, sms = num_sms(m->device);
    CWB_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    const int budget = optin - 1024 - 512;          // alignment slack and mbarriers
    const int cmax = m->accel ? 2 : 1;
    const int elem = m->ind_bytes;
    const int nbins = (m->nstar_max + 3) & ~3;     // bins per binning rounded to 16-byte rows
    const int B = m->B;
    int pow2B = 1;
    while (pow2B < B) pow2B <<= 1;
    ScatterPlan P{};
    P.cmax = cmax;
    P.stage_rows = kStageRows;
    P.nb_box = 1;
    P.bin_ranges = 1;
    auto ch_stride_for = [&](int nb, int F) {
        int base = nb * F;
        int pad = (cmax == 2) ? ((16 - base % 32) + 32) % 32 : 0;
        return base + pad;
    };
    auto hist_bytes = [&](int nb, int F) { return ((cmax * ch_stride_for(nb, F) * 4 + 1023) / 1024) * 1024; };
    // a stage's index box starts on a 1024-byte boundary (the 128-byte swizzle pattern repeats every 1 KB)
    auto stage_bytes = [&](int F) { return ((F * P.stage_rows * elem + 1023) / 1024) * 1024 + cmax * P.stage_rows * 4; };
    P.f_lane = 0;
    int f_req = 0;
    if (const char* env = std::getenv("CWB_F_LANE")) f_req = std::atoi(env);
    for (int F = 32; F >= 1; F >>= 1) {
        if (F * cmax > 32 || F > pow2B) continue;
        if (f_req > 0 && F > f_req) continue;
        if (hist_bytes(nbins, F) + 3 * stage_bytes(F) <= budget) {
            P.f_lane = F;
            break;
        }
    }
    if (P.f_lane == 0) {
        P.f_lane = 1;
        while (hist_bytes((nbins + P.bin_ranges - 1) / P.bin_ranges, 1) + 3 * stage_bytes(1) > budget) ++P.bin_ranges;
    }
    const int F = P.f_lane;
    P.groups = (B + F - 1) / F;
    P.fe = (B + P.groups - 1) / P.groups;          // binnings per group, balanced across groups
    P.nb_cta = (((nbins + P.bin_ranges - 1) / P.bin_ranges) + 3) & ~3;
    P.nbins_pad = P.nb_cta * P.bin_ranges;
    P.ch_stride = ch_stride_for(P.nb_cta, F);
    P.box_bytes = P.fe * P.stage_rows * elem;
    P.stage_ind_bytes = (uint32_t)(((P.box_bytes + 1023) / 1024) * 1024);
    P.stage_r_bytes = (uint32_t)(cmax * P.stage_rows * 4);
    const int hb = hist_bytes(P.nb_cta, F);
    P.stages = std::min(kMaxScatterStages, (budget - hb) / stage_bytes(P.fe));
    for (;;) {
        P.ind_off = 0;
        P.r_off = P.ind_off + (uint32_t)P.stages * P.stage_ind_bytes;
        P.q_off = P.r_off;                              // fixed point replaces the residuals in place
        P.hist_off = ((P.q_off + (uint32_t)P.stages * P.stage_r_bytes + 1023) / 1024) * 1024;
        P.bar_off = P.hist_off + (uint32_t)hb;
        P.smem = (size_t)P.bar_off + 3 * 8 * P.stages + 1024;   // + alignment slack of the dynamic base
        if (P.smem <= (size_t)optin || P.stages <= 1) break;
        --P.stages;
    }
    P.slots = P.groups * P.bin_ranges;
    P.threads = kScatterThreads;
    m->plan = P;

    // cluster size: the largest that keeps (nearly) every SM busy; CWB_CLUSTER_SIZE
    // (1, 2, 4, 8 or 16) overrides the choice when that size can be resident
    int best_cs = 1, best_used = 0;
    for (int cs : {8, 4, 2, 1}) {
        int act = 0;
        CWB_TRY(active_clusters_for(m, cs, &act));
        int used = act * cs;
        P.active_ctas[cs == 8 ? 3 : cs == 4 ? 2 : cs == 2 ? 1 : 0] = used;
        if (used > best_used + sms / 50) {
            best_used = used;
            best_cs = cs;
        }
    }
    int want = cs_req;
    if (want <= 0)
        if (const char* env = std::getenv("CWB_CLUSTER_SIZE")) want = std::atoi(env);
    if (want > 0) {
        if (want == 1 || want == 2 || want == 4 || want == 8 || want == 16) {
            int act = 0;
            CWB_TRY(active_clusters_for(m, want, &act));
            if (act > 0) {
                best_cs = want;
                best_used = act * want;
            }
        }
    }
    if (best_used == 0) {
        set_error("the scatter kernel does not fit on this device");
        return CWB_ECUDA;
    }
    P.cs = best_cs;
    // clusters spread evenly over the slots (groups hold balanced numbers of binnings)
    int ctas = best_used;
    {
        const int64_t tiles = (m->n + kStageRows - 1) / kStageRows;
        const int64_t by_work = (tiles * P.slots + kTilesPerCta - 1) / kTilesPerCta;
        if (max_ctas > 0) ctas = std::min(ctas, max_ctas);
        else ctas = (int)std::min<int64_t>(ctas, by_work);
        ctas = std::max(ctas, P.slots * best_cs);
    }
    int total = std::max(ctas / best_cs, P.slots);
    std::vector<int> per(P.slots, total / P.slots);
    for (int sl = 0; sl < total % P.slots; ++sl) per[sl] += 1;
    // clusters are dealt to the slots in turn, so neighbouring CTAs stream the same rows of
    // different binning groups; partial histograms stay grouped by slot (slot_c0)
    std::vector<int32_t> slot_c0(P.slots + 1, 0), cl_slot, cl_in;
    int per_max = 0;
    for (int sl = 0; sl < P.slots; ++sl) {
        slot_c0[sl + 1] = slot_c0[sl] + per[sl];
        per_max = std::max(per_max, per[sl]);
    }
    for (int r = 0; r < per_max; ++r)
        for (int sl = 0; sl < P.slots; ++sl)
            if (r < per[sl]) {
                cl_slot.push_back(sl);
                cl_in.push_back(r);
            }
    P.clusters = (int)cl_slot.size();
    cl_slot.insert(cl_slot.end(), cl_in.begin(), cl_in.end());
    P.part_floats = (size_t)P.clusters * cmax * P.nb_cta * F;
    {
        // the cluster epilogue stages [F][cb + 1] values in the ring, which precedes the histograms
        const int bpr = ((P.nb_cta + P.cs - 1) / P.cs + 3) & ~3;
        const int fit = (((int)P.hist_off / (4 * F)) - 1) & ~3;
        P.stage_cb = std::min(bpr, fit);
        if (P.stage_cb < 4) {
            set_error("scatter plan: no room for the epilogue stage");
            return CWB_ECUDA;
        }
    }
    // the solve stages the learner's column-major design when it fits
    {
        const int solve_static = 8 * 1024;
        P.solve_stage_v = (int)solve_smem(m, true, false) + solve_static <= optin;
        P.solve_stage_z = P.solve_stage_v && (int)solve_smem(m, true, true) + solve_static <= optin;
        const int need = (int)solve_smem(m, P.solve_stage_v, P.solve_stage_z);
        if (need + solve_static > optin) {
            set_error("solve kernel: basis dimension too large for shared memory");
            return CWB_EINVAL;
        }
        for (const void* kf : {(const void*)k_solve<true, 512>, (const void*)k_solve<false, 512>,
                               (const void*)k_solve<true, 256>, (const void*)k_solve<false, 256>})
            CWB_CUDA_TRY(allow_max_dynamic_smem(kf, m->device));
    }
    m->plan = P;
    release_scatter_plan(m);
    CWB_TRY(dev_alloc((void**)&m->cluster_slot, sizeof(int32_t) * cl_slot.size(), m->stream));
    CWB_TRY(dev_alloc((void**)&m->slot_c0, sizeof(int32_t) * slot_c0.size(), m->stream));
    CWB_TRY(dev_alloc((void**)&m->part, sizeof(float) * std::max<size_t>(P.part_floats, 1), m->stream));
    CWB_CUDA_TRY(cudaMemcpyAsync(m->cluster_slot, cl_slot.data(), sizeof(int32_t) * cl_slot.size(),
                                 cudaMemcpyHostToDevice, m->stream));
    CWB_CUDA_TRY(cudaMemcpyAsync(m->slot_c0, slot_c0.data(), sizeof(int32_t) * slot_c0.size(), cudaMemcpyHostToDevice,
                                 m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));

    // tensor map of the index matrix [B][n_pad] viewed as {E rows, B binnings, n_pad / E chunks} with
    // E = 128 bytes of rows: one box is a tile's 256 rows of FE binnings, landing as 128-byte rows
    // [chunk][binning] with the 128-byte swizzle
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return CWB_ECUDA;
    }
    const int E = 128 / elem;
    cuuint64_t dims[3] = {(cuuint64_t)E, (cuuint64_t)B, (cuuint64_t)(m->n_pad / E)};
    cuuint64_t strides[2] = {(cuuint64_t)m->n_pad * elem, 128};
    cuuint32_t box[3] = {(cuuint32_t)E, (cuuint32_t)P.fe, (cuuint32_t)(P.stage_rows / E)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&m->tmap, elem == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, m->ind,
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return CWB_ECUDA;
    }
    return CWB_OK;
}

// Counting pass of the scatter (every row adds 1): the largest bin count any
// cluster accumulates bounds the fixed-point scale; extreme skew (> 8192 rows of
// one cluster in one bin) selects the FP32 accumulation instead.
cwb_status scatter_count_pass(cwb_model* m)
{
    const ScatterPlan& P = m->plan;
    const int passes = m->hybrid ? 2 : 1;
    CWB_CUDA_TRY(cudaMemsetAsync(&m->state->cnt_max[0], 0, sizeof(m->state->cnt_max), m->stream));
    for (int idx = 0; idx < passes; ++idx) {
        ScatterArgs a = scatter_args(m);
        a.count_rows = idx == 1 ? m->n_tr : m->n;
        a.wait_cycles = kWaitCycles;             // setup work: the default limit
        a.withhold = -1;
        a.direct = 0;                            // the converter writes the counting pass's ones
        CWB_CUDA_TRY(launch_scatter_args(m, m->stream, a, true));
        const int64_t total = (int64_t)P.clusters * P.nb_cta * P.f_lane;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(4 * num_sms(m->device), (total + 255) / 256));
        k_count_max<<<blocks, 256, 0, m->stream>>>(reinterpret_cast<const int*>(m->part), P.clusters, P.cmax,
                                                   P.nb_cta * P.f_lane, m->state, idx);
        k_count_log2<<<1, 32, 0, m->stream>>>(m->state, idx);
        CWB_CUDA_TRY(cudaGetLastError());
    }
    DevState st;
    CWB_CUDA_TRY(cudaMemcpyAsync(&st, m->state, sizeof(st), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (st.err) {
        set_error("scatter counting pass failed (device error flag " + std::to_string(st.err) + ")");
        return CWB_ECUDA;
    }
    const int worst = std::max(st.cnt_log2[0], passes > 1 ? st.cnt_log2[1] : 0);
    m->plan.int_acc = worst <= 13;
    return CWB_OK;
}

// Autotuner of the scatter decomposition: times `trials` scatter launches for each candidate
// grid size x cluster size on the model's own data and keeps the best.  objective 0 minimises the
// scatter's time (one fit on the GPU); 1 minimises its SM-time (CTAs x time), for fits that share
// the GPU.  The scatter alone changes no model state (its partial histograms are rewritten by the
// next iteration before they are read).
cwb_status autotune_scatter(cwb_model* m, int objective, int trials, double* best_us)
{
    const int sms = num_sms(m->device);
    trials = std::max(trials, 1);
    const int64_t tiles = (m->n + kStageRows - 1) / kStageRows;
    std::vector<std::pair<int, int>> cand;
    for (int cs : {2, 1})
        for (int ctas : {0, sms, sms / 2, sms / 4, sms / 8}) cand.push_back({ctas, cs});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CWB_CUDA_TRY(cudaEventCreate(&e0));
    CWB_CUDA_TRY(cudaEventCreate(&e1));
    double best = INFINITY, best_t = 0.0;
    std::pair<int, int> pick = {0, 0};
    cwb_status st = CWB_OK;
    std::vector<std::pair<int, int>> seen;
    for (auto c : cand) {
        if (c.first > 0 && (int64_t)c.first > tiles * 4 * m->plan.slots) continue;   // mostly idle CTAs
        st = plan_scatter(m, c.first, c.second);
        if (st != CWB_OK) break;
        const std::pair<int, int> got = {m->plan.clusters, m->plan.cs};
        if (std::find(seen.begin(), seen.end(), got) != seen.end()) continue;
        seen.push_back(got);
        st = scatter_count_pass(m);
        if (st != CWB_OK) break;
        launch_scatter(m, m->stream);                      // warm-up
        cudaEventRecord(e0, m->stream);
        for (int t = 0; t < trials; ++t) launch_scatter(m, m->stream);
        cudaEventRecord(e1, m->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = cuda_status(e, "autotune");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double t_us = 1e3 * ms / trials;
        const double cost = objective == 1 ? t_us * m->plan.clusters * m->plan.cs / sms : t_us;
        if (cost < best) {
            best = cost;
            best_t = t_us;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CWB_TRY(st);
    CWB_TRY(plan_scatter(m, pick.first, pick.second));
    CWB_TRY(scatter_count_pass(m));
    if (best_us) *best_us = best_t;
    return read_device_error(m);
}

cwb_status ensure_trace(cwb_model* m, int32_t need)
{
    if (need <= m->trace_cap) return CWB_OK;
    int32_t cap = std::max<int32_t>(need, std::max<int32_t>(1024, m->trace_cap * 2));
    const int D = m->d_max;
    cudaStream_t s = m->stream;
    int32_t *tk = nullptr, *tm = nullptr, *fo = nullptr;
    double *tt = nullptr, *tq = nullptr;
    CWB_TRY(dev_alloc((void**)&tk, sizeof(int32_t) * 2 * cap, s));
    CWB_TRY(dev_alloc((void**)&tm, sizeof(int32_t) * cap, s));
    CWB_TRY(dev_alloc((void**)&fo, sizeof(int32_t) * cap, s));
    CWB_TRY(dev_alloc((void**)&tt, sizeof(double) * 2 * (size_t)cap * D, s));
    CWB_TRY(dev_alloc((void**)&tq, sizeof(double) * 2 * (size_t)cap, s));
    CWB_CUDA_TRY(cudaMemsetAsync(fo, 0xff, sizeof(int32_t) * cap, s));   // -1: no override
    if (m->trace_cap > 0) {
        const size_t old = m->trace_cap;
        CWB_CUDA_TRY(cudaMemcpyAsync(tk, m->tr_k, sizeof(int32_t) * 2 * old, cudaMemcpyDeviceToDevice, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(tm, m->tr_mode, sizeof(int32_t) * old, cudaMemcpyDeviceToDevice, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(fo, m->forced, sizeof(int32_t) * old, cudaMemcpyDeviceToDevice, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(tt, m->tr_theta, sizeof(double) * 2 * old * D, cudaMemcpyDeviceToDevice, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(tq, m->tr_q, sizeof(double) * 2 * old, cudaMemcpyDeviceToDevice, s));
        CWB_CUDA_TRY(cudaStreamSynchronize(s));
        dev_free(m->tr_k);
        dev_free(m->tr_mode);
        dev_free(m->forced);
        dev_free(m->tr_theta);
        dev_free(m->tr_q);
    }
    m->tr_k = tk;
    m->tr_mode = tm;
    m->forced = fo;
    m->tr_theta = tt;
    m->tr_q = tq;
    m->trace_cap = cap;
    release_graphs(m);                   // pointers baked into the graphs changed
    return CWB_OK;
}

void release_graphs(cwb_model* m)
{
    m->graph_valid_for_batch = false;    // batches that captured this model capture it again
    if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
    if (m->graph1_exec) cudaGraphExecDestroy(m->graph1_exec);
    if (m->prof_exec) cudaGraphExecDestroy(m->prof_exec);
    if (m->prof_graph) cudaGraphDestroy(m->prof_graph);
    m->graph_exec = m->graph1_exec = m->prof_exec = nullptr;
    m->prof_graph = nullptr;
    m->prof_nodes.clear();
}

// Captures `iters` iterations into an executable graph (profiling mask: see enqueue_iteration).
static cwb_status capture_graph(cwb_model* m, int iters, int mask, cudaGraphExec_t* out)
{
    if (!m->capture_stream) CWB_CUDA_TRY(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
    if (mask && !m->prof_ph[0])
        for (auto& e : m->prof_ph) CWB_CUDA_TRY(cudaEventCreate(&e));
    cudaGraph_t graph = nullptr;
    CWB_CUDA_TRY(cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < iters; ++i) enqueue_iteration(m, m->capture_stream, mask);
    cudaError_t e = cudaStreamEndCapture(m->capture_stream, &graph);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    if (mask) {
        // find the event-record nodes of each profiled class
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
        cudaGraphNode_t found[8] = {};
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
            for (int i = 0; i < 8; ++i)
                if (ev == m->prof_ph[i]) found[i] = nd;
        }
        m->prof_nodes.clear();
        for (int c = 0; c < 4; ++c)
            if ((mask & (1 << c)) && found[2 * c] && found[2 * c + 1]) m->prof_nodes.push_back({c, {found[2 * c], found[2 * c + 1]}});
    }
    e = cudaGraphInstantiate(out, graph, 0);
    if (mask) {
        if (m->prof_graph) cudaGraphDestroy(m->prof_graph);
        m->prof_graph = graph;
    } else {
        cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
    return CWB_OK;
}

static cudaEvent_t take_event(cwb_model* m)
{
    if (!m->prof_pool.empty()) {
        cudaEvent_t e = m->prof_pool.back();
        m->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Trace capacity for `iters` more iterations and any pending forced selections on the device.
cwb_status prepare_launch(cwb_model* m, int32_t iters)
{
    CWB_TRY(ensure_trace(m, m->done + iters));
    if (!m->forced_host.empty()) {
        int32_t cnt = (int32_t)std::min<size_t>(m->forced_host.size(), (size_t)(m->trace_cap - m->done));
        CWB_CUDA_TRY(cudaMemcpyAsync(m->forced + m->done, m->forced_host.data(), sizeof(int32_t) * cnt,
                                     cudaMemcpyHostToDevice, m->stream));
        CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
        m->forced_host.clear();
    }
    return CWB_OK;
}

void note_iterations_queued(cwb_model* m, int32_t iters)
{
    m->done += iters;
    m->coef_valid_at = -1;
    m->update_pending = true;
}

cwb_status launch_iterations(cwb_model* m, int32_t iters)
{
    if (iters <= 0) return CWB_OK;
    CWB_TRY(prepare_launch(m, iters));
    if (m->persist_ok && m->iter_mode != kIterKernels) {
        CWB_TRY(launch_persistent(m, iters));
        note_iterations_queued(m, iters);
        return CWB_OK;
    }
    if (m->prof_on) {
        if (!m->prof_exec) CWB_TRY(capture_graph(m, 1, m->prof_mask, &m->prof_exec));
        for (int32_t i = 0; i < iters; ++i) {
            for (auto& pn : m->prof_nodes) {
                cudaEvent_t e0 = take_event(m), e1 = take_event(m);
                CWB_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(m->prof_exec, pn.second.first, e0));
                CWB_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(m->prof_exec, pn.second.second, e1));
                m->prof_pending.push_back({pn.first, {e0, e1}});
            }
            CWB_CUDA_TRY(cudaGraphLaunch(m->prof_exec, m->stream));
        }
    } else {
        int32_t left = iters;
        if (left >= kGraphIters) {
            if (!m->graph_exec) CWB_TRY(capture_graph(m, kGraphIters, 0, &m->graph_exec));
            while (left >= kGraphIters) {
                CWB_CUDA_TRY(cudaGraphLaunch(m->graph_exec, m->stream));
                left -= kGraphIters;
            }
        }
        if (left > 0 && !m->graph1_exec) CWB_TRY(capture_graph(m, 1, 0, &m->graph1_exec));
        for (int32_t i = 0; i < left; ++i) CWB_CUDA_TRY(cudaGraphLaunch(m->graph1_exec, m->stream));
    }
    CWB_CUDA_TRY(cudaGetLastError());
    note_iterations_queued(m, iters);
    return CWB_OK;
}

cwb_status launch_final_update(cwb_model* m)
{
    launch_rows<kRowsUpdate>(m, m->stream);
    CWB_CUDA_TRY(cudaGetLastError());
    return CWB_OK;
}

// Applies the last iteration's update to the fitted values (and, for HCWB, takes
// its validation risk) unless the next iteration's row pass has done so already.
cwb_status materialize(cwb_model* m)
{
    if (!m->update_pending) return CWB_OK;
    CWB_TRY(launch_final_update(m));
    m->update_pending = false;
    return CWB_OK;
}

cwb_status launch_initial_rows(cwb_model* m)
{
    if (m->hybrid) launch_rows<kRowsUpdate>(m, m->stream);
    CWB_CUDA_TRY(cudaGetLastError());
    return CWB_OK;
}

cwb_status launch_aggregate(cwb_model* m)
{
    CWB_TRY(materialize(m));           // the trace holds the last selected coefficients once applied
    if (m->coef_valid_at == m->done) return CWB_OK;
    const int threads = ((m->d_max + 31) / 32) * 32;
    k_aggregate<<<m->K, threads, 0, m->stream>>>(m->K, m->d_max, m->done, m->l_d, m->tr_k, m->tr_mode, m->tr_theta,
                                                 m->cfg.nu, m->cfg.gamma, m->coef);
    CWB_CUDA_TRY(cudaGetLastError());
    m->coef_valid_at = m->done;
    return CWB_OK;
}

cwb_status profile_collect(cwb_model* m)
{
    if (m->prof_pending.empty()) return CWB_OK;
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (auto& it : m->prof_pending) {
        float ms = 0.0f;
        CWB_CUDA_TRY(cudaEventElapsedTime(&ms, it.second.first, it.second.second));
        m->prof_ms[it.first] += ms;
        m->prof_launches[it.first] += 1;
        m->prof_pool.push_back(it.second.first);
        m->prof_pool.push_back(it.second.second);
    }
    m->prof_pending.clear();
    return CWB_OK;
}

void profile_release(cwb_model* m)
{
    for (auto& it : m->prof_pending) {
        cudaEventDestroy(it.second.first);
        cudaEventDestroy(it.second.second);
    }
    m->prof_pending.clear();
    for (cudaEvent_t e : m->prof_pool) cudaEventDestroy(e);
    m->prof_pool.clear();
}

// ---- row shards: one iteration split at its two exchange points (see cwb_shard_* in cwb.h)
cwb_status shard_rows(cwb_model* m, float* rmax, int device_ptrs)
{
    CWB_TRY(prepare_launch(m, 1));
    launch_rows<kRowsFused>(m, m->stream);
    CWB_CUDA_TRY(cudaGetLastError());
    CWB_CUDA_TRY(cudaMemcpyAsync(rmax, &m->state->rmax_bits[0], sizeof(float),
                                 device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
    if (!device_ptrs) CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return CWB_OK;
}

cwb_status shard_scatter(cwb_model* m, const float* rmax, int rmax_device, long long* u, int u_device)
{
    const ScatterPlan& P = m->plan;
    if (!P.int_acc) {
        set_error("row shards need the exact fixed-point histograms");
        return CWB_ESTATE;
    }
    CWB_CUDA_TRY(cudaMemcpyAsync(&m->state->rmax_bits[0], rmax, sizeof(float),
                                 rmax_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
    launch_scatter(m, m->stream);
    const int64_t total = (int64_t)m->B * m->nstar_max;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(4 * num_sms(m->device), (total + 255) / 256));
    k_partials_to_u<<<blocks, 256, 0, m->stream>>>(reinterpret_cast<const int*>(m->part), m->slot_c0, m->B, m->nstar_max,
                                                   P.fe, P.f_lane, P.nb_cta, P.bin_ranges, P.cmax, m->u_shard);
    CWB_CUDA_TRY(cudaGetLastError());
    if (u != m->u_shard)
        CWB_CUDA_TRY(cudaMemcpyAsync(u, m->u_shard, sizeof(long long) * total,
                                     u_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
    if (!u_device) CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return CWB_OK;
}

cwb_status shard_solve(cwb_model* m, const long long* u, int device_ptrs)
{
    const int64_t total = (int64_t)m->B * m->nstar_max;
    if (u != m->u_shard)
        CWB_CUDA_TRY(cudaMemcpyAsync(m->u_shard, u, sizeof(long long) * total,
                                     device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
    m->solve_u64 = m->u_shard;
    launch_solve(m, m->stream);
    m->solve_u64 = nullptr;
    CWB_CUDA_TRY(cudaGetLastError());
    note_iterations_queued(m, 1);
    return CWB_OK;
}

cwb_status read_device_error(cwb_model* m)
{
    DevState st;
    CWB_CUDA_TRY(cudaMemcpyAsync(&st, m->state, sizeof(DevState), cudaMemcpyDeviceToHost, m->stream));
    CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (st.err & kErrTimeout) {
        set_error("a device-side wait ran out");
        return CWB_ETIMEOUT;
    }
    if (st.err & kErrNonFinite) {
        set_error("non-finite base-learner criterion (diverging fit?)");
        return CWB_ENUMERIC;
    }
    if (st.err & kErrBound) {
        set_error("a pseudo residual exceeded the bound of its fixed-point scale");
        return CWB_ENUMERIC;
    }
    if (st.err) {
        set_error("internal device error flag " + std::to_string(st.err));
        return CWB_ECUDA;
    }
    return CWB_OK;
}

}  // namespace cwb
