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
//   k_solve    per learner: u -> s = Z^b^T u -> theta = P s (FP64) -> criterion
//              Q_k = theta^T G theta - 2 theta^T s = SSE_k - r^T W r (FP64);
//              the last CTA takes the argmin (ties: lowest k), writes the update
//              table v = Z^b theta of the winner and the trace.
#include <math.h>

#include <algorithm>
#include <string>

#include "cwb_internal.cuh"

namespace cwb {

namespace {

constexpr int kRowThreads = 256;
constexpr int kSolveThreads = 256;
constexpr int kScatterThreads = 512;
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
    const float* v;       // [2][S]
    const int32_t* l_bin;
    int S;
    int loss;
    double nu, gamma;
    int hybrid;
    int patience;
    double* risk_part;
};

template <typename IndT>
__device__ __forceinline__ void load_ind4(const IndT* p, int64_t i, int out[4]);

template <>
__device__ __forceinline__ void load_ind4<uint16_t>(const uint16_t* p, int64_t i, int out[4])
{
    uint2 u = *reinterpret_cast<const uint2*>(p + i);
    out[0] = u.x & 0xffff;
    out[1] = u.x >> 16;
    out[2] = u.y & 0xffff;
    out[3] = u.y >> 16;
}

template <>
__device__ __forceinline__ void load_ind4<uint8_t>(const uint8_t* p, int64_t i, int out[4])
{
    uint32_t u = *reinterpret_cast<const uint32_t*>(p + i);
    out[0] = u & 0xff;
    out[1] = (u >> 8) & 0xff;
    out[2] = (u >> 16) & 0xff;
    out[3] = u >> 24;
}

// ---- compensated ("double-float") arithmetic: a value is hi + lo, two FP32 numbers.
// The models f and h and the per-iteration coefficients (1 - theta_m, theta_m,
// nu, eta_m, m/(m+1)) are carried this way so that the only FP32 rounding left
// in a residual is its own final rounding.  Error-free transforms: TwoSum
// (Knuth) and the FMA product error.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ DF two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_mul_f(DF a, float b)
{
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_of(double x)
{
    float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// r = -dL/df at f = g (L2: y - g; binomial: y - sigmoid(g), first order in g.lo).
__device__ __forceinline__ float neg_gradient(int loss, float y, float ylo, DF g)
{
    if (loss == CWB_LOSS_L2) return ((y - g.hi) + ylo) - g.lo;
    float sg = 1.0f / (1.0f + expf(-g.hi));
    return (y - sg) - sg * (1.0f - sg) * g.lo;
}

__device__ __forceinline__ float loss_value(int loss, float y, float ylo, DF f)
{
    if (loss == CWB_LOSS_L2) {
        float e = ((y - f.hi) + ylo) - f.lo;
        return 0.5f * e * e;
    }
    float lse = f.hi > 0.0f ? f.hi + log1pf(expf(-f.hi)) : log1pf(expf(f.hi));
    float sg = 1.0f / (1.0f + expf(-f.hi));
    return (lse - y * f.hi) + (sg - y) * f.lo;
}

__device__ __forceinline__ float get4(const float4& v, int t)
{
    return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

__device__ __forceinline__ void set4(float4& v, int t, float x)
{
    if (t == 0) v.x = x; else if (t == 1) v.y = x; else if (t == 2) v.z = x; else v.w = x;
}

__device__ __forceinline__ void load_df4(const float* p, int64_t i4, DF out[4])
{
    float4 a = *reinterpret_cast<const float4*>(p + 2 * i4);
    float4 b = *reinterpret_cast<const float4*>(p + 2 * i4 + 4);
    out[0] = {a.x, a.y};
    out[1] = {a.z, a.w};
    out[2] = {b.x, b.y};
    out[3] = {b.z, b.w};
}

__device__ __forceinline__ void store_df4(float* p, int64_t i4, const DF v[4])
{
    *reinterpret_cast<float4*>(p + 2 * i4) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    *reinterpret_cast<float4*>(p + 2 * i4 + 4) = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
}

template <int KIND, typename IndT>
__global__ void __launch_bounds__(kRowThreads) k_rows(RowArgs a)
{
    const DevState st = *a.state;
    const bool pend = (KIND != kRowsResid) && (st.m > st.m_applied);
    const int pm = st.pend_mode;
    const IndT* ind = static_cast<const IndT*>(a.ind);
    const IndT* ind_sel = (st.k_sel >= 0) ? ind + (int64_t)a.l_bin[st.k_sel] * a.n_pad : nullptr;
    const IndT* ind_cor = (st.k_cor >= 0) ? ind + (int64_t)a.l_bin[st.k_cor] * a.n_pad : nullptr;
    const float* v0 = a.v;
    const float* v1 = a.v + a.S;
    const DF nu = df_of(a.nu);

    // pending update of iteration st.m (Algorithm 1 line "f = f + nu b"; Algorithm 3: f = g + nu b, h += eta b_cor)
    DF om_p = {1.0f, 0.0f}, th_p = {0.0f, 0.0f}, eta_p = {0.0f, 0.0f};
    if (pend && pm == kModeACWB) {
        const double thm = 2.0 / ((double)st.m + 1.0);
        om_p = df_of(1.0 - thm);
        th_p = df_of(thm);
        eta_p = df_of(a.gamma * a.nu / thm);
    }
    // residuals of iteration st.m + 1
    const int mode_n = st.mode;
    const int m_n = st.m + 1;
    const bool acwb_n = (mode_n == kModeACWB);
    const int64_t n_act = (acwb_n && a.hybrid) ? a.n_tr : a.n;
    const double thn_d = 2.0 / ((double)m_n + 1.0);
    const DF om_n = df_of(1.0 - thn_d), th_n = df_of(thn_d);
    const DF cmul = df_of((double)m_n / ((double)m_n + 1.0));
    const bool first_acwb = (m_n == 1);
    const bool need_bc = pend && pm == kModeACWB;
    const bool need_bc_resid = (KIND != kRowsUpdate) && acwb_n && !first_acwb;
    const bool eval_risk = (KIND == kRowsUpdate) && a.hybrid && (!st.risk_valid || (pend && pm == kModeACWB));

    double risk_acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t i4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i4 < a.n_pad; i4 += stride) {
        DF fv[4], hv[4];
        load_df4(a.f, i4, fv);
        if (a.h) load_df4(a.h, i4, hv);
        else for (int t = 0; t < 4; ++t) hv[t] = {0.0f, 0.0f};
        float bc[4] = {0.f, 0.f, 0.f, 0.f};
        if ((need_bc || need_bc_resid) && ind_cor) {
            int kc[4];
            load_ind4<IndT>(ind_cor, i4, kc);
#pragma unroll
            for (int t = 0; t < 4; ++t) bc[t] = __ldg(v1 + kc[t]);
        }
        if (pend && ind_sel) {
            int ks[4];
            load_ind4<IndT>(ind_sel, i4, ks);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float b0 = __ldg(v0 + ks[t]);
                if (pm == kModeCWB) {
                    fv[t] = df_add(fv[t], df_mul_f(nu, b0));
                } else {
                    DF g = df_add(df_mul(fv[t], om_p), df_mul(hv[t], th_p));
                    fv[t] = df_add(g, df_mul_f(nu, b0));
                    hv[t] = df_add(hv[t], df_mul_f(eta_p, bc[t]));
                }
            }
            store_df4(a.f, i4, fv);
            if (pm == kModeACWB && a.h) store_df4(a.h, i4, hv);
        }
        if (eval_risk) {
            if (i4 + 4 > a.n_tr && i4 < a.n) {
                float4 y4 = *reinterpret_cast<const float4*>(a.y + i4);
                float4 yl4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (a.y_lo) yl4 = *reinterpret_cast<const float4*>(a.y_lo + i4);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    int64_t i = i4 + t;
                    if (i >= a.n_tr && i < a.n)
                        risk_acc += (double)loss_value(a.loss, get4(y4, t), get4(yl4, t), fv[t]);
                }
            }
        }
        if (KIND != kRowsUpdate) {
            float4 y4 = *reinterpret_cast<const float4*>(a.y + i4);
            float4 yl4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.y_lo) yl4 = *reinterpret_cast<const float4*>(a.y_lo + i4);
            float4 w4 = make_float4(1.f, 1.f, 1.f, 1.f);
            if (a.w) w4 = *reinterpret_cast<const float4*>(a.w + i4);
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
            float4 c4 = r0;
            if (acwb_n) c4 = *reinterpret_cast<const float4*>(a.c + i4);
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
            *reinterpret_cast<float4*>(a.rw + i4) = r0;
            if (acwb_n) {
                *reinterpret_cast<float4*>(a.rw + a.n_pad + i4) = r1;
                *reinterpret_cast<float4*>(a.c + i4) = c4;
            }
        }
    }

    // block partial of the validation risk, then the last block finishes the iteration bookkeeping
    __shared__ double red[kRowThreads];
    __shared__ bool is_last;
    red[threadIdx.x] = risk_acc;
    __syncthreads();
    for (int s = kRowThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (a.risk_part) a.risk_part[blockIdx.x] = red[0];
        __threadfence();
        unsigned t = atomicAdd(&a.state->ticket_rows, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        DevState* S = a.state;
        if (eval_risk) {
            double sum = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) sum += __ldcg(a.risk_part + b);
            double risk = sum / (double)(a.n - a.n_tr);
            if (!S->risk_valid) {
                S->risk_prev = risk;
                S->risk_valid = 1;
            } else {
                S->counter = (risk > S->risk_prev) ? S->counter + 1 : 0;
                S->risk_prev = risk;
            }
        }
        if (KIND == kRowsUpdate && a.hybrid && S->mode == kModeACWB && S->counter >= a.patience) {
            S->mode = kModeCWB;
            S->phase = 1;
            S->switch_iter = S->m + 1;
        }
        if (pend) S->m_applied = st.m;
        S->ticket_rows = 0;
    }
}

// ---------------------------------------------------------------------------
// binMatVec scatter (Algorithm 2).  A CTA owns f_lane binnings x one row chunk
// (x one bin range).  Lane l of a warp works on binning (l % f_lane), channel
// and row set (l / f_lane); its histogram column lives at hist[ch][bin][lane's
// binning], so lanes of one warp never share an address and, for f_lane = 32
// (or 16 with two channels), never share a bank.

struct ScatterArgs {
    const DevState* state;
    const void* ind;
    int64_t n, n_tr, n_pad;
    const float* rw;
    int B, f_lane, groups, chunks, nb_cta, nbins_pad, ch_stride, hybrid;
    float* part;
};

template <typename IndT>
__device__ __forceinline__ void load_ind16(const IndT* p, int64_t i, int out[16]);

template <>
__device__ __forceinline__ void load_ind16<uint16_t>(const uint16_t* p, int64_t i, int out[16])
{
    const uint4* q = reinterpret_cast<const uint4*>(p + i);
    uint4 a = __ldcs(q), b = __ldcs(q + 1);
    uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        out[2 * t] = w[t] & 0xffff;
        out[2 * t + 1] = w[t] >> 16;
    }
}

template <>
__device__ __forceinline__ void load_ind16<uint8_t>(const uint8_t* p, int64_t i, int out[16])
{
    uint4 a = __ldcs(reinterpret_cast<const uint4*>(p + i));
    uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        out[4 * t] = w[t] & 0xff;
        out[4 * t + 1] = (w[t] >> 8) & 0xff;
        out[4 * t + 2] = (w[t] >> 16) & 0xff;
        out[4 * t + 3] = w[t] >> 24;
    }
}

template <typename IndT, int CMAX>
__global__ void __launch_bounds__(kScatterThreads) k_scatter(ScatterArgs a)
{
    extern __shared__ float hist[];
    const int mode = a.state->mode;
    const int C = (CMAX == 2 && mode == kModeACWB) ? 2 : 1;
    const int64_t n_act = (mode == kModeACWB && a.hybrid) ? a.n_tr : a.n;
    const int64_t n16 = (n_act + 15) & ~(int64_t)15;
    const int F = a.f_lane;
    const int chunk = blockIdx.x, g = blockIdx.y, br = blockIdx.z;
    const int b_lo = br * a.nb_cta;
    const int nb = min(a.nb_cta, a.nbins_pad - b_lo);

    for (int i = threadIdx.x; i < CMAX * a.ch_stride; i += blockDim.x) hist[i] = 0.0f;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int f = lane % F, q = lane / F;
    const int ch = q % C, rs = q / C;
    const int RS = 32 / (F * C);
    const int bidx = g * F + f;
    const bool active = bidx < a.B;
    const IndT* row = static_cast<const IndT*>(a.ind) + (int64_t)(active ? bidx : 0) * a.n_pad;
    const float* r = a.rw + (int64_t)ch * a.n_pad;
    float* hc = hist + ch * a.ch_stride;

    const int64_t csize = (((n16 + a.chunks - 1) / a.chunks) + 15) & ~(int64_t)15;
    const int64_t lo = (int64_t)chunk * csize;
    const int64_t hi = min(lo + csize, n16);
    for (int64_t row0 = lo + (int64_t)warp * 16 * RS; row0 < hi; row0 += (int64_t)nwarps * 16 * RS) {
        const int64_t i = row0 + 16 * rs;
        if (active && i < hi) {
            int idx[16];
            load_ind16<IndT>(row, i, idx);
            const float4* r4p = reinterpret_cast<const float4*>(r + i);
            float4 r4[4] = {__ldg(r4p), __ldg(r4p + 1), __ldg(r4p + 2), __ldg(r4p + 3)};
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                unsigned bl = (unsigned)(idx[t] - b_lo);
                if (bl < (unsigned)nb) atomicAdd(&hc[bl * F + f], get4(r4[t >> 2], t & 3));
            }
        }
    }
    __syncthreads();
    for (int c2 = 0; c2 < C; ++c2) {
        float* dst = a.part + ((((int64_t)chunk * a.groups + g) * CMAX + c2) * a.nbins_pad + b_lo) * F;
        const float* src = hist + c2 * a.ch_stride;
        for (int i = threadIdx.x; i < nb * F; i += blockDim.x) dst[i] = src[i];
    }
}

// ---------------------------------------------------------------------------
// Per-learner fit, criterion and argmin.

struct SolveArgs {
    DevState* state;
    int K, D, S;
    int f_lane, groups, chunks, nbins_pad, cmax;
    const float* part;
    float* u;                 // [2][K][S] scratch
    const float* zb;
    const int32_t* zcol;
    const int32_t* crange;
    const int32_t* l_bin;
    const int32_t* l_d;
    const int32_t* l_nstar;
    const double* G;          // [2][K][D][D]
    const double* P;
    double* theta_it;         // [2][K][D]
    double* q_it;             // [2][K]
    float* v;                 // [2][S]
    int32_t* tr_k;            // [cap][2]
    int32_t* tr_mode;         // [cap]
    double* tr_theta;         // [cap][2][D]
    double* tr_q;             // [cap][2]
    const int32_t* forced;    // [cap]
    int trace_cap;
};

__global__ void __launch_bounds__(kSolveThreads) k_solve(SolveArgs a)
{
    const int k = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevState st = *a.state;
    const int mode = st.mode;
    const int C = (mode == kModeACWB) ? 2 : 1;
    const int ph = (mode == kModeACWB) ? 0 : st.phase;
    const int b = a.l_bin[k], d = a.l_d[k], nst = a.l_nstar[k];
    const int F = a.f_lane;
    const int g = b / F, f = b % F;
    __shared__ double s_s[kMaxD], th_s[kMaxD], term[kMaxD];
    __shared__ bool is_last;
    const int64_t chunk_stride = (int64_t)a.groups * a.cmax * a.nbins_pad * F;
    const double* Pk = a.P + ((int64_t)ph * a.K + k) * a.D * a.D;
    const double* Gk = a.G + ((int64_t)ph * a.K + k) * a.D * a.D;

    for (int ch = 0; ch < C; ++ch) {
        float* u = a.u + ((int64_t)ch * a.K + k) * a.S;
        // 1. u_l: compensated sum of the per-chunk partial histograms
        const float* p0 = a.part + ((int64_t)g * a.cmax + ch) * a.nbins_pad * F + f;
        for (int l = tid; l < nst; l += blockDim.x) {
            float s = 0.0f, comp = 0.0f;
            const float* p = p0 + (int64_t)l * F;
            for (int c = 0; c < a.chunks; ++c) {
                float y = __ldcg(p + c * chunk_stride) - comp;
                float t = s + y;
                comp = (t - s) - y;
                s = t;
            }
            u[l] = s;
        }
        __syncthreads();
        // 2. s = Z^b^T u over each column's contiguous bin range (warp tree sums)
        for (int j = warp; j < d; j += blockDim.x / 32) {
            const int lo = a.crange[((int64_t)k * a.D + j) * 2], hi = a.crange[((int64_t)k * a.D + j) * 2 + 1];
            float acc = 0.0f;
            for (int l = lo + lane; l < hi; l += 32) {
                int c0 = a.zcol[(int64_t)k * a.S + l];
                acc += a.zb[((int64_t)k * a.S + l) * kMaxNnz + (j - c0)] * u[l];
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) s_s[j] = (double)acc;
        }
        __syncthreads();
        // 3. theta = P s (FP64)
        if (tid < d) {
            double t = 0.0;
            for (int i = 0; i < d; ++i) t += Pk[tid * a.D + i] * s_s[i];
            th_s[tid] = t;
        }
        __syncthreads();
        // 4. Q = theta^T G theta - 2 theta^T s (FP64)
        if (tid < d) {
            double gt = 0.0;
            for (int i = 0; i < d; ++i) gt += Gk[tid * a.D + i] * th_s[i];
            term[tid] = th_s[tid] * (gt - 2.0 * s_s[tid]);
        }
        __syncthreads();
        if (tid < a.D) a.theta_it[((int64_t)ch * a.K + k) * a.D + tid] = tid < d ? th_s[tid] : 0.0;
        if (tid == 0) {
            double q = 0.0;
            for (int j = 0; j < d; ++j) q += term[j];
            a.q_it[(int64_t)ch * a.K + k] = q;
        }
        __syncthreads();
    }

    if (tid == 0) {
        __threadfence();
        unsigned t = atomicAdd(&a.state->ticket_solve, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // ---- last CTA: argmin per channel, update tables, trace, state
    __shared__ double cand_q[2 * kSolveThreads];
    __shared__ int cand_k[2 * kSolveThreads];
    __shared__ int best_k[2];
    __shared__ float th32[kMaxD];
    __shared__ uint32_t bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    const int it = st.m;
    const bool trace_ok = it < a.trace_cap;
    for (int ch = 0; ch < C; ++ch) {
        double q1 = INFINITY, q2 = INFINITY;
        int k1 = -1, k2 = -1;
        for (int kk = tid; kk < a.K; kk += blockDim.x) {
            double q = __ldcg(a.q_it + (int64_t)ch * a.K + kk);
            if (!(q == q) || isinf(q)) {
                atomicOr(&bad, 1u);
                q = INFINITY;
            }
            if (q < q1) { q2 = q1; k2 = k1; q1 = q; k1 = kk; }
            else if (q < q2) { q2 = q; k2 = kk; }
        }
        cand_q[2 * tid] = q1; cand_k[2 * tid] = k1;
        cand_q[2 * tid + 1] = q2; cand_k[2 * tid + 1] = k2;
        __syncthreads();
        if (tid == 0) {
            double b1 = INFINITY, b2 = INFINITY;
            int i1 = -1;
            for (int c = 0; c < 2 * (int)blockDim.x; ++c) {
                double q = cand_q[c];
                int kk = cand_k[c];
                if (kk < 0) continue;
                if (i1 < 0 || q < b1 || (q == b1 && kk < i1)) {
                    if (i1 >= 0) b2 = fmin(b2, b1);
                    b1 = q;
                    i1 = kk;
                } else {
                    b2 = fmin(b2, q);
                }
            }
            if (i1 < 0) i1 = 0;
            if (ch == 0 && trace_ok && a.forced) {
                int fk = a.forced[it];
                if (fk >= 0 && fk < a.K) i1 = fk;
            }
            best_k[ch] = i1;
            if (trace_ok) {
                a.tr_k[2 * it + ch] = i1;
                if (ch == 0) {
                    a.tr_q[2 * it] = b1;
                    a.tr_q[2 * it + 1] = b2;
                }
            }
        }
        __syncthreads();
        const int kb = best_k[ch];
        if (tid < a.D) {
            double tv = __ldcg(a.theta_it + ((int64_t)ch * a.K + kb) * a.D + tid);
            th32[tid] = (float)tv;
            if (trace_ok) a.tr_theta[((int64_t)2 * it + ch) * a.D + tid] = tv;
        }
        __syncthreads();
        const int nstb = a.l_nstar[kb];
        for (int l = tid; l < nstb; l += blockDim.x) {
            const int c0 = a.zcol[(int64_t)kb * a.S + l];
            const float* z = a.zb + ((int64_t)kb * a.S + l) * kMaxNnz;
            float acc = 0.0f;
#pragma unroll
            for (int t = 0; t < kMaxNnz; ++t)
                if (c0 + t < a.D) acc += z[t] * th32[c0 + t];
            a.v[(int64_t)ch * a.S + l] = acc;
        }
        __syncthreads();
    }
    if (tid == 0) {
        DevState* S = a.state;
        if (trace_ok) {
            a.tr_mode[it] = mode;
            if (C == 1) a.tr_k[2 * it + 1] = -1;
        } else {
            atomicOr(&S->err, kErrIndex);
        }
        if (bad) atomicOr(&S->err, kErrNonFinite);
        S->k_sel = best_k[0];
        S->k_cor = (C == 2) ? best_k[1] : -1;
        S->pend_mode = mode;
        S->m = st.m + 1;
        S->ticket_solve = 0;
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
    int64_t g = (m->n_pad / 4 + kRowThreads - 1) / kRowThreads;
    int64_t cap = (int64_t)num_sms(m->device) * 8;
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
    a.loss = m->cfg.loss;
    a.nu = m->cfg.nu;
    a.gamma = m->cfg.gamma;
    a.hybrid = m->hybrid ? 1 : 0;
    a.patience = m->cfg.patience;
    a.risk_part = m->risk_part;
    return a;
}

template <int KIND>
void launch_rows(cwb_model* m, cudaStream_t s)
{
    RowArgs a = row_args(m);
    const int g = rows_grid(m);
    if (m->ind_bytes == 1) k_rows<KIND, uint8_t><<<g, kRowThreads, 0, s>>>(a);
    else k_rows<KIND, uint16_t><<<g, kRowThreads, 0, s>>>(a);
}

void launch_scatter(cwb_model* m, cudaStream_t s)
{
    const ScatterPlan& P = m->plan;
    ScatterArgs a{m->state, m->ind, m->n, m->n_tr, m->n_pad, m->rw, m->B, P.f_lane, P.groups, P.chunks,
                  P.nb_cta, P.nbins_pad, P.ch_stride, m->hybrid ? 1 : 0, m->part};
    dim3 grid(P.chunks, P.groups, P.bin_ranges);
    const bool two = m->accel;
    if (m->ind_bytes == 1) {
        if (two) k_scatter<uint8_t, 2><<<grid, P.threads, P.smem, s>>>(a);
        else k_scatter<uint8_t, 1><<<grid, P.threads, P.smem, s>>>(a);
    } else {
        if (two) k_scatter<uint16_t, 2><<<grid, P.threads, P.smem, s>>>(a);
        else k_scatter<uint16_t, 1><<<grid, P.threads, P.smem, s>>>(a);
    }
}

void launch_solve(cwb_model* m, cudaStream_t s)
{
    const ScatterPlan& P = m->plan;
    SolveArgs a;
    a.state = m->state;
    a.K = m->K;
    a.D = m->d_max;
    a.S = m->nstar_max;
    a.f_lane = P.f_lane;
    a.groups = P.groups;
    a.chunks = P.chunks;
    a.nbins_pad = P.nbins_pad;
    a.cmax = m->accel ? 2 : 1;
    a.part = m->part;
    a.u = m->v + 2 * (int64_t)m->nstar_max;    // scratch lives after the two update tables
    a.zb = m->zb;
    a.zcol = m->zcol;
    a.crange = m->crange;
    a.l_bin = m->l_bin;
    a.l_d = m->l_d;
    a.l_nstar = m->l_nstar;
    a.G = m->G;
    a.P = m->P;
    a.theta_it = m->theta_it;
    a.q_it = m->q_it;
    a.v = m->v;
    a.tr_k = m->tr_k;
    a.tr_mode = m->tr_mode;
    a.tr_theta = m->tr_theta;
    a.tr_q = m->tr_q;
    a.forced = m->forced;
    a.trace_cap = m->trace_cap;
    k_solve<<<m->K, kSolveThreads, 0, s>>>(a);
}

// Event pair around one launch when profiling (never while capturing a graph).
struct ProfScope {
    cwb_model* m;
    cudaStream_t s;
    int cls;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    static cudaEvent_t take(cwb_model* m)
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
    ProfScope(cwb_model* mm, cudaStream_t ss, int c) : m(mm), s(ss), cls(c)
    {
        if (m->prof_on && s == m->stream) {
            e0 = take(m);
            e1 = take(m);
            if (e0) cudaEventRecord(e0, s);
        }
    }
    ~ProfScope()
    {
        if (e0 && e1) {
            cudaEventRecord(e1, s);
            m->prof_pending.push_back({cls, {e0, e1}});
        }
    }
};

void enqueue_iteration(cwb_model* m, cudaStream_t s)
{
    {
        ProfScope p(m, s, 0);
        if (m->hybrid) {
            launch_rows<kRowsUpdate>(m, s);
            launch_rows<kRowsResid>(m, s);
        } else {
            launch_rows<kRowsFused>(m, s);
        }
    }
    {
        ProfScope p(m, s, 1);
        launch_scatter(m, s);
    }
    {
        ProfScope p(m, s, 2);
        launch_solve(m, s);
    }
}

cwb_status set_scatter_attrs(cwb_model* m)
{
    const int smem = (int)m->plan.smem;
    if (m->ind_bytes == 1) {
        CWB_CUDA_TRY(cudaFuncSetAttribute(k_scatter<uint8_t, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        CWB_CUDA_TRY(cudaFuncSetAttribute(k_scatter<uint8_t, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    } else {
        CWB_CUDA_TRY(cudaFuncSetAttribute(k_scatter<uint16_t, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        CWB_CUDA_TRY(cudaFuncSetAttribute(k_scatter<uint16_t, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    }
    return CWB_OK;
}

}  // namespace

cwb_status plan_scatter(cwb_model* m)
{
    int optin = 0, per_sm = 0;
    CWB_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    CWB_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device));
    const int budget = std::min(optin, 200 * 1024);
    const int cmax = m->accel ? 2 : 1;
    const int nbins = m->nstar_max;
    const int B = m->B;
    int pow2B = 1;
    while (pow2B < B) pow2B <<= 1;
    ScatterPlan P{};
    P.bin_ranges = 1;
    P.f_lane = 0;
    for (int F = 32; F >= 1; F >>= 1) {
        if (F * cmax > 32 || F > pow2B) continue;
        int64_t bytes = (int64_t)cmax * ((int64_t)nbins * F + 32) * 4;
        if (bytes <= budget) {
            P.f_lane = F;
            break;
        }
    }
    if (P.f_lane == 0) {
        P.f_lane = 1;
        int64_t need = (int64_t)cmax * ((int64_t)nbins + 32) * 4;
        P.bin_ranges = (int)((need + budget - 1) / budget);
    }
    P.nb_cta = (nbins + P.bin_ranges - 1) / P.bin_ranges;
    P.nbins_pad = P.nb_cta * P.bin_ranges;
    int base = P.nb_cta * P.f_lane;
    int pad = (cmax == 2) ? ((16 - base % 32) + 32) % 32 : 0;
    P.ch_stride = base + pad;
    P.smem = (size_t)cmax * P.ch_stride * sizeof(float);
    P.groups = (B + P.f_lane - 1) / P.f_lane;
    P.threads = kScatterThreads;
    int by_smem = (int)(per_sm / (P.smem + 1024));
    int ctas_per_sm = std::max(1, std::min(by_smem, 2048 / P.threads));
    int target = num_sms(m->device) * ctas_per_sm;
    int chunks = std::max(1, target / (P.groups * P.bin_ranges));
    int64_t max_chunks = std::max<int64_t>(1, m->n_pad / 256);
    P.chunks = (int)std::min<int64_t>(chunks, max_chunks);
    P.part_floats = (size_t)P.chunks * P.groups * cmax * P.nbins_pad * P.f_lane;
    m->plan = P;
    return set_scatter_attrs(m);
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
    if (m->graph_exec) {                 // pointers baked into the graph changed
        cudaGraphExecDestroy(m->graph_exec);
        m->graph_exec = nullptr;
    }
    return CWB_OK;
}

static cwb_status build_graph(cwb_model* m)
{
    if (!m->capture_stream) CWB_CUDA_TRY(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    CWB_CUDA_TRY(cudaStreamBeginCapture(m->capture_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kGraphIters; ++i) enqueue_iteration(m, m->capture_stream);
    cudaError_t e = cudaStreamEndCapture(m->capture_stream, &graph);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&m->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
    m->graph_iters = kGraphIters;
    return CWB_OK;
}

cwb_status launch_iterations(cwb_model* m, int32_t iters)
{
    if (iters <= 0) return CWB_OK;
    CWB_TRY(ensure_trace(m, m->done + iters));
    if (!m->forced_host.empty()) {
        int32_t cnt = (int32_t)std::min<size_t>(m->forced_host.size(), (size_t)(m->trace_cap - m->done));
        CWB_CUDA_TRY(cudaMemcpyAsync(m->forced + m->done, m->forced_host.data(), sizeof(int32_t) * cnt,
                                     cudaMemcpyHostToDevice, m->stream));
        CWB_CUDA_TRY(cudaStreamSynchronize(m->stream));
        m->forced_host.clear();
    }
    int32_t left = iters;
    if (left >= kGraphIters && !m->prof_on) {
        if (!m->graph_exec) CWB_TRY(build_graph(m));
        while (left >= kGraphIters) {
            CWB_CUDA_TRY(cudaGraphLaunch(m->graph_exec, m->stream));
            left -= kGraphIters;
        }
    }
    for (int32_t i = 0; i < left; ++i) enqueue_iteration(m, m->stream);
    CWB_CUDA_TRY(cudaGetLastError());
    m->done += iters;
    m->coef_valid_at = -1;
    return CWB_OK;
}

cwb_status launch_final_update(cwb_model* m)
{
    ProfScope p(m, m->stream, 0);
    launch_rows<kRowsUpdate>(m, m->stream);
    CWB_CUDA_TRY(cudaGetLastError());
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
    if (st.err) {
        set_error("internal device error flag " + std::to_string(st.err));
        return CWB_ECUDA;
    }
    return CWB_OK;
}

}  // namespace cwb
