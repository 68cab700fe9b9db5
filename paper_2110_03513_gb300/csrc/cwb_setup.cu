// cwb_setup.cu -- one-time model setup on the device (FP64 where the paper's
// algebra needs it): binning (Sec. 3.1.1), reduced designs at the design
// points (Sec. 2.2), weighted bin counts and Z^T W Z (binMatMat, Algorithm 2),
// lambda from df via the Demmler-Reinsch orthogonalisation (App. A.2) and the
// cached inverse (Z^T W Z + lambda K)^-1 (Sec. 2.4, Sec. 3.1.2).
#include <math.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "cwb_internal.cuh"
#include "cwb_bspline.cuh"

namespace cwb {

namespace {

constexpr int kThreads = 256;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

// ---------------------------------------------------------------------------
// Gathers and conversions (rows permuted train-first: new row q holds original row perm[q]).

template <typename T>
__global__ void k_gather_to_f32(const T* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                                int64_t n_pad, float* __restrict__ dst)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pad; q += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (q < n) v = (float)src[perm ? perm[q] : q];
        dst[q] = v;
    }
}

template <typename T>
__global__ void k_gather_f64(const T* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                             double* __restrict__ dst)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = (double)src[perm ? perm[q] : q];
}

// FP64 values as hi + lo FP32 pairs (lo omitted when NULL); zero past n.
__global__ void k_split_f64(const double* __restrict__ src, int64_t n, int64_t n_pad, float* __restrict__ hi,
                            float* __restrict__ lo)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pad; q += (int64_t)gridDim.x * blockDim.x) {
        double v = q < n ? src[q] : 0.0;
        float h = (float)v;
        hi[q] = h;
        if (lo) lo[q] = (float)(v - (double)h);
    }
}

// FP64 values from FP32 high parts and optional low parts (the split of FP64 targets).
__global__ void k_join_f64(const float* __restrict__ hi, const float* __restrict__ lo, int64_t n, double* __restrict__ out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (double)hi[q] + (lo ? (double)lo[q] : 0.0);
}

template <typename T>
__global__ void k_check_binary(const T* __restrict__ y, int64_t n, uint32_t* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = y[i];
        if (!(v == (T)0 || v == (T)1)) atomicOr(bad, 1u);
    }
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ v, int64_t n, uint32_t* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite((double)v[i])) atomicOr(bad, 1u);
}

template <typename T>
__global__ void k_check_weights(const T* __restrict__ w, int64_t n, uint32_t* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = w[i];
        if (!(v > (T)0) || !isfinite((double)v)) atomicOr(bad, 1u);
    }
}

// Categorical feature: every value must be an integer class code in [0, c).
template <typename T>
__global__ void k_check_codes(const T* __restrict__ X, int64_t feat, int64_t n, int c, uint32_t* bad)
{
    const T* x = X + feat * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        if (!(v >= 0.0 && v < (double)c && v == floor(v))) atomicOr(bad, 1u);
    }
}

// ---------------------------------------------------------------------------
// Feature range: per binning min and max over all rows (FP64 compare).

template <typename T>
__global__ void k_minmax_partial(const T* __restrict__ X, const int32_t* __restrict__ feat, int64_t n,
                                 double* __restrict__ pmin, double* __restrict__ pmax, uint32_t* nonfinite)
{
    const int b = blockIdx.y;
    const T* x = X + (int64_t)feat[b] * n;
    // compared in the input type (exact; FP64 arithmetic is slow on this part)
    T lo = T(INFINITY), hi = T(-INFINITY);
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = x[i];
        if (!isfinite(v)) { bad = true; continue; }
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    if (bad) atomicOr(nonfinite, 1u);
    __shared__ double slo[kThreads], shi[kThreads];
    slo[threadIdx.x] = (double)lo;
    shi[threadIdx.x] = (double)hi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pmin[(int64_t)b * gridDim.x + blockIdx.x] = slo[0];
        pmax[(int64_t)b * gridDim.x + blockIdx.x] = shi[0];
    }
}

__global__ void k_minmax_final(const double* __restrict__ pmin, const double* __restrict__ pmax, int nblk,
                               double* __restrict__ xmin, double* __restrict__ xmax)
{
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        double lo = INFINITY, hi = -INFINITY;
        for (int i = 0; i < nblk; ++i) {
            lo = fmin(lo, pmin[(int64_t)b * nblk + i]);
            hi = fmax(hi, pmax[(int64_t)b * nblk + i]);
        }
        xmin[b] = lo;
        xmax[b] = hi;
    }
}

// ---------------------------------------------------------------------------
// Index vectors (Sec. 3.1.1).

// Equidistant design points z_l = xmin + l h: closest point, half-way values to the
// lower one, i.e. l = ceil((x - xmin)/h - 1/2) clamped to [0, n*-1], defined on correctly
// rounded FP64 operations so that the index is reproducible bit for bit.  The FP64
// division is slow on this GPU, so the quotient is first formed in FP32: its relative
// error is below 3 x 2^-24 (the rounding of x - xmin, of 1/h and of the product), so
// when no integer lies within 4e-7 |t| + 1e-6 of t - 1/2 (the interval is evaluated in
// FP32, whose own roundings the margin also covers) the FP32 and FP64 rules agree;
// only values that close to a half-way point take the FP64 path.
// One equidistant binning of the fit: its feature, range and design-point count.
struct BinJob {
    int64_t feature;
    double xmin, h;
    int32_t nstar, binning;
};

// Every equidistant binning of a fit in one launch (blockIdx.y = job).
template <typename T, typename IndT>
__global__ void k_bin_equidistant(const T* __restrict__ X, const BinJob* __restrict__ jobs,
                                  const int32_t* __restrict__ perm, int64_t n, int64_t n_pad, IndT* __restrict__ ind)
{
    const BinJob jb = jobs[blockIdx.y];
    const T* x = X + jb.feature * n;
    const double xmin = jb.xmin, h = jb.h;
    const int nstar = jb.nstar;
    IndT* out = ind + (int64_t)jb.binning * n_pad;
    const float inv_h = (float)(1.0 / h);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pad; q += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        if (q < n) {
            const T xv = x[perm ? perm[q] : q];
            double dv = 0.0;
            float d32;
            if (sizeof(T) == 4) {
                // x and xmin are FP32 values here (xmin is the feature's minimum, or 0 for class
                // codes): the FP32 difference is the exact difference rounded once
                d32 = (float)xv - (float)xmin;
            } else {
                dv = __dsub_rn((double)xv, xmin);
                d32 = (float)dv;
            }
            const float t32 = d32 * inv_h;
            const float e = 4.0e-7f * fabsf(t32) + 1.0e-6f;
            const float c_lo = ceilf(t32 - 0.5f - e), c_hi = ceilf(t32 - 0.5f + e);
            if (c_lo == c_hi && isfinite(t32)) {
                // the common case stays on the FP32 pipe (c_lo holds an integer; n* - 1 < 2^24 is exact)
                l = (int)fminf(fmaxf(c_lo, 0.0f), (float)(nstar - 1));
            } else {
                if (sizeof(T) == 4) dv = __dsub_rn((double)xv, xmin);
                double c = ceil(__dsub_rn(__ddiv_rn(dv, h), 0.5));
                c = fmax(c, 0.0);
                c = fmin(c, (double)(nstar - 1));
                l = (int)c;
            }
        }
        out[q] = (IndT)l;
    }
}

// Exact binning: the design points are the sorted unique values.
template <typename T>
__global__ void k_load_sort_keys(const T* __restrict__ X, int64_t feat, int64_t n, int64_t npow2,
                                 double* __restrict__ keys)
{
    const T* x = X + feat * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npow2; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = i < n ? (double)x[i] : INFINITY;
}

// One compare-exchange pass of a bitonic sorting network (ascending).
__global__ void k_bitonic_pass(double* __restrict__ a, int64_t npow2, int64_t j, int64_t k)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npow2; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = i ^ j;
        if (l > i) {
            double ai = a[i], al = a[l];
            bool up = (i & k) == 0;
            if ((up && ai > al) || (!up && ai < al)) {
                a[i] = al;
                a[l] = ai;
            }
        }
    }
}

// Single-block scan of "first of its value" flags: writes the unique values in order.
__global__ void k_unique_single_block(const double* __restrict__ s, int64_t n, double* __restrict__ z,
                                      int32_t* __restrict__ count)
{
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int flag = 0;
        double v = 0.0;
        if (i < n) {
            v = s[i];
            flag = (i == 0 || s[i - 1] != v) ? 1 : 0;
        }
        int incl = flag;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int ws = lane < nw ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += t;
            }
            if (lane < nw) warp_sums[lane] = ws;
        }
        __syncthreads();
        int before = (wid > 0 ? warp_sums[wid - 1] : 0) + incl - flag;
        if (flag) z[carry + before] = v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + flag;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

template <typename T, typename IndT>
__global__ void k_bin_exact(const T* __restrict__ X, int64_t feat, const int32_t* __restrict__ perm, int64_t n,
                            int64_t n_pad, const double* __restrict__ z, int nstar, IndT* __restrict__ out,
                            uint32_t* err)
{
    const T* x = X + feat * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_pad; q += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        if (q < n) {
            double v = (double)x[perm ? perm[q] : q];
            int lo = 0, hi = nstar - 1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (z[mid] < v) lo = mid + 1; else hi = mid;
            }
            if (z[lo] != v) atomicOr(err, kErrIndex);
            l = lo;
        }
        out[q] = (IndT)l;
    }
}

// ---------------------------------------------------------------------------
// Weighted bin counts cnt[b][l] = sum over rows [r0, r1) with ind = l of w (binMatMat input).

// Unweighted counts: a CTA counts its rows in a shared-memory histogram (int32) and adds the
// non-zero bins to the FP64 totals; integer-valued sums, so the result is exact and does not
// depend on the order of the additions.  nstar <= kCountSmemBins (48 KB, no opt-in needed).
constexpr int kCountSmemBins = 12288;

template <typename IndT>
__global__ void k_counts_smem(const IndT* __restrict__ ind, int64_t n_pad, int64_t r1, int nstar, int stride,
                              double* __restrict__ cnt)
{
    extern __shared__ int hc[];
    const int b = blockIdx.y;
    const IndT* row = ind + (int64_t)b * n_pad;
    for (int l = threadIdx.x; l < nstar; l += blockDim.x) hc[l] = 0;
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < r1; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hc[row[q]], 1);
    __syncthreads();
    double* c = cnt + (int64_t)b * stride;
    for (int l = threadIdx.x; l < nstar; l += blockDim.x)
        if (hc[l]) atomicAdd(&c[l], (double)hc[l]);
}

template <typename IndT>
__global__ void k_counts(const IndT* __restrict__ ind, int64_t n_pad, int64_t r0, int64_t r1,
                         const double* __restrict__ w, int stride, double* __restrict__ cnt)
{
    const int b = blockIdx.y;
    const IndT* row = ind + (int64_t)b * n_pad;
    double* c = cnt + (int64_t)b * stride;
    for (int64_t q = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < r1; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[row[q]], w ? w[q] : 1.0);
}

struct BasisArgs {
    int K, S;
    const int32_t* l_bin;
    const int32_t* l_type;
    const int32_t* l_degree;
    const int32_t* l_nknots;
    const int32_t* l_nstar;
    const double* b_xmin;
    const double* b_xmax;
    const double* b_h;           // equidistant step, 0 for exact binnings
    const double* b_z;           // [B][S] exact design points
    float* zb;                   // [K][S][4]
    double* zb64;                // [K][S][4]
    int32_t* zcol;               // [K][S]
};

__global__ void k_basis(BasisArgs a)
{
    const int k = blockIdx.x;
    const int b = a.l_bin[k];
    const int nst = a.l_nstar[k];
    const double xmin = a.b_xmin[b], xmax = a.b_xmax[b], h = a.b_h[b];
    for (int l = threadIdx.x; l < a.S; l += blockDim.x) {
        double N[kMaxNnz] = {0.0, 0.0, 0.0, 0.0};
        int col = 0;
        if (l < nst) {
            double z = (h > 0.0) ? __dadd_rn(xmin, __dmul_rn((double)l, h)) : a.b_z[(int64_t)b * a.S + l];
            if (a.l_type[k] == CWB_BL_LINEAR) {
                N[0] = 1.0;
                N[1] = z;
            } else if (a.l_type[k] == CWB_BL_CATEGORICAL) {
                N[0] = 1.0;                            // dummy design: class l has column l
                col = l;
            } else if (a.l_type[k] == CWB_BL_CATEGORICAL_BINARY) {
                N[0] = l == a.l_degree[k] ? 1.0 : 0.0; // indicator of the learner's class
            } else {
                col = bspline_nonzero(z, xmin, xmax, a.l_degree[k], a.l_nknots[k], N);
            }
        }
        int64_t o = ((int64_t)k * a.S + l) * kMaxNnz;
        for (int t = 0; t < kMaxNnz; ++t) {
            a.zb64[o + t] = N[t];
            a.zb[o + t] = (float)N[t];
        }
        a.zcol[(int64_t)k * a.S + l] = col;
    }
}

// Contiguous bin range [lo, hi) whose rows have a non-zero in column j (first
// non-zero columns are non-decreasing in the bin index).
__global__ void k_col_ranges(int S, int D, const int32_t* __restrict__ l_nstar, const int32_t* __restrict__ l_d,
                             const int32_t* __restrict__ l_nnz, const int32_t* __restrict__ zcol,
                             int32_t* __restrict__ crange)
{
    const int k = blockIdx.x;
    const int nst = l_nstar[k], d = l_d[k], nnz = l_nnz[k];
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        int lo = nst, hi = 0;
        if (j < d) {
            for (int l = 0; l < nst; ++l) {
                int c0 = zcol[(int64_t)k * S + l];
                if (c0 <= j && j < c0 + nnz) {
                    if (l < lo) lo = l;
                    hi = l + 1;
                }
            }
        }
        if (lo > hi) lo = hi = 0;
        crange[((int64_t)k * D + j) * 2] = lo;
        crange[((int64_t)k * D + j) * 2 + 1] = hi;
    }
}

// Column-major copy of the reduced design for the per-iteration s = Z^b^T u: column j's
// values over its contiguous bin range are stored contiguously at ztab[k][toff[k][j] ...].
__global__ void k_build_ztab(int S, int D, const int32_t* __restrict__ l_d, const float* __restrict__ zb,
                             const int32_t* __restrict__ zcol, const int32_t* __restrict__ crange,
                             int32_t* __restrict__ toff, float* __restrict__ ztab)
{
    const int k = blockIdx.x;
    const int d = l_d[k];
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        int off = 0;
        for (int jj = 0; jj < j && jj < d; ++jj)
            off += crange[((int64_t)k * D + jj) * 2 + 1] - crange[((int64_t)k * D + jj) * 2];
        toff[(int64_t)k * D + j] = off;
        if (j >= d) continue;
        const int lo = crange[((int64_t)k * D + j) * 2], hi = crange[((int64_t)k * D + j) * 2 + 1];
        float* out = ztab + (int64_t)k * kMaxNnz * S + off;
        for (int l = lo; l < hi; ++l) {
            const int t = j - zcol[(int64_t)k * S + l];
            out[l - lo] = (t >= 0 && t < kMaxNnz) ? zb[((int64_t)k * S + l) * kMaxNnz + t] : 0.0f;
        }
    }
}

// Low parts of the column-major design, ztab_lo = z - (float)z from the FP64 basis values: with
// ztab they hold every design value as a float-float pair for the solve's s = Z^b^T u.
__global__ void k_build_ztab_lo(int S, int D, const int32_t* __restrict__ l_d, const double* __restrict__ zb64,
                                const int32_t* __restrict__ zcol, const int32_t* __restrict__ crange,
                                const int32_t* __restrict__ toff, float* __restrict__ ztab_lo)
{
    const int k = blockIdx.x;
    const int d = l_d[k];
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const int lo = crange[((int64_t)k * D + j) * 2], hi = crange[((int64_t)k * D + j) * 2 + 1];
        float* out = ztab_lo + (int64_t)k * kMaxNnz * S + toff[(int64_t)k * D + j];
        for (int l = lo; l < hi; ++l) {
            const int t = j - zcol[(int64_t)k * S + l];
            const double z = (t >= 0 && t < kMaxNnz) ? zb64[((int64_t)k * S + l) * kMaxNnz + t] : 0.0;
            out[l - lo] = (float)(z - (double)(float)z);
        }
    }
}

// G = Z^b^T diag(cnt) Z^b (binMatMat, Algorithm 2), FP64, bins visited in order.
__global__ void k_gram(int S, int D, int K, const int32_t* __restrict__ l_bin, const int32_t* __restrict__ l_d,
                       const int32_t* __restrict__ l_nnz, const double* __restrict__ zb64,
                       const int32_t* __restrict__ zcol, const int32_t* __restrict__ crange,
                       const double* __restrict__ cnt /* [phase][B][S] */, int B, double* __restrict__ G)
{
    const int k = blockIdx.x, ph = blockIdx.y;
    const int d = l_d[k], nnz = l_nnz[k], b = l_bin[k];
    const double* c = cnt + ((int64_t)ph * B + b) * S;
    double* g = G + ((int64_t)ph * K + k) * D * D;
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
        int i = e / D, j = e % D;
        double s = 0.0;
        if (i < d && j < d && (i - j < nnz && j - i < nnz)) {
            int lo = max(crange[((int64_t)k * D + i) * 2], crange[((int64_t)k * D + j) * 2]);
            int hi = min(crange[((int64_t)k * D + i) * 2 + 1], crange[((int64_t)k * D + j) * 2 + 1]);
            for (int l = lo; l < hi; ++l) {
                int c0 = zcol[(int64_t)k * S + l];
                const double* z = zb64 + ((int64_t)k * S + l) * kMaxNnz;
                s += c[l] * z[i - c0] * z[j - c0];
            }
        }
        g[e] = s;
    }
}

// ---------------------------------------------------------------------------
// lambda from df and P = (G + lambda K)^-1 (App. A.2), one CTA of kLamThreads
// threads per learner and phase, everything in shared memory (d <= 64).
//
// With A = G + lambda K = L L^T and K = Dp^T Dp (Dp: the difference matrix),
//   df1(lambda) = tr(A^-1 G) = d - lambda tr(A^-1 K) = d - lambda ||Y||_F^2,
//   d df1 / d ln(lambda) = -lambda tr(A^-1 K) + lambda^2 tr((A^-1 K)^2)
//                        = -lambda ||Y||_F^2 + lambda^2 ||Y^T Y||_F^2,
// where Y = L^-1 Dp^T.  The root of df1 = df is bracketed in log10(lambda) within
// twelve decades of tr(G) / tr(K), as in the reference computation, and found by
// Newton steps in log(lambda) that fall back to bisection whenever a step leaves
// the bracket or does not halve the residual.  Every evaluation is a fresh
// factorisation of A on the definition (no eigen-decomposition).

constexpr int kLamThreads = 256;

struct LamArgs {
    int K, D;
    const int32_t* l_type;
    const int32_t* l_d;
    const int32_t* l_diff;
    const double* l_df;
    const double* l_lambda;
    const double* G;        // [2][K][D][D]
    double* P;              // [2][K][D][D]
    double* A;              // [2][K][D][D] criterion matrix P G P - 2 P
    double* lambda;         // [2][K]
    int32_t* status;        // [2][K]: 0 ok, 1 not positive definite, 2 df unreachable
    int phases;
};

// In-place Cholesky of the lower triangle of A (d x d, leading dimension d), right-looking:
// column j is scaled by 1 / L_jj, then the trailing lower triangle takes the rank-1 update.
// rinv[j] = 1 / L_jj.  Returns false (uniformly) if a pivot is not positive.
__device__ bool blk_cholesky(double* A, int d, double* rinv, int* fail)
{
    const int tid = threadIdx.x;
    if (tid == 0) *fail = 0;
    __syncthreads();
    for (int j = 0; j < d; ++j) {
        if (tid == 0) {
            const double p = A[j * d + j];
            if (!(p > 0.0)) {
                *fail = 1;
            } else {
                const double l = sqrt(p);
                A[j * d + j] = l;
                rinv[j] = 1.0 / l;
            }
        }
        __syncthreads();
        if (*fail) return false;
        for (int i = j + 1 + tid; i < d; i += blockDim.x) A[i * d + j] *= rinv[j];
        __syncthreads();
        const int m = d - j - 1;                 // trailing size; its lower triangle is updated
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int p = e / m, q = e - (e / m) * m;
            if (q > p) continue;
            const int r = j + 1 + p, c = j + 1 + q;
            A[r * d + c] -= A[r * d + j] * A[c * d + j];
        }
        __syncthreads();
    }
    return true;
}

// Block sum of one value per thread (fixed order: warp shuffles, then warps in order).
__device__ double blk_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kLamThreads) k_lambda(LamArgs a)
{
    const int k = blockIdx.x, ph = blockIdx.y;
    if (ph >= a.phases) return;
    const int tid = threadIdx.x;
    const int d = a.l_d[k];
    extern __shared__ double sm[];
    double* G = sm;                 // d x d
    double* A = G + d * d;          // d x d: G + lambda K, then its Cholesky factor
    double* Dp = A + d * d;         // nr x d difference matrix
    double* Y = Dp + d * d;         // d x nr: L^-1 Dp^T
    double* rinv = Y + d * d;       // d
    __shared__ double red[kLamThreads / 32];
    __shared__ int fail;
    __shared__ double sh_x;
    __shared__ int sh_done, sh_status;
    const double* Gs = a.G + ((int64_t)ph * a.K + k) * a.D * a.D;
    for (int e = tid; e < d * d; e += blockDim.x) G[e] = Gs[(e / d) * a.D + e % d];
    // P-splines: difference penalty of order diff_order; categorical ridge: the identity
    // (difference matrix of order 0); linear and binary learners: unpenalised
    const bool pspline = a.l_type[k] == CWB_BL_PSPLINE || a.l_type[k] == CWB_BL_CATEGORICAL;
    const int ord = a.l_type[k] == CWB_BL_PSPLINE ? a.l_diff[k] : 0;
    const int nr = d - ord;
    if (pspline) {
        // row r of the order-`ord` difference matrix: (-1)^(ord - t) binom(ord, t) at column r + t
        for (int e = tid; e < nr * d; e += blockDim.x) {
            const int r = e / d, c = e % d, t = c - r;
            double v = 0.0;
            if (t >= 0 && t <= ord) {
                double bin = 1.0;
                for (int u = 1; u <= t; ++u) bin = bin * (ord - u + 1) / u;
                v = ((ord - t) & 1) ? -bin : bin;
            }
            Dp[e] = v;
        }
    }
    __syncthreads();
    // A = G + lam K, K = Dp^T Dp
    auto form = [&](double lam) {
        for (int e = tid; e < d * d; e += blockDim.x) {
            const int i = e / d, j = e % d;
            double kv = 0.0;
            if (pspline)
                for (int r = max(0, max(i, j) - ord); r <= min(nr - 1, min(i, j)); ++r) kv += Dp[r * d + i] * Dp[r * d + j];
            A[e] = G[e] + lam * kv;
        }
        __syncthreads();
    };
    // df1(lam) and its derivative in ln(lam) from the factor in A; false if A is not PD
    auto evaluate = [&](double lam, double* v, double* dv) -> bool {
        form(lam);
        if (!blk_cholesky(A, d, rinv, &fail)) return false;
        // Y = L^-1 Dp^T: one column (difference row) per thread, forward substitution
        for (int r = tid; r < nr; r += blockDim.x) {
            for (int i = 0; i < d; ++i) {
                double t = Dp[r * d + i];
                for (int q = 0; q < i; ++q) t -= A[i * d + q] * Y[q * nr + r];
                Y[i * nr + r] = t * rinv[i];
            }
        }
        __syncthreads();
        double t1 = 0.0, t2 = 0.0;
        for (int e = tid; e < d * nr; e += blockDim.x) t1 += Y[e] * Y[e];
        for (int e = tid; e < nr * nr; e += blockDim.x) {
            const int r = e / nr, c = e % nr;
            double g = 0.0;
            for (int i = 0; i < d; ++i) g += Y[i * nr + r] * Y[i * nr + c];
            t2 += g * g;
        }
        t1 = blk_sum(t1, red);
        t2 = blk_sum(t2, red);
        *v = (double)d - lam * t1;
        *dv = -lam * t1 + lam * lam * t2;
        return true;
    };

    int status = 0;
    double lam = 0.0;
    if (pspline) {
        const double df = a.l_df[k];
        if (!(df > 0.0)) {
            lam = a.l_lambda[k];
        } else {
            // unpenalised fit: df1(0) = d when G is positive definite
            form(0.0);
            const bool g_pd = blk_cholesky(A, d, rinv, &fail);
            if (g_pd && df >= (double)d) {
                lam = 0.0;
            } else {
                double trg = 0.0, trk = 0.0;
                for (int i = 0; i < d; ++i) {
                    trg += G[i * d + i];
                    for (int r = max(0, i - ord); r <= min(nr - 1, i); ++r) trk += Dp[r * d + i] * Dp[r * d + i];
                }
                const double c = log10(trg / trk);
                double lo = c - 12.0, hi = c + 12.0, v = 0.0, dv = 0.0;
                if (!(trg > 0.0) || !(trk > 0.0)) status = 1;
                else if (!evaluate(pow(10.0, lo), &v, &dv)) status = 1;
                else if (v < df) lam = pow(10.0, lo);
                else if (!evaluate(pow(10.0, hi), &v, &dv)) status = 1;
                else if (v > df) status = 2;
                else {
                    if (tid == 0) {
                        sh_x = c;
                        sh_done = 0;
                        sh_status = 0;
                    }
                    __syncthreads();
                    double prev_res = INFINITY;
                    for (int it = 0; it < 200; ++it) {
                        const double x = sh_x;
                        if (!evaluate(pow(10.0, x), &v, &dv)) {
                            if (tid == 0) sh_status = 1;
                            __syncthreads();
                            break;
                        }
                        if (tid == 0) {
                            const double res = v - df;
                            if (res > 0.0) lo = x; else hi = x;
                            const double slope = dv * 2.302585092994046;     // d df1 / d log10(lambda)
                            const double xt = slope < 0.0 ? x - res / slope : x;
                            const bool in = xt > lo && xt < hi;
                            double xn;
                            if (fabs(res) <= 1e-13 * df) {            // converged: one last Newton step
                                xn = in ? xt : x;
                                sh_done = 1;
                            } else {
                                xn = (in && fabs(res) <= 0.5 * prev_res) ? xt : 0.5 * (lo + hi);
                                if (hi - lo < 1e-15 || xn == x) sh_done = 1;
                            }
                            prev_res = fabs(res);
                            sh_x = xn;
                        }
                        __syncthreads();
                        if (sh_done) break;
                    }
                    status = sh_status;
                    lam = pow(10.0, sh_x);
                }
            }
        }
    }
    // P = (G + lam K)^-1, zero outside d x d
    double* Pout = a.P + ((int64_t)ph * a.K + k) * a.D * a.D;
    for (int e = tid; e < a.D * a.D; e += blockDim.x) Pout[e] = 0.0;
    __syncthreads();
    if (status == 0) {
        form(lam);
        if (!blk_cholesky(A, d, rinv, &fail)) {
            status = 1;
        } else {
            // column j of A^-1: forward then backward substitution, one column per thread
            for (int j = tid; j < d; j += blockDim.x) {
                double* col = Y + j * d;          // Y is free now: d columns of length d
                for (int i = 0; i < d; ++i) {
                    double t = (i == j) ? 1.0 : 0.0;
                    for (int q = 0; q < i; ++q) t -= A[i * d + q] * col[q];
                    col[i] = t * rinv[i];
                }
                for (int i = d - 1; i >= 0; --i) {
                    double t = col[i];
                    for (int q = i + 1; q < d; ++q) t -= A[q * d + i] * col[q];
                    col[i] = t * rinv[i];
                }
                for (int i = 0; i < d; ++i) Pout[i * a.D + j] = col[i];
            }
            __syncthreads();
            // criterion matrix Acrit = P G P - 2 P: with theta = P s, theta^T G theta - 2 theta^T s =
            // s^T Acrit s, so the iteration's criterion needs no second product after theta.
            // T = G P overwrites the factor (no longer needed); Y holds P column by column.
            for (int e = tid; e < d * d; e += blockDim.x) {
                const int i = e / d, j = e % d;
                double t = 0.0;
                for (int q = 0; q < d; ++q) t += G[i * d + q] * Y[j * d + q];
                A[i * d + j] = t;
            }
            __syncthreads();
            double* Aout = a.A + ((int64_t)ph * a.K + k) * a.D * a.D;
            for (int e = tid; e < a.D * a.D; e += blockDim.x) {
                const int i = e / a.D, j = e % a.D;
                double v = 0.0;
                if (i < d && j < d) {
                    for (int q = 0; q < d; ++q) v += Y[q * d + i] * A[q * d + j];     // (P T)_ij, P symmetric
                    v -= 2.0 * Y[j * d + i];
                }
                Aout[e] = v;
            }
        }
    }
    if (tid == 0) {
        a.lambda[(int64_t)ph * a.K + k] = lam;
        a.status[(int64_t)ph * a.K + k] = status;
    }
}

// FP64 values as float-float pairs: hi = x rounded to FP32, lo = (x - hi) rounded (the solve
// evaluates its matrix products on the FP32 pipes; FP64 is a small fraction of the FP32 rate).
__global__ void k_split_df(const double* __restrict__ x, int64_t n, float2* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        const float hi = __double2float_rn(v);
        out[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

// ---------------------------------------------------------------------------
// Offset: loss-optimal constant over the fitting rows (L2: weighted mean,
// binomial: logit of the weighted mean).

constexpr int kOffsetBlocks = 256;

__global__ void k_offset_partial(const double* __restrict__ y, const double* __restrict__ w, int64_t n_fit,
                                 double* __restrict__ part /* [2][kOffsetBlocks] */)
{
    __shared__ double s1[kThreads], s2[kThreads];
    double a = 0.0, b = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_fit; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w ? w[i] : 1.0;
        a += wi * y[i];
        b += wi;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1[0];
        part[gridDim.x + blockIdx.x] = s2[0];
    }
}

__global__ void k_offset(const double* __restrict__ part, int nblk, int loss, double* __restrict__ out /* [0] offset, [1] mean */)
{
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblk; ++i) {
        a += part[i];
        b += part[nblk + i];
    }
    const double mean = a / b;
    out[1] = mean;
    out[0] = (loss == CWB_LOSS_L2) ? mean : log(mean / (1.0 - mean));
}

__global__ void k_init_rows(int64_t n_pad, float off_hi, float off_lo, float* f, float* h, float* c, float* rw)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
        f[2 * i] = off_hi;
        f[2 * i + 1] = off_lo;
        if (h) {
            h[2 * i] = off_hi;
            h[2 * i + 1] = off_lo;
        }
        if (c) c[i] = 0.0f;
        rw[i] = 0.0f;
        rw[n_pad + i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------

// Temporaries of a setup step: stream-ordered allocations on the model's stream, released in stream
// order when the step ends.  Unlike cudaFree, which waits for all work on the device, this never stalls
// on other models' kernels, so the setups of many fits (cwb_create_many) overlap.
struct TempBuf {
    std::vector<std::pair<void*, cudaStream_t>> ptrs;
    ~TempBuf()
    {
        for (auto& ps : ptrs) cudaFreeAsync(ps.first, ps.second);
    }
    template <typename T>
    cwb_status get(T** out, size_t count, cudaStream_t s)
    {
        void* p = nullptr;
        const size_t bytes = sizeof(T) * (count ? count : 1);
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
            return CWB_ENOMEM;
        }
        ptrs.push_back({p, s});
        *out = static_cast<T*>(p);
        return CWB_OK;
    }
};

int64_t isqrt64(int64_t n)
{
    int64_t s = (int64_t)sqrt((double)n);
    while (s > 0 && s * s > n) --s;
    while ((s + 1) * (s + 1) <= n) ++s;
    return s;
}

int grid_for(int64_t work, int device)
{
    int64_t g = ceil_div(work, kThreads);
    int64_t cap = (int64_t)num_sms(device) * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// Z^T W Z = Z^b^T diag(cnt) Z^b from the bin counts cnt [2 phases][B][S] (device), lambda from df and
// the cached P = (G + lambda K)^-1 with the criterion matrix, for `phases` caches (with one phase
// the second cache is a copy of the first).  Allocates the cache arrays on first use.
cwb_status build_caches(cwb_model* m, const double* cnt, int phases)
{
    cudaStream_t s = m->stream;
    const int K = m->K, D = m->d_max, S = m->nstar_max, B = m->B;
    const size_t dd = (size_t)D * D;
    TempBuf tmp;
    std::vector<int32_t> lnnz(K), ldiff(K);
    std::vector<double> ldf(K), llam(K);
    for (int k = 0; k < K; ++k) {
        lnnz[k] = m->lrn[k].nnz;
        ldiff[k] = m->lrn[k].spec.diff_order;
        ldf[k] = m->lrn[k].spec.df;
        llam[k] = m->lrn[k].spec.lambda;
    }
    int32_t *nnz_d = nullptr, *ldiff_d = nullptr, *lstat = nullptr;
    double *ldf_d = nullptr, *llam_d = nullptr;
    CWB_TRY(tmp.get(&nnz_d, (size_t)K, s));
    CWB_TRY(tmp.get(&ldiff_d, (size_t)K, s));
    CWB_TRY(tmp.get(&ldf_d, (size_t)K, s));
    CWB_TRY(tmp.get(&llam_d, (size_t)K, s));
    CWB_TRY(tmp.get(&lstat, (size_t)2 * K, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(nnz_d, lnnz.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(ldiff_d, ldiff.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(ldf_d, ldf.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(llam_d, llam.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
    if (!m->G) {
        CWB_TRY(dev_alloc((void**)&m->G, sizeof(double) * 2 * K * dd, s));
        CWB_TRY(dev_alloc((void**)&m->P, sizeof(double) * 2 * K * dd, s));
        CWB_TRY(dev_alloc((void**)&m->Acrit, sizeof(double) * 2 * K * dd, s));
        CWB_TRY(dev_alloc((void**)&m->Pdf, sizeof(float2) * 2 * K * dd, s));
        CWB_TRY(dev_alloc((void**)&m->Adf, sizeof(float2) * 2 * K * dd, s));
        CWB_TRY(dev_alloc((void**)&m->lambda, sizeof(double) * 2 * K, s));
    }
    k_gram<<<dim3(K, 2), kThreads, 0, s>>>(S, D, K, m->l_bin, m->l_d, nnz_d, m->zb64, m->zcol, m->crange, cnt, B, m->G);
    {
        LamArgs a{K, D, m->l_type, m->l_d, ldiff_d, ldf_d, llam_d, m->G, m->P, m->Acrit, m->lambda, lstat, phases};
        size_t smem = sizeof(double) * (4 * dd + D);
        CWB_CUDA_TRY(allow_max_dynamic_smem((const void*)k_lambda, m->device));
        k_lambda<<<dim3(K, phases), kLamThreads, smem, s>>>(a);
        if (phases == 1) {           // one cache serves both phases
            CWB_CUDA_TRY(cudaMemcpyAsync(m->P + (size_t)K * dd, m->P, sizeof(double) * K * dd, cudaMemcpyDeviceToDevice, s));
            CWB_CUDA_TRY(cudaMemcpyAsync(m->Acrit + (size_t)K * dd, m->Acrit, sizeof(double) * K * dd,
                                         cudaMemcpyDeviceToDevice, s));
            CWB_CUDA_TRY(cudaMemcpyAsync(m->lambda + K, m->lambda, sizeof(double) * K, cudaMemcpyDeviceToDevice, s));
            CWB_CUDA_TRY(cudaMemsetAsync(lstat + K, 0, sizeof(int32_t) * K, s));
        }
        const int gs = (int)std::min<int64_t>(1024, ((int64_t)2 * K * dd + kThreads - 1) / kThreads);
        k_split_df<<<gs, kThreads, 0, s>>>(m->P, (int64_t)2 * K * dd, m->Pdf);
        k_split_df<<<gs, kThreads, 0, s>>>(m->Acrit, (int64_t)2 * K * dd, m->Adf);
    }
    CWB_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> lstat_h(2 * K);
    CWB_CUDA_TRY(cudaMemcpyAsync(lstat_h.data(), lstat, sizeof(int32_t) * 2 * K, cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    for (int ph = 0; ph < phases; ++ph)
        for (int k = 0; k < K; ++k) {
            int st = lstat_h[(size_t)ph * K + k];
            if (st == 1) {
                set_error("learner " + std::to_string(k) + ": Z^T W Z + lambda K is not positive definite");
                return CWB_ENUMERIC;
            }
            if (st == 2) {
                set_error("learner " + std::to_string(k) + ": df is not reachable (at or below the penalty null space)");
                return CWB_ENUMERIC;
            }
        }
    return CWB_OK;
}

// Local statistics of a row shard for the setup exchange: unweighted bin counts [B][S] (host),
// sum of the targets and the row count, and the shard's bin-count bound of the scatter.
cwb_status shard_stats(cwb_model* m, double* counts_h, double sums_h[2], int32_t* cnt_log2)
{
    cudaStream_t s = m->stream;
    const int B = m->B, S = m->nstar_max;
    TempBuf tmp;
    double* cnt = nullptr;
    CWB_TRY(tmp.get(&cnt, (size_t)B * S, s));
    CWB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(double) * (size_t)B * S, s));
    if (S <= kCountSmemBins) {
        dim3 grid(std::min<int>(grid_for(m->n, m->device), 16), B);
        const size_t smem = sizeof(int) * (size_t)S;
        if (m->ind_bytes == 1) k_counts_smem<<<grid, kThreads, smem, s>>>((const uint8_t*)m->ind, m->n_pad, m->n, S, S, cnt);
        else k_counts_smem<<<grid, kThreads, smem, s>>>((const uint16_t*)m->ind, m->n_pad, m->n, S, S, cnt);
    } else {
        dim3 grid(std::min<int>(grid_for(m->n, m->device), 64), B);
        if (m->ind_bytes == 1) k_counts<<<grid, kThreads, 0, s>>>((const uint8_t*)m->ind, m->n_pad, 0, m->n, nullptr, S, cnt);
        else k_counts<<<grid, kThreads, 0, s>>>((const uint16_t*)m->ind, m->n_pad, 0, m->n, nullptr, S, cnt);
    }
    // sum of the targets: FP32 high parts and the low parts of FP64 targets, in FP64
    double* part = nullptr;
    CWB_TRY(tmp.get(&part, 2 * (size_t)kOffsetBlocks, s));
    double* y64 = nullptr;
    CWB_TRY(tmp.get(&y64, (size_t)m->n, s));
    k_join_f64<<<grid_for(m->n, m->device), kThreads, 0, s>>>(m->y, m->y_lo, m->n, y64);
    k_offset_partial<<<kOffsetBlocks, kThreads, 0, s>>>(y64, nullptr, m->n, part);
    std::vector<double> part_h(2 * kOffsetBlocks);
    CWB_CUDA_TRY(cudaGetLastError());
    CWB_CUDA_TRY(cudaMemcpyAsync(counts_h, cnt, sizeof(double) * (size_t)B * S, cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(part_h.data(), part, sizeof(double) * 2 * kOffsetBlocks, cudaMemcpyDeviceToHost, s));
    DevState st;
    CWB_CUDA_TRY(cudaMemcpyAsync(&st, m->state, sizeof(st), cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    double sy = 0.0, sn = 0.0;
    for (int i = 0; i < kOffsetBlocks; ++i) {
        sy += part_h[i];
        sn += part_h[kOffsetBlocks + i];
    }
    sums_h[0] = sy;
    sums_h[1] = sn;
    *cnt_log2 = st.cnt_log2[0];
    return CWB_OK;
}

// Completes a row shard's setup from the exchanged statistics: the caches from the global bin
// counts, the offset from the global target sum and row count, and the common fixed-point bound.
cwb_status shard_finish(cwb_model* m, const double* counts_h, const double sums_h[2], int32_t cnt_log2)
{
    cudaStream_t s = m->stream;
    const int B = m->B, S = m->nstar_max;
    if (cnt_log2 > 13) {
        set_error("shards: more than 8192 rows of one scatter cluster share a bin (heavily skewed bins are not supported "
                  "for row shards)");
        return CWB_EINVAL;
    }
    TempBuf tmp;
    double* cnt = nullptr;
    CWB_TRY(tmp.get(&cnt, (size_t)2 * B * S, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(cnt, counts_h, sizeof(double) * (size_t)B * S, cudaMemcpyHostToDevice, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(cnt + (size_t)B * S, counts_h, sizeof(double) * (size_t)B * S, cudaMemcpyHostToDevice, s));
    CWB_TRY(build_caches(m, cnt, 1));
    const double mean = sums_h[0] / sums_h[1];
    if (m->cfg.loss == CWB_LOSS_BINOMIAL && !(mean > 0.0 && mean < 1.0)) {
        set_error("binomial loss needs both classes among the rows of all shards");
        return CWB_EINVAL;
    }
    m->offset = m->cfg.loss == CWB_LOSS_L2 ? mean : log(mean / (1.0 - mean));
    const float off_hi = (float)m->offset;
    const float off_lo = (float)(m->offset - (double)off_hi);
    k_init_rows<<<grid_for(m->n_pad, m->device), kThreads, 0, s>>>(m->n_pad, off_hi, off_lo, m->f, m->h, m->c, m->rw);
    CWB_CUDA_TRY(cudaMemcpyAsync(&m->state->cnt_log2[0], &cnt_log2, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CWB_CUDA_TRY(cudaGetLastError());
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    return CWB_OK;
}

cwb_status setup_model(cwb_model* m, const void* X_in, int x_dtype, const void* y_in, const double* w_in,
                       const uint8_t* val_mask, int device_ptrs)
{
    cudaStream_t s = m->stream;
    const int64_t n = m->n;
    const int32_t p = m->p;
    const size_t xsz = x_dtype == CWB_F64 ? 8 : 4;
    TempBuf tmp;

    // --- row order: training rows first (HCWB), original order otherwise
    std::vector<int32_t> perm_h;
    if (m->hybrid) {
        std::vector<uint8_t> mask(n);
        if (device_ptrs) {
            CWB_CUDA_TRY(cudaMemcpyAsync(mask.data(), val_mask, (size_t)n, cudaMemcpyDeviceToHost, s));
            CWB_CUDA_TRY(cudaStreamSynchronize(s));
        } else {
            std::memcpy(mask.data(), val_mask, (size_t)n);
        }
        perm_h.reserve(n);
        for (int64_t i = 0; i < n; ++i)
            if (!mask[i]) perm_h.push_back((int32_t)i);
        m->n_tr = (int64_t)perm_h.size();
        for (int64_t i = 0; i < n; ++i)
            if (mask[i]) perm_h.push_back((int32_t)i);
        if (m->n_tr < 2 || m->n_tr == n) {
            set_error("HCWB needs at least two training rows and one validation row");
            return CWB_EINVAL;
        }
        CWB_TRY(dev_alloc((void**)&m->perm, sizeof(int32_t) * n, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(m->perm, perm_h.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    } else {
        m->n_tr = n;
    }
    m->n_pad = ceil_div(n, kRowAlign) * kRowAlign;
    const int64_t n_pad = m->n_pad;

    // --- inputs on the device (caller's buffers are only read during this call)
    const void* Xd = X_in;
    const void* yd = y_in;
    const double* wd = w_in;
    if (!device_ptrs) {
        void* xb = nullptr;
        CWB_TRY(tmp.get((char**)&xb, xsz * (size_t)n * p, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(xb, X_in, xsz * (size_t)n * p, cudaMemcpyHostToDevice, s));
        Xd = xb;
        void* yb = nullptr;
        CWB_TRY(tmp.get((char**)&yb, xsz * (size_t)n, s));
        CWB_CUDA_TRY(cudaMemcpyAsync(yb, y_in, xsz * (size_t)n, cudaMemcpyHostToDevice, s));
        yd = yb;
        if (w_in) {
            double* wb = nullptr;
            CWB_TRY(tmp.get(&wb, (size_t)n, s));
            CWB_CUDA_TRY(cudaMemcpyAsync(wb, w_in, sizeof(double) * n, cudaMemcpyHostToDevice, s));
            wd = wb;
        }
    }
    const int g_rows = grid_for(n_pad, m->device);

    // --- validity checks on the data
    uint32_t* flags = nullptr;
    CWB_TRY(tmp.get(&flags, 8, s));
    CWB_CUDA_TRY(cudaMemsetAsync(flags, 0, 32, s));
    if (m->cfg.loss == CWB_LOSS_BINOMIAL) {
        if (x_dtype == CWB_F64) k_check_binary<<<g_rows, kThreads, 0, s>>>((const double*)yd, n, flags);
        else k_check_binary<<<g_rows, kThreads, 0, s>>>((const float*)yd, n, flags);
    }
    {
        if (x_dtype == CWB_F64) k_check_finite<<<g_rows, kThreads, 0, s>>>((const double*)yd, n, flags + 5);
        else k_check_finite<<<g_rows, kThreads, 0, s>>>((const float*)yd, n, flags + 5);
    }
    if (wd) k_check_weights<<<g_rows, kThreads, 0, s>>>(wd, n, flags + 1);

    // --- y, w in the fitting order (FP64 copies kept for the offset and the counts)
    double* y64 = nullptr;
    CWB_TRY(tmp.get(&y64, (size_t)n, s));
    if (x_dtype == CWB_F64) k_gather_f64<<<g_rows, kThreads, 0, s>>>((const double*)yd, m->perm, n, y64);
    else k_gather_f64<<<g_rows, kThreads, 0, s>>>((const float*)yd, m->perm, n, y64);
    CWB_TRY(dev_alloc((void**)&m->y, sizeof(float) * n_pad, s));
    if (x_dtype == CWB_F64) CWB_TRY(dev_alloc((void**)&m->y_lo, sizeof(float) * n_pad, s));
    k_split_f64<<<g_rows, kThreads, 0, s>>>(y64, n, n_pad, m->y, m->y_lo);
    double* w64 = nullptr;
    if (wd) {
        m->weighted = true;
        CWB_TRY(tmp.get(&w64, (size_t)n, s));
        k_gather_f64<<<g_rows, kThreads, 0, s>>>(wd, m->perm, n, w64);
        CWB_TRY(dev_alloc((void**)&m->w, sizeof(float) * n_pad, s));
        k_split_f64<<<g_rows, kThreads, 0, s>>>(w64, n, n_pad, m->w, nullptr);
    }
    CWB_CUDA_TRY(cudaGetLastError());

    // --- binnings: one per distinct (feature, n_bins) pair
    const int B = (int)m->bins.size();
    std::vector<int32_t> feat_h(B);
    for (int b = 0; b < B; ++b) feat_h[b] = m->bins[b].feature;
    int32_t* feat_d = nullptr;
    CWB_TRY(tmp.get(&feat_d, (size_t)B, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(feat_d, feat_h.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s));
    const int nblk = std::max(1, std::min<int>(std::max(1, 2048 / std::max(B, 1)), (int)ceil_div(n, kThreads)));
    double *pmin = nullptr, *pmax = nullptr, *xmin_d = nullptr, *xmax_d = nullptr;
    CWB_TRY(tmp.get(&pmin, (size_t)B * nblk, s));
    CWB_TRY(tmp.get(&pmax, (size_t)B * nblk, s));
    CWB_TRY(tmp.get(&xmin_d, (size_t)B, s));
    CWB_TRY(tmp.get(&xmax_d, (size_t)B, s));
    {
        dim3 grid(nblk, B);
        if (x_dtype == CWB_F64) k_minmax_partial<<<grid, kThreads, 0, s>>>((const double*)Xd, feat_d, n, pmin, pmax, flags + 2);
        else k_minmax_partial<<<grid, kThreads, 0, s>>>((const float*)Xd, feat_d, n, pmin, pmax, flags + 2);
        k_minmax_final<<<B, 32, 0, s>>>(pmin, pmax, nblk, xmin_d, xmax_d);
    }
    for (int b = 0; b < B; ++b) {
        const HostBinning& hb = m->bins[b];
        if (!hb.categories) continue;
        if (x_dtype == CWB_F64) k_check_codes<<<g_rows, kThreads, 0, s>>>((const double*)Xd, hb.feature, n, hb.categories, flags + 4);
        else k_check_codes<<<g_rows, kThreads, 0, s>>>((const float*)Xd, hb.feature, n, hb.categories, flags + 4);
    }
    std::vector<double> xmin_h(B), xmax_h(B);
    uint32_t flags_h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    CWB_CUDA_TRY(cudaMemcpyAsync(xmin_h.data(), xmin_d, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(xmax_h.data(), xmax_d, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaMemcpyAsync(flags_h, flags, sizeof(flags_h), cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags_h[0]) { set_error("binomial loss needs targets in {0, 1}"); return CWB_EINVAL; }
    if (flags_h[1]) { set_error("observation weights must be finite and > 0"); return CWB_EINVAL; }
    if (flags_h[2]) { set_error("features must be finite"); return CWB_EINVAL; }
    if (flags_h[5]) { set_error("targets must be finite"); return CWB_EINVAL; }
    if (flags_h[4]) { set_error("a categorical feature holds a value that is not a class code 0..c-1"); return CWB_EINVAL; }
    if (m->shard) {
        // a row shard bins on the ranges of all shards' rows (equidistant design points are then
        // the same on every shard); the local rows must lie inside them
        for (int b = 0; b < B; ++b) {
            if (m->bins[b].categories) continue;
            const int f = m->bins[b].feature;
            const double gl = m->shard_xmin[f], gh = m->shard_xmax[f];
            if (!(xmin_h[b] >= gl && xmax_h[b] <= gh)) {
                set_error("shard rows of feature " + std::to_string(f) + " lie outside the given global range");
                return CWB_EINVAL;
            }
            xmin_h[b] = gl;
            xmax_h[b] = gh;
        }
    }
    for (int b = 0; b < B; ++b) {
        if (!(xmax_h[b] > xmin_h[b])) {
            set_error("feature " + std::to_string(m->bins[b].feature) + " is constant (max == min)");
            return CWB_EINVAL;
        }
        if (m->bins[b].categories) {
            // class codes: design point l is class l, i.e. equidistant points 0, 1, ..., c-1
            xmin_h[b] = 0.0;
            xmax_h[b] = (double)(m->bins[b].categories - 1);
        }
        m->bins[b].xmin = xmin_h[b];
        m->bins[b].xmax = xmax_h[b];
    }

    // --- exact binnings: sorted unique values on the device
    int64_t npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    int S = 2;
    bool any_exact = false;
    for (int b = 0; b < B; ++b) {
        HostBinning& hb = m->bins[b];
        if (hb.categories) {
            hb.exact = 0;
            hb.nstar = hb.categories;
        } else if (hb.nbins_spec == CWB_BINS_EXACT) {
            hb.exact = 1;
            any_exact = true;
        } else {
            hb.exact = 0;
            const int64_t n_sqrt = m->shard ? m->shard_n_global : n;      // a shard uses the global row count
            hb.nstar = hb.nbins_spec == CWB_BINS_SQRT ? (int)std::min<int64_t>(isqrt64(n_sqrt), 1 << 30) : hb.nbins_spec;
        }
    }
    double* keys = nullptr;
    std::vector<double*> zvals(B, nullptr);
    if (any_exact) {
        CWB_TRY(tmp.get(&keys, (size_t)npow2, s));
        int32_t* cnt_d = nullptr;
        CWB_TRY(tmp.get(&cnt_d, (size_t)B, s));
        const int gp = grid_for(npow2, m->device);
        for (int b = 0; b < B; ++b) {
            if (!m->bins[b].exact) continue;
            CWB_TRY(tmp.get(&zvals[b], (size_t)n, s));
            if (x_dtype == CWB_F64) k_load_sort_keys<<<gp, kThreads, 0, s>>>((const double*)Xd, m->bins[b].feature, n, npow2, keys);
            else k_load_sort_keys<<<gp, kThreads, 0, s>>>((const float*)Xd, m->bins[b].feature, n, npow2, keys);
            for (int64_t k2 = 2; k2 <= npow2; k2 <<= 1)
                for (int64_t j = k2 >> 1; j > 0; j >>= 1) k_bitonic_pass<<<gp, kThreads, 0, s>>>(keys, npow2, j, k2);
            k_unique_single_block<<<1, 1024, 0, s>>>(keys, n, zvals[b], cnt_d + b);
        }
        std::vector<int32_t> cnt_h(B, 0);
        CWB_CUDA_TRY(cudaMemcpyAsync(cnt_h.data(), cnt_d, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s));
        CWB_CUDA_TRY(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b)
            if (m->bins[b].exact) m->bins[b].nstar = cnt_h[b];
    }
    for (int b = 0; b < B; ++b) {
        int ns = m->bins[b].nstar;
        if (ns < 2 || ns > CWB_MAX_BINS) {
            set_error("feature " + std::to_string(m->bins[b].feature) + ": number of design points " +
                      std::to_string(ns) + " outside [2, 65535]");
            return CWB_EINVAL;
        }
        S = std::max(S, ns);
    }
    m->nstar_max = S;
    m->ind_bytes = S <= 256 ? 1 : 2;

    // --- index vectors [B][n_pad]
    CWB_TRY(dev_alloc(&m->ind, (size_t)m->ind_bytes * B * n_pad, s));
    std::vector<double> h_h(B, 0.0);
    std::vector<BinJob> jobs_h;
    for (int b = 0; b < B; ++b) {
        const HostBinning& hb = m->bins[b];
        if (hb.exact) {
            uint32_t* errp = flags + 3;
            if (m->ind_bytes == 1) {
                uint8_t* out = (uint8_t*)m->ind + (int64_t)b * n_pad;
                if (x_dtype == CWB_F64) k_bin_exact<<<g_rows, kThreads, 0, s>>>((const double*)Xd, hb.feature, m->perm, n, n_pad, zvals[b], hb.nstar, out, errp);
                else k_bin_exact<<<g_rows, kThreads, 0, s>>>((const float*)Xd, hb.feature, m->perm, n, n_pad, zvals[b], hb.nstar, out, errp);
            } else {
                uint16_t* out = (uint16_t*)m->ind + (int64_t)b * n_pad;
                if (x_dtype == CWB_F64) k_bin_exact<<<g_rows, kThreads, 0, s>>>((const double*)Xd, hb.feature, m->perm, n, n_pad, zvals[b], hb.nstar, out, errp);
                else k_bin_exact<<<g_rows, kThreads, 0, s>>>((const float*)Xd, hb.feature, m->perm, n, n_pad, zvals[b], hb.nstar, out, errp);
            }
        } else {
            const double h = (hb.xmax - hb.xmin) / (double)(hb.nstar - 1);
            h_h[b] = h;
            jobs_h.push_back(BinJob{(int64_t)hb.feature, hb.xmin, h, hb.nstar, b});
        }
    }
    if (!jobs_h.empty()) {
        // all equidistant binnings in one launch: the row grid of one binning, once per binning
        // (a thread takes a few rows, so the loads of the launch are in flight together)
        BinJob* jobs = nullptr;
        CWB_TRY(tmp.get(&jobs, jobs_h.size(), s));
        CWB_CUDA_TRY(cudaMemcpyAsync(jobs, jobs_h.data(), sizeof(BinJob) * jobs_h.size(), cudaMemcpyHostToDevice, s));
        const int nj = (int)jobs_h.size();
        const dim3 grid((unsigned)g_rows, (unsigned)nj);
        if (m->ind_bytes == 1) {
            if (x_dtype == CWB_F64) k_bin_equidistant<<<grid, kThreads, 0, s>>>((const double*)Xd, jobs, m->perm, n, n_pad, (uint8_t*)m->ind);
            else k_bin_equidistant<<<grid, kThreads, 0, s>>>((const float*)Xd, jobs, m->perm, n, n_pad, (uint8_t*)m->ind);
        } else {
            if (x_dtype == CWB_F64) k_bin_equidistant<<<grid, kThreads, 0, s>>>((const double*)Xd, jobs, m->perm, n, n_pad, (uint16_t*)m->ind);
            else k_bin_equidistant<<<grid, kThreads, 0, s>>>((const float*)Xd, jobs, m->perm, n, n_pad, (uint16_t*)m->ind);
        }
    }
    CWB_CUDA_TRY(cudaGetLastError());

    // --- per-learner tables
    const int K = m->K;
    int D = 0;
    for (const HostLearner& L : m->lrn) D = std::max(D, L.d);
    m->d_max = D;
    std::vector<int32_t> lb(K), lt(K), ldeg(K), lnk(K), lns(K), ld(K), lnnz(K), ldiff(K);
    std::vector<double> ldf(K), llam(K), lxmin(K), lxmax(K);
    for (int k = 0; k < K; ++k) {
        const HostLearner& L = m->lrn[k];
        lb[k] = L.binning;
        lt[k] = L.spec.type;
        ldeg[k] = L.spec.type == CWB_BL_CATEGORICAL_BINARY ? L.spec.level : L.spec.degree;   // binary: its class
        lnk[k] = L.spec.n_knots;
        lns[k] = m->bins[L.binning].nstar;
        ld[k] = L.d;
        lnnz[k] = L.nnz;
        ldiff[k] = L.spec.diff_order;
        ldf[k] = L.spec.df;
        llam[k] = L.spec.lambda;
        lxmin[k] = m->bins[L.binning].xmin;
        lxmax[k] = m->bins[L.binning].xmax;
    }
    auto upload_i = [&](int32_t** dst, const std::vector<int32_t>& v, bool keep) -> cwb_status {
        if (keep) CWB_TRY(dev_alloc((void**)dst, sizeof(int32_t) * v.size(), s));
        else CWB_TRY(tmp.get(dst, v.size(), s));
        CWB_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice, s));
        return CWB_OK;
    };
    auto upload_d = [&](double** dst, const std::vector<double>& v, bool keep) -> cwb_status {
        if (keep) CWB_TRY(dev_alloc((void**)dst, sizeof(double) * v.size(), s));
        else CWB_TRY(tmp.get(dst, v.size(), s));
        CWB_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, s));
        return CWB_OK;
    };
    int32_t *nnz_d = nullptr, *ldiff_d = nullptr;
    double *ldf_d = nullptr, *llam_d = nullptr, *bxmin_d = nullptr, *bxmax_d = nullptr, *bh_d = nullptr;
    CWB_TRY(upload_i(&m->l_bin, lb, true));
    CWB_TRY(upload_i(&m->l_type, lt, true));
    CWB_TRY(upload_i(&m->l_degree, ldeg, true));
    CWB_TRY(upload_i(&m->l_nknots, lnk, true));
    CWB_TRY(upload_i(&m->l_nstar, lns, true));
    CWB_TRY(upload_i(&m->l_d, ld, true));
    CWB_TRY(upload_d(&m->l_xmin, lxmin, true));
    CWB_TRY(upload_d(&m->l_xmax, lxmax, true));
    CWB_TRY(upload_i(&nnz_d, lnnz, false));
    CWB_TRY(upload_i(&ldiff_d, ldiff, false));
    CWB_TRY(upload_d(&ldf_d, ldf, false));
    CWB_TRY(upload_d(&llam_d, llam, false));
    CWB_TRY(upload_d(&bxmin_d, xmin_h, false));
    CWB_TRY(upload_d(&bxmax_d, xmax_h, false));
    CWB_TRY(upload_d(&bh_d, h_h, false));
    double* bz_d = nullptr;
    if (any_exact) {
        CWB_TRY(tmp.get(&bz_d, (size_t)B * S, s));
        for (int b = 0; b < B; ++b)
            if (m->bins[b].exact)
                CWB_CUDA_TRY(cudaMemcpyAsync(bz_d + (int64_t)b * S, zvals[b], sizeof(double) * m->bins[b].nstar,
                                             cudaMemcpyDeviceToDevice, s));
    }
    CWB_TRY(dev_alloc((void**)&m->zb, sizeof(float) * (size_t)K * S * kMaxNnz, s));
    CWB_TRY(dev_alloc((void**)&m->zb64, sizeof(double) * (size_t)K * S * kMaxNnz, s));
    CWB_TRY(dev_alloc((void**)&m->zcol, sizeof(int32_t) * (size_t)K * S, s));
    CWB_TRY(dev_alloc((void**)&m->crange, sizeof(int32_t) * (size_t)K * D * 2, s));
    {
        BasisArgs a{K, S, m->l_bin, m->l_type, m->l_degree, m->l_nknots, m->l_nstar, bxmin_d, bxmax_d, bh_d, bz_d,
                    m->zb, m->zb64, m->zcol};
        k_basis<<<K, kThreads, 0, s>>>(a);
        k_col_ranges<<<K, 64, 0, s>>>(S, D, m->l_nstar, m->l_d, nnz_d, m->zcol, m->crange);
        CWB_TRY(dev_alloc((void**)&m->toff, sizeof(int32_t) * (size_t)K * D, s));
        CWB_TRY(dev_alloc((void**)&m->ztab, sizeof(float) * (size_t)K * kMaxNnz * S, s));
        CWB_CUDA_TRY(cudaMemsetAsync(m->ztab, 0, sizeof(float) * (size_t)K * kMaxNnz * S, s));
        k_build_ztab<<<K, 64, 0, s>>>(S, D, m->l_d, m->zb, m->zcol, m->crange, m->toff, m->ztab);
        CWB_TRY(dev_alloc((void**)&m->ztab_lo, sizeof(float) * (size_t)K * kMaxNnz * S, s));
        CWB_CUDA_TRY(cudaMemsetAsync(m->ztab_lo, 0, sizeof(float) * (size_t)K * kMaxNnz * S, s));
        k_build_ztab_lo<<<K, 64, 0, s>>>(S, D, m->l_d, m->zb64, m->zcol, m->crange, m->toff, m->ztab_lo);
    }

    // --- weighted bin counts per phase: phase 0 = fitting rows of the first phase, phase 1 = all rows
    const int phases = m->hybrid ? 2 : 1;
    double* cnt = nullptr;
    CWB_TRY(tmp.get(&cnt, (size_t)2 * B * S, s));
    CWB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(double) * (size_t)2 * B * S, s));
    for (int ph = 0; ph < phases; ++ph) {
        int64_t r1 = (ph == 0) ? m->n_tr : n;
        double* out = cnt + (int64_t)ph * B * S;
        if (!w64 && S <= kCountSmemBins) {
            // nstar_max bins per CTA (every binning's counts fit); a few CTAs per binning
            dim3 grid(std::min<int>(grid_for(r1, m->device), 16), B);
            const size_t smem = sizeof(int) * (size_t)S;
            if (m->ind_bytes == 1) k_counts_smem<<<grid, kThreads, smem, s>>>((const uint8_t*)m->ind, n_pad, r1, S, S, out);
            else k_counts_smem<<<grid, kThreads, smem, s>>>((const uint16_t*)m->ind, n_pad, r1, S, S, out);
        } else {
            dim3 grid(std::min<int>(grid_for(r1, m->device), 64), B);
            if (m->ind_bytes == 1) k_counts<<<grid, kThreads, 0, s>>>((const uint8_t*)m->ind, n_pad, 0, r1, w64, S, out);
            else k_counts<<<grid, kThreads, 0, s>>>((const uint16_t*)m->ind, n_pad, 0, r1, w64, S, out);
        }
    }
    if (phases == 1)
        CWB_CUDA_TRY(cudaMemcpyAsync(cnt + (int64_t)B * S, cnt, sizeof(double) * (size_t)B * S, cudaMemcpyDeviceToDevice, s));

    // --- G, lambda, P per learner and phase
    CWB_CUDA_TRY(cudaMemcpyAsync(flags_h, flags, sizeof(flags_h), cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags_h[3]) { set_error("internal: exact binning lookup failed"); return CWB_ENUMERIC; }
    CWB_TRY(build_caches(m, cnt, phases));

    // --- offset and initial models
    double *off_d = nullptr, *off_part = nullptr;
    CWB_TRY(tmp.get(&off_d, 2, s));
    CWB_TRY(tmp.get(&off_part, 2 * kOffsetBlocks, s));
    k_offset_partial<<<kOffsetBlocks, kThreads, 0, s>>>(y64, w64, m->n_tr, off_part);
    k_offset<<<1, 32, 0, s>>>(off_part, kOffsetBlocks, m->cfg.loss, off_d);
    double off_h[2] = {0.0, 0.0};
    CWB_CUDA_TRY(cudaMemcpyAsync(off_h, off_d, sizeof(off_h), cudaMemcpyDeviceToHost, s));
    CWB_CUDA_TRY(cudaStreamSynchronize(s));
    if (m->cfg.loss == CWB_LOSS_BINOMIAL && !(off_h[1] > 0.0 && off_h[1] < 1.0)) {
        set_error("binomial loss needs both classes among the fitting rows");
        return CWB_EINVAL;
    }
    m->offset = off_h[0];
    CWB_TRY(dev_alloc((void**)&m->f, sizeof(float) * 2 * n_pad, s));
    if (m->accel) {
        CWB_TRY(dev_alloc((void**)&m->h, sizeof(float) * 2 * n_pad, s));
        CWB_TRY(dev_alloc((void**)&m->c, sizeof(float) * n_pad, s));
    }
    CWB_TRY(dev_alloc((void**)&m->rw, sizeof(float) * 2 * n_pad, s));
    const float off_hi = (float)m->offset;
    const float off_lo = (float)(m->offset - (double)off_hi);
    k_init_rows<<<g_rows, kThreads, 0, s>>>(n_pad, off_hi, off_lo, m->f, m->h, m->c, m->rw);
    CWB_CUDA_TRY(cudaGetLastError());
    CWB_CUDA_TRY(cudaStreamSynchronize(s));     // temporaries are released on return
    return CWB_OK;
}

}  // namespace cwb
