// cwb_device.cuh -- device helpers shared by the iteration kernels (cwb_iter.cu, cwb_persist.cu):
// programmatic-dependency and fence wrappers, index-vector loads, compensated float-float
// arithmetic, losses, mbarrier / TMA wrappers, the fixed-point scale of the histograms and the
// order-preserving keys of the argmin.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "cwb_internal.cuh"

namespace cwb {
namespace {

// Programmatic dependent launch: the iteration's kernels are launched so that each may start
// while its predecessor drains.  grid_dep_wait() blocks until the predecessor grid has completed
// and its memory is visible (a no-op without a programmatic dependency); grid_dep_launch() lets
// the successor grid be scheduled.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Release / acquire fence at GPU scope for the last-block tickets (the data behind a ticket is
// read with L2 loads); cheaper than the sequentially consistent fence of __threadfence().
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

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

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// The same test with an explicit suspend-time hint: the thread sleeps until the phase completes or
// kSuspendNs nanoseconds pass.  In the scatter's deep rings (1M x 50: 7 stages) the waits of idle
// pipeline warps otherwise return often enough to take issue slots from the working warps (measured
// on one GPU, same process: scatter 36.8 us with the hint, 37.1 us without); with the HCWB plan's
// 4 stages the hint costs time (363 us against 357 us), so the plan chooses (ScatterArgs::sleep_waits).
constexpr uint32_t kSuspendNs = 100000;

__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false once the deadline (SM clock) passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long deadline, bool sleep = false)
{
    if (sleep) {
        while (!mbar_try_wait_sleep(bar, parity))
            if (clock64() > deadline) return false;
        return true;
    }
    while (!mbar_try_wait(bar, parity))
        if (clock64() > deadline) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz: a stuck pipeline reports an error

template <typename IndT>
__device__ __forceinline__ void unpack16(uint4 raw, int out[16 / sizeof(IndT)]);

template <>
__device__ __forceinline__ void unpack16<uint16_t>(uint4 raw, int out[8])
{
    uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        out[2 * t] = w[t] & 0xffff;
        out[2 * t + 1] = w[t] >> 16;
    }
}

template <>
__device__ __forceinline__ void unpack16<uint8_t>(uint4 raw, int out[16])
{
    uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        out[4 * t] = w[t] & 0xff;
        out[4 * t + 1] = (w[t] >> 8) & 0xff;
        out[4 * t + 2] = (w[t] >> 16) & 0xff;
        out[4 * t + 3] = w[t] >> 24;
    }
}

// Fixed-point exponent of a histogram channel: values are w r * 2^s rounded to
// int32.  With max|w r| < 2^e and at most 2^c rows of one cluster in one bin,
// s = 30 - c - e keeps every cluster sum below 2^30 in magnitude.
__device__ __forceinline__ int fixed_scale(uint32_t rmax_bits, int cnt_log2)
{
    if (rmax_bits == 0) return 100;
    const int E = (int)((rmax_bits >> 23) & 0xff);
    const int e = (E == 0) ? -126 : E - 126;
    return max(-120, min(100, 30 - cnt_log2 - e));
}

// Upper bound (FP32 bits) on max |w r| of the residuals a row pass is about to form, known before
// the pass: binomial |y - sigmoid(f)| < 1, so max w bounds it; L2 residuals move by at most
// nu max|w| max|v_k*| from the previous ones (max |w r| of the previous pass, rprev) when an update
// is pending.  A relative margin of 2^-12 covers the rounding of the compensated update.
__device__ __forceinline__ uint32_t residual_bound(int loss, bool pending, uint32_t rprev_bits, float vmax_sel,
                                                   float nu, float wmax)
{
    float b;
    if (loss == CWB_LOSS_BINOMIAL) b = wmax;
    else b = __uint_as_float(rprev_bits) + (pending ? nu * wmax * vmax_sel : 0.0f);
    b = b * (1.0f + 1.0f / 4096.0f);
    return __float_as_uint(b);
}

// 2^e as an FP32 value for -126 <= e <= 127 (fixed_scale keeps every exponent used here in range).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Criteria are compared as integers: an FP64 value maps to a signed 64-bit key with the
// same order (negative values have their magnitude bits flipped); the map is its own
// inverse.  Integer compares keep the argmin off the (slow) FP64 pipe.
__device__ __forceinline__ long long order_key(double q)
{
    const long long b = __double_as_longlong(q);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_value(long long k) { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL)); }

// (best key, index of best, second best key); ties go to the lowest index.
struct Best2 {
    long long q1, q2;
    int k1;
};

__device__ __forceinline__ Best2 best2_merge(Best2 a, Best2 b)
{
    const bool take_b = b.k1 >= 0 && (a.k1 < 0 || b.q1 < a.q1 || (b.q1 == a.q1 && b.k1 < a.k1));
    Best2 r;
    if (take_b) {
        r.q1 = b.q1;
        r.k1 = b.k1;
        r.q2 = min(a.q1, min(a.q2, b.q2));
    } else {
        r.q1 = a.q1;
        r.k1 = a.k1;
        r.q2 = min(a.q2, min(b.q1, b.q2));
    }
    return r;
}

__device__ __forceinline__ Best2 best2_shfl(Best2 x, int o)
{
    Best2 y;
    y.q1 = __shfl_xor_sync(0xffffffffu, x.q1, o);
    y.q2 = __shfl_xor_sync(0xffffffffu, x.q2, o);
    y.k1 = __shfl_xor_sync(0xffffffffu, x.k1, o);
    return y;
}

// DF of an exact integer |x| < 2^62: high part rounded to FP32, the remainder (exact in int64,
// below 2^39 in magnitude) rounded to FP32 (together 48 significant bits).
__device__ __forceinline__ DF df_of_ll(long long x)
{
    const float hi = __ll2float_rn(x);
    const long long rem = x - (long long)hi;
    return {hi, __ll2float_rn(rem)};
}

__device__ __forceinline__ DF df_scale(DF a, float p2) { return {a.hi * p2, a.lo * p2}; }

__device__ __forceinline__ DF df_shfl_xor(DF x, int o, unsigned mask = 0xffffffffu)
{
    return {__shfl_xor_sync(mask, x.hi, o), __shfl_xor_sync(mask, x.lo, o)};
}

}  // namespace
}  // namespace cwb
