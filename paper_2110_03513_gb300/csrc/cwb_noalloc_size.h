/*
 * cwb_noalloc_size.h -- size check of cwb_predict_noalloc (host code, plain C).
 *
 * The allocation-free prediction stages a request in one fixed device array:
 * the p x n_new input rows (xsz bytes per value) rounded up to 256 bytes, then
 * n_new FP32 predictions.  cwb_noalloc_need() decides whether a request fits
 * before it forms any of these products, so that a huge n_new cannot wrap a
 * size around and slip past the limit.
 */
#ifndef CWB_NOALLOC_SIZE_H
#define CWB_NOALLOC_SIZE_H

#include <stdint.h>

/* Returns 1 and sets *need (bytes used in the array) when n_new rows of p features of xsz bytes
 * fit in `limit` bytes; returns 0, leaving *need untouched, when they do not or when an argument
 * is out of range (n_new < 0, p < 1, xsz not 4 or 8, limit < 256). */
static inline int cwb_noalloc_need(int64_t n_new, int64_t p, int64_t xsz, uint64_t limit, uint64_t* need)
{
    if (n_new < 0 || p < 1 || p > INT32_MAX || (xsz != 4 && xsz != 8) || limit < 256) return 0;
    /* per row: the staged features and one prediction; p <= 2^31 keeps this below 2^35 */
    const uint64_t per_row = (uint64_t)xsz * (uint64_t)p + 4u;
    /* the rounding of the staged rows adds at most 255 bytes */
    if ((uint64_t)n_new > (limit - 255u) / per_row) return 0;
    const uint64_t x_bytes = (uint64_t)xsz * (uint64_t)p * (uint64_t)n_new;
    const uint64_t out_off = (x_bytes + 255u) & ~(uint64_t)255u;
    *need = out_off + 4u * (uint64_t)n_new;
    return 1;
}

#endif /* CWB_NOALLOC_SIZE_H */
