// cwb_bspline.cuh -- the one device evaluator of the B-spline basis, shared by the setup (the
// reduced design Z^b at the design points) and prediction (the basis at new x).
#pragma once

#include "cwb_internal.cuh"

namespace cwb {
namespace {

// B-spline basis on an equidistant extended knot vector (Sec. 2.2, P-splines).  Knots
// t_i = xmin + (i - q) delta, delta = (xmax - xmin) / (n_knots + 1).  The q + 1 non-zero functions
// on the knot interval holding x come from the triangular form of the Cox-de Boor recursion;
// returns the first non-zero column.  Degrees 1..3; x must lie in [xmin, xmax].
__device__ __forceinline__ double knot_at(double xmin, double delta, int i_minus_q)
{
    return __dadd_rn(xmin, __dmul_rn((double)i_minus_q, delta));
}

__device__ int bspline_nonzero(double x, double xmin, double xmax, int q, int nk, double* N /* q+1 */)
{
    const double delta = __ddiv_rn(__dsub_rn(xmax, xmin), (double)(nk + 1));
    const int last = nk + q;                      // last interval with a full set of functions: [t_last, t_last+1]
    int mu = (int)floor(__ddiv_rn(__dsub_rn(x, xmin), delta)) + q;
    if (mu < q) mu = q;
    if (mu > last) mu = last;
    // agree with the half-open rule t_mu <= x < t_mu+1 on the rounded knot values
    while (mu > q && x < knot_at(xmin, delta, mu - q)) --mu;
    while (mu < last && x >= knot_at(xmin, delta, mu + 1 - q)) ++mu;
    double left[kMaxNnz], right[kMaxNnz];
    N[0] = 1.0;
    for (int j = 1; j <= q; ++j) {
        left[j] = x - knot_at(xmin, delta, mu + 1 - j - q);
        right[j] = knot_at(xmin, delta, mu + j - q) - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double tmp = N[r] / (right[r + 1] + left[j - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
    }
    return mu - q;
}

}  // namespace
}  // namespace cwb
