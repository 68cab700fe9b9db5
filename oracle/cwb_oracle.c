/*
 * cwb_oracle.c -- plain, slow FP64 CPU oracle for componentwise boosting.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA path, and the CUDA path never calls it.
 *
 * Everything is FP64, sequential, rows visited in index order i = 0..n-1.
 * Each function states the passage of the paper (Schalk, Bischl, Ruegamer,
 * "Accelerated componentwise gradient boosting using efficient data
 * representation and momentum-based optimization", arXiv 2110.03513) that it
 * restates:
 *
 *   binning (design points, index vector)   Sec. 3.1.1
 *   binMatMat / binMatVec                    Sec. 3.1.2, Algorithm 2
 *   P-spline / linear base learners          Sec. 2.2
 *   penalised least squares, hat matrix      App. A.2, Eq. (pen-regr), Eq. (modelfit)
 *   degrees of freedom df1 = tr(H)           App. A.2, Eq. (df1)
 *   CWB                                      App. A.1, Algorithm 1
 *   ACWB and parameter aggregation           Sec. 3.2, Algorithm 3, Sec. 3.2.1
 *   HCWB                                     Sec. 3.2.3, Algorithm 4
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - index vector: closest design point, a value exactly half-way between
 *     two design points goes to the lower one (right-closed intervals);
 *   - n* = floor(sqrt(n)) when requested as "sqrt";
 *   - P-splines: n_knots interior equidistant knots on [min, max], extended
 *     by `degree` equidistant knots on each side, d = n_knots + degree + 1;
 *   - base-learner fits are penalised (Eq. pen-regr) with lambda chosen so
 *     that df1 = tr(H) equals the requested df; linear learners (1, x) are
 *     unpenalised;
 *   - SSE_k is the (weighted) residual sum of squares of the fitted learner;
 *     argmin ties go to the lowest learner index;
 *   - L2 loss L = (y-f)^2/2, offset mean(y); binomial loss with y in {0,1},
 *     L = log(1+e^f) - y f, offset logit(mean y);
 *   - ACWB: the error-corrected residual uses the previous correction fit
 *     (unscaled); eta_m = gamma * nu / theta_m with theta_m = 2/(m+1);
 *   - HCWB: ACWB on the training rows while the patience counter is below
 *     pat_0; the counter grows when the validation risk strictly increases
 *     and resets otherwise; afterwards CWB on all rows, permanently.
 *     The offset is the loss-optimal constant on the training rows.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, brute force, library routines, hand-computed recursions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENUMERIC 3

/* ------------------------------------------------------------------------ */
/* Small dense FP64 linear algebra (row-major d x d).                        */
/* ------------------------------------------------------------------------ */

/* Cholesky A = L L^T (lower); returns 0 on success, -1 if A is not positive definite. */
int orc_cholesky(const double* A, int d, double* L)
{
    memset(L, 0, sizeof(double) * (size_t)d * d);
    for (int j = 0; j < d; ++j) {
        double s = A[j * d + j];
        for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        L[j * d + j] = ljj;
        for (int i = j + 1; i < d; ++i) {
            double t = A[i * d + j];
            for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
            L[i * d + j] = t / ljj;
        }
    }
    return 0;
}

/* Solve (L L^T) x = b in place. */
static void chol_solve(const double* L, int d, double* b)
{
    for (int i = 0; i < d; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * d + k] * b[k];
        b[i] = t / L[i * d + i];
    }
    for (int i = d - 1; i >= 0; --i) {
        double t = b[i];
        for (int k = i + 1; k < d; ++k) t -= L[k * d + i] * b[k];
        b[i] = t / L[i * d + i];
    }
}

/* Inverse of a symmetric positive definite matrix via Cholesky. */
int orc_spd_inverse(const double* A, int d, double* Ainv)
{
    double* L = (double*)malloc(sizeof(double) * (size_t)d * d);
    double* col = (double*)malloc(sizeof(double) * (size_t)d);
    if (!L || !col) { free(L); free(col); return ORC_ENOMEM; }
    if (orc_cholesky(A, d, L) != 0) { free(L); free(col); return ORC_ENUMERIC; }
    for (int j = 0; j < d; ++j) {
        for (int i = 0; i < d; ++i) col[i] = (i == j) ? 1.0 : 0.0;
        chol_solve(L, d, col);
        for (int i = 0; i < d; ++i) Ainv[i * d + j] = col[i];
    }
    free(L); free(col);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Binning, Sec. 3.1.1.                                                      */
/* ------------------------------------------------------------------------ */

/* floor(sqrt(n)) computed on integers (the n* = sqrt(n) rule of Sec. 3.1.1). */
int64_t orc_isqrt(int64_t n)
{
    int64_t s = (int64_t)sqrt((double)n);
    while (s > 0 && s * s > n) --s;
    while ((s + 1) * (s + 1) <= n) ++s;
    return s;
}

/* Equidistant design points z_l = xmin + l (xmax - xmin)/(n*-1), l = 0..n*-1,
 * and the index vector: each x goes to its closest design point; a value
 * exactly half-way between two points goes to the lower one.  With
 * t = (x - xmin)/h the closest point with that tie rule is ceil(t - 1/2). */
int orc_bin_equidistant(const double* x, int64_t n, int32_t nstar, double xmin, double xmax,
                        int32_t* ind, double* z)
{
    if (nstar < 2 || !(xmax > xmin)) return ORC_EINVAL;
    double h = (xmax - xmin) / (double)(nstar - 1);
    for (int32_t l = 0; l < nstar && z; ++l) z[l] = xmin + (double)l * h;
    for (int64_t i = 0; i < n; ++i) {
        double t = (x[i] - xmin) / h;
        double l = ceil(t - 0.5);
        if (l < 0.0) l = 0.0;
        if (l > (double)(nstar - 1)) l = (double)(nstar - 1);
        ind[i] = (int32_t)l;
    }
    return ORC_OK;
}

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Exact binning: the design points are the sorted unique values of x, so every
 * value sits exactly on its design point.  Writes z (capacity n) and ind;
 * returns the number of unique values through *nstar. */
int orc_bin_exact(const double* x, int64_t n, double* z, int32_t* ind, int32_t* nstar)
{
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!s) return ORC_ENOMEM;
    memcpy(s, x, sizeof(double) * (size_t)n);
    qsort(s, (size_t)n, sizeof(double), cmp_double);
    int64_t u = 0;
    for (int64_t i = 0; i < n; ++i)
        if (u == 0 || s[i] != z[u - 1]) z[u++] = s[i];
    for (int64_t i = 0; i < n; ++i) {
        int64_t lo = 0, hi = u - 1;
        while (lo < hi) {                 /* first z >= x[i] */
            int64_t mid = (lo + hi) / 2;
            if (z[mid] < x[i]) lo = mid + 1; else hi = mid;
        }
        ind[i] = (int32_t)lo;
    }
    *nstar = (int32_t)u;
    free(s);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Base-learner representations, Sec. 2.2.                                   */
/* ------------------------------------------------------------------------ */

/* All d = n_knots + degree + 1 B-spline basis functions at x, by the Cox-de Boor
 * recursion (the definition) on the equidistant knot vector
 *   t_i = xmin + (i - degree) * (xmax - xmin)/(n_knots + 1),  i = 0 .. n_knots + 2 degree + 1,
 * with half-open order-0 indicators [t_i, t_{i+1}). */
int orc_bspline_basis(const double* x, int64_t m, double xmin, double xmax, int32_t degree,
                      int32_t n_knots, double* out /* m x d */)
{
    int q = degree;
    int nt = n_knots + 2 * q + 2;
    int d = n_knots + q + 1;
    if (q < 0 || n_knots < 0 || !(xmax > xmin)) return ORC_EINVAL;
    double* t = (double*)malloc(sizeof(double) * (size_t)nt);
    double* B = (double*)malloc(sizeof(double) * (size_t)nt);
    if (!t || !B) { free(t); free(B); return ORC_ENOMEM; }
    double delta = (xmax - xmin) / (double)(n_knots + 1);
    for (int i = 0; i < nt; ++i) t[i] = xmin + (double)(i - q) * delta;
    for (int64_t r = 0; r < m; ++r) {
        double xv = x[r];
        for (int i = 0; i < nt - 1; ++i) B[i] = (t[i] <= xv && xv < t[i + 1]) ? 1.0 : 0.0;
        for (int deg = 1; deg <= q; ++deg) {
            for (int i = 0; i < nt - 1 - deg; ++i) {
                double a = (xv - t[i]) / (t[i + deg] - t[i]);
                double b = (t[i + deg + 1] - xv) / (t[i + deg + 1] - t[i + 1]);
                B[i] = a * B[i] + b * B[i + 1];
            }
        }
        for (int j = 0; j < d; ++j) out[r * d + j] = B[j];
    }
    free(t); free(B);
    return ORC_OK;
}

/* Linear base learner on one feature: g(x) = (1, x). */
void orc_linear_basis(const double* x, int64_t m, double* out /* m x 2 */)
{
    for (int64_t r = 0; r < m; ++r) { out[2 * r] = 1.0; out[2 * r + 1] = x[r]; }
}

/* Difference penalty K = D^T D with D the order-`order` difference matrix
 * ((d - order) x d), App. A.2 (rows (1, -2, 1) for order 2). */
int orc_penalty(int32_t d, int32_t order, double* K /* d x d */)
{
    if (order < 0 || order >= d) return ORC_EINVAL;
    /* D starts as the identity and is differenced `order` times. */
    double* D = (double*)calloc((size_t)d * d, sizeof(double));
    if (!D) return ORC_ENOMEM;
    for (int i = 0; i < d; ++i) D[i * d + i] = 1.0;
    int rows = d;
    for (int o = 0; o < order; ++o) {
        for (int i = 0; i < rows - 1; ++i)
            for (int j = 0; j < d; ++j) D[i * d + j] = D[(i + 1) * d + j] - D[i * d + j];
        rows -= 1;
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int i = 0; i < rows; ++i) s += D[i * d + a] * D[i * d + b];
            K[a * d + b] = s;
        }
    free(D);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: binMatMat and binMatVec.                                     */
/* ------------------------------------------------------------------------ */

/* binMatVec, first half: u_l = sum over rows i (in `rows` if given) with ind_i = l of w_i r_i. */
void orc_bin_matvec_u(const int32_t* ind, int64_t n, const double* w, const double* r,
                      const uint8_t* rows, int32_t nstar, double* u)
{
    for (int32_t l = 0; l < nstar; ++l) u[l] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (rows && !rows[i]) continue;
        u[ind[i]] += (w ? w[i] : 1.0) * r[i];
    }
}

/* binMatVec: returns Zb^T u (d values). */
void orc_bin_matvec(const int32_t* ind, int64_t n, const double* w, const double* r,
                    const uint8_t* rows, int32_t nstar, const double* Zb, int32_t d, double* out)
{
    double* u = (double*)malloc(sizeof(double) * (size_t)nstar);
    orc_bin_matvec_u(ind, n, w, r, rows, nstar, u);
    for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int32_t l = 0; l < nstar; ++l) s += Zb[(int64_t)l * d + j] * u[l];
        out[j] = s;
    }
    free(u);
}

/* binMatMat: U (d x n*) with column ind_i accumulating w_i Zb(ind_i)^T, returns U Zb (d x d). */
void orc_bin_matmat(const int32_t* ind, int64_t n, const double* w, const uint8_t* rows,
                    int32_t nstar, const double* Zb, int32_t d, double* out)
{
    double* U = (double*)calloc((size_t)d * nstar, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        if (rows && !rows[i]) continue;
        double wi = w ? w[i] : 1.0;
        for (int j = 0; j < d; ++j) U[(int64_t)j * nstar + ind[i]] += wi * Zb[(int64_t)ind[i] * d + j];
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int32_t l = 0; l < nstar; ++l) s += U[(int64_t)a * nstar + l] * Zb[(int64_t)l * d + b];
            out[a * d + b] = s;
        }
    free(U);
}

/* ------------------------------------------------------------------------ */
/* Degrees of freedom and smoothing parameter, App. A.2.                     */
/* ------------------------------------------------------------------------ */

/* df1(lambda) = tr(H(lambda)) = tr((G + lambda K)^{-1} G) (cyclic trace of Eq. (modelfit)). */
int orc_df1(const double* G, const double* K, int32_t d, double lambda, double* df)
{
    double* A = (double*)malloc(sizeof(double) * (size_t)d * d);
    double* L = (double*)malloc(sizeof(double) * (size_t)d * d);
    double* col = (double*)malloc(sizeof(double) * (size_t)d);
    if (!A || !L || !col) { free(A); free(L); free(col); return ORC_ENOMEM; }
    for (int i = 0; i < d * d; ++i) A[i] = G[i] + lambda * K[i];
    if (orc_cholesky(A, d, L) != 0) { free(A); free(L); free(col); return ORC_ENUMERIC; }
    double tr = 0.0;
    for (int j = 0; j < d; ++j) {
        for (int i = 0; i < d; ++i) col[i] = G[i * d + j];
        chol_solve(L, d, col);
        tr += col[j];
    }
    *df = tr;
    free(A); free(L); free(col);
    return ORC_OK;
}

/* lambda >= 0 with df1(lambda) = df, by bisection on log(lambda) (a plain root
 * search on the monotone map lambda -> df1; every evaluation is a fresh
 * factorisation).  df >= df1(0) gives lambda = 0. */
int orc_lambda_for_df(const double* G, const double* K, int32_t d, double df, double* lambda)
{
    double v;
    int st;
    /* lambda = 0: unpenalised. */
    st = orc_df1(G, K, d, 0.0, &v);
    if (st == ORC_OK && df >= v) { *lambda = 0.0; return ORC_OK; }
    /* bracket log10(lambda) within 12 decades of the scale tr(G)/tr(K) */
    double trg = 0.0, trk = 0.0;
    for (int i = 0; i < d; ++i) { trg += G[i * d + i]; trk += K[i * d + i]; }
    if (!(trg > 0.0) || !(trk > 0.0)) return ORC_ENUMERIC;
    double c = log10(trg / trk);
    double lo = c - 12.0, hi = c + 12.0;
    st = orc_df1(G, K, d, pow(10.0, lo), &v);
    if (st != ORC_OK) return st;
    if (v < df) { *lambda = pow(10.0, lo); return ORC_OK; }
    st = orc_df1(G, K, d, pow(10.0, hi), &v);
    if (st != ORC_OK) return st;
    if (v > df) return ORC_ENUMERIC;      /* df at or below the penalty's null-space dimension */
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        st = orc_df1(G, K, d, pow(10.0, mid), &v);
        if (st != ORC_OK) return st;
        if (v > df) lo = mid; else hi = mid;
        if (hi - lo < 1e-15) break;
    }
    *lambda = pow(10.0, 0.5 * (lo + hi));
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Losses (Sec. 2.1 / 2.3).                                                   */
/* ------------------------------------------------------------------------ */

#define LOSS_L2 0
#define LOSS_BINOMIAL 1

static double loss_value(int loss, double y, double f)
{
    if (loss == LOSS_L2) return 0.5 * (y - f) * (y - f);
    /* log(1 + e^f) - y f, written to avoid overflow for large |f| */
    double lse = (f > 0.0) ? f + log1p(exp(-f)) : log1p(exp(f));
    return lse - y * f;
}

/* Pseudo residual r = -dL/df. */
static double pseudo_residual(int loss, double y, double f)
{
    if (loss == LOSS_L2) return y - f;
    return y - 1.0 / (1.0 + exp(-f));
}

/* Loss-optimal constant over the rows in `rows` (all if NULL). */
int orc_offset(int loss, const double* y, const double* w, const uint8_t* rows, int64_t n, double* offset)
{
    double sw = 0.0, swy = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (rows && !rows[i]) continue;
        double wi = w ? w[i] : 1.0;
        sw += wi; swy += wi * y[i];
    }
    if (!(sw > 0.0)) return ORC_EINVAL;
    double ybar = swy / sw;
    if (loss == LOSS_L2) { *offset = ybar; return ORC_OK; }
    if (!(ybar > 0.0 && ybar < 1.0)) return ORC_EINVAL;
    *offset = log(ybar / (1.0 - ybar));
    return ORC_OK;
}

/* Derivative exposed for the finite-difference pin. */
double orc_loss(int loss, double y, double f) { return loss_value(loss, y, f); }
double orc_pseudo_residual(int loss, double y, double f) { return pseudo_residual(loss, y, f); }

/* ------------------------------------------------------------------------ */
/* Boosting: Algorithms 1, 3, 4.                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t type;        /* 0: P-spline, 1: linear, 2: categorical ridge, 3: categorical binary (App. B.1) */
    int32_t feature;
    int32_t degree;
    int32_t n_knots;     /* categorical: number of classes c; the feature holds the codes 0..c-1 */
    int32_t diff_order;
    double df;           /* > 0: choose lambda so that df1 = df */
    double lambda;       /* used when df <= 0 */
    int32_t n_bins;      /* 0: exact (unique values), -1: floor(sqrt n), -2: unbinned (dense), >1: explicit */
    int32_t level;       /* categorical binary: the class the learner indicates, 0 <= level < c */
} orc_learner;

typedef struct {
    int32_t loss;        /* 0 L2, 1 binomial */
    int32_t opt;         /* 0 CWB, 1 ACWB, 2 HCWB */
    double nu;
    double gamma;
    int32_t iterations;
    int32_t patience;
    int32_t use_offset;  /* nonzero: start from `offset` instead of the loss-optimal constant */
    double offset;
} orc_config;

typedef struct {
    double offset;
    int32_t dmax;
    int32_t switch_iter;     /* HCWB: first CWB iteration (1-based), 0 if never switched */
    double* theta_f;         /* K x dmax, primary model's aggregated coefficients */
    double* theta_h;         /* K x dmax or NULL, momentum model's aggregated coefficients */
    double* f;               /* n, fitted primary model */
    int32_t* k_sel;          /* M */
    int32_t* k_cor;          /* M or NULL (-1 where no correction fit ran) */
    double* sse_best;        /* M or NULL */
    double* sse_second;      /* M or NULL */
    double* sse_best_cor;    /* M or NULL */
    double* sse_second_cor;  /* M or NULL */
    double* val_risk;        /* M or NULL (NaN where not evaluated) */
    double* lambda;          /* K or NULL: lambda on the fitting rows of the first phase */
    double* lambda_full;     /* K or NULL: lambda on all rows (HCWB second phase) */
    int32_t* nstar;          /* K or NULL */
    int32_t* forced_k;       /* M or NULL: if non-NULL and >= 0, overrides the selected learner */
} orc_result;

typedef struct {
    int d;
    int dense;               /* unbinned: Z is n x d */
    int32_t nstar;
    double xmin, xmax;
    int32_t* ind;            /* n */
    double* Zb;              /* nstar x d (binned) or n x d (dense) */
    double* K;               /* d x d */
    double lam[2];
    double* G[2];
    double* P[2];
} bl_state;

static int learner_d(const orc_learner* b)
{
    if (b->type == 2) return b->n_knots;            /* one coefficient per class */
    if (b->type == 3) return 1;                     /* one coefficient for one class */
    return b->type == 1 ? 2 : b->n_knots + b->degree + 1;
}

static void free_state(bl_state* s)
{
    free(s->ind); free(s->Zb); free(s->K);
    for (int a = 0; a < 2; ++a) { free(s->G[a]); free(s->P[a]); }
}

/* Design of one learner: binning + reduced design (or dense design). */
static int setup_design(const orc_learner* b, const double* x, int64_t n, bl_state* s)
{
    int d = learner_d(b);
    s->d = d;
    double xmin = x[0], xmax = x[0];
    for (int64_t i = 1; i < n; ++i) { if (x[i] < xmin) xmin = x[i]; if (x[i] > xmax) xmax = x[i]; }
    if (!(xmax > xmin)) return ORC_EINVAL;
    s->xmin = xmin; s->xmax = xmax;
    s->ind = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!s->ind) return ORC_ENOMEM;
    if (b->type == 2 || b->type == 3) {
        /* categorical learners: the values are class codes 0..c-1 and each class is one bin, so
           the lookup k_i is the code itself.  Ridge: the design is the dummy matrix (identity on
           the bins) and the penalty the identity.  Binary: one column, the indicator of `level`,
           unpenalised. */
        const int c = b->n_knots;
        if (c < 2 || (b->type == 3 && (b->level < 0 || b->level >= c))) return ORC_EINVAL;
        for (int64_t i = 0; i < n; ++i) {
            if (!(x[i] >= 0.0 && x[i] < (double)c && x[i] == floor(x[i]))) return ORC_EINVAL;
            s->ind[i] = (int32_t)x[i];
        }
        s->nstar = c;
        s->Zb = (double*)calloc((size_t)c * d, sizeof(double));
        s->K = (double*)calloc((size_t)d * d, sizeof(double));
        if (!s->Zb || !s->K) return ORC_ENOMEM;
        if (b->type == 2) {
            for (int j = 0; j < c; ++j) {
                s->Zb[(int64_t)j * c + j] = 1.0;
                s->K[(int64_t)j * c + j] = 1.0;
            }
        } else {
            s->Zb[b->level] = 1.0;
        }
        return ORC_OK;
    }
    double* pts;
    int64_t npts;
    if (b->n_bins == -2) {
        s->dense = 1;
        pts = (double*)malloc(sizeof(double) * (size_t)n);
        memcpy(pts, x, sizeof(double) * (size_t)n);
        npts = n;
        for (int64_t i = 0; i < n; ++i) s->ind[i] = (int32_t)i;
        s->nstar = (int32_t)n;
    } else if (b->n_bins == 0) {
        pts = (double*)malloc(sizeof(double) * (size_t)n);
        int32_t ns = 0;
        int st = orc_bin_exact(x, n, pts, s->ind, &ns);
        if (st) { free(pts); return st; }
        s->nstar = ns; npts = ns;
    } else {
        int64_t ns = b->n_bins == -1 ? orc_isqrt(n) : b->n_bins;
        if (ns < 2) return ORC_EINVAL;
        pts = (double*)malloc(sizeof(double) * (size_t)ns);
        int st = orc_bin_equidistant(x, n, (int32_t)ns, xmin, xmax, s->ind, pts);
        if (st) { free(pts); return st; }
        s->nstar = (int32_t)ns; npts = ns;
    }
    s->Zb = (double*)malloc(sizeof(double) * (size_t)npts * d);
    s->K = (double*)calloc((size_t)d * d, sizeof(double));
    if (!s->Zb || !s->K) { free(pts); return ORC_ENOMEM; }
    if (b->type == 1) {
        orc_linear_basis(pts, npts, s->Zb);
    } else {
        int st = orc_bspline_basis(pts, npts, xmin, xmax, b->degree, b->n_knots, s->Zb);
        if (st) { free(pts); return st; }
        st = orc_penalty(d, b->diff_order, s->K);
        if (st) { free(pts); return st; }
    }
    free(pts);
    return ORC_OK;
}

/* G = Z^T W Z over the rows in `rows`, lambda and P = (G + lambda K)^{-1} for phase a. */
static int setup_phase(const orc_learner* b, bl_state* s, int64_t n, const double* w,
                       const uint8_t* rows, int a)
{
    int d = s->d;
    s->G[a] = (double*)malloc(sizeof(double) * (size_t)d * d);
    s->P[a] = (double*)malloc(sizeof(double) * (size_t)d * d);
    if (!s->G[a] || !s->P[a]) return ORC_ENOMEM;
    orc_bin_matmat(s->ind, n, w, rows, s->nstar, s->Zb, d, s->G[a]);
    double lam = 0.0;
    if (b->type == 0 || b->type == 2) {             /* penalised learners */
        if (b->df > 0.0) {
            int st = orc_lambda_for_df(s->G[a], s->K, d, b->df, &lam);
            if (st) return st;
        } else {
            lam = b->lambda;
        }
    }
    s->lam[a] = lam;
    double* A = (double*)malloc(sizeof(double) * (size_t)d * d);
    for (int i = 0; i < d * d; ++i) A[i] = s->G[a][i] + lam * s->K[i];
    int st = orc_spd_inverse(A, d, s->P[a]);
    free(A);
    return st;
}

/* Fitted learner values at row i. */
static double learner_value(const bl_state* s, int64_t i, const double* theta)
{
    const double* z = s->Zb + (int64_t)s->ind[i] * s->d;
    double v = 0.0;
    for (int j = 0; j < s->d; ++j) v += z[j] * theta[j];
    return v;
}

/* Threads of the learner loop in find_best (1 unless orc_set_threads asks for more; without
 * OpenMP the loop runs on one thread whatever is asked). */
static int orc_threads = 1;

int orc_set_threads(int t)
{
    orc_threads = t < 1 ? 1 : t;
#ifdef _OPENMP
    return orc_threads;
#else
    return 1;
#endif
}

/* findBestBaselearner (Algorithm 1, inner loop; Sec. 3.2): fit every learner to
 * r on the rows in `rows` by penalised least squares, theta_k = P_k Z_k^T W r,
 * compute SSE_k by its definition and return the argmin (ties: lowest k). */
static void find_best(int32_t K, bl_state* S, int a, int64_t n, const double* w, const uint8_t* rows,
                      const double* r, double* theta_all /* K x dmax */, int dmax,
                      int32_t* k_best, double* sse1, double* sse2, int32_t forced)
{
    double best = INFINITY, second = INFINITY;
    int32_t kb = -1;
    double* sse_all = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    /* The learners' fits are independent: with OpenMP they run on several threads, each learner's
     * sums still in row order, so every theta_k and SSE_k is the same as on one thread. */
#pragma omp parallel num_threads(orc_threads)
    {
        double* s_vec = (double*)malloc(sizeof(double) * (size_t)dmax);
#pragma omp for schedule(dynamic, 1)
        for (int32_t k = 0; k < K; ++k) {
            bl_state* s = &S[k];
            int d = s->d;
            orc_bin_matvec(s->ind, n, w, r, rows, s->nstar, s->Zb, d, s_vec);
            double* th = theta_all + (int64_t)k * dmax;
            for (int i = 0; i < dmax; ++i) th[i] = 0.0;
            for (int i = 0; i < d; ++i) {
                double t = 0.0;
                for (int j = 0; j < d; ++j) t += s->P[a][i * d + j] * s_vec[j];
                th[i] = t;
            }
            double sse = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (rows && !rows[i]) continue;
                double e = r[i] - learner_value(s, i, th);
                sse += (w ? w[i] : 1.0) * e * e;
            }
            sse_all[k] = sse;
        }
        free(s_vec);
    }
    /* the argmin in learner order (ties: lowest k) */
    for (int32_t k = 0; k < K; ++k) {
        const double sse = sse_all[k];
        if (sse < best) { second = best; best = sse; kb = k; }
        else if (sse < second) { second = sse; }
    }
    free(sse_all);
    if (forced >= 0 && forced < K) kb = forced;
    *k_best = kb;
    if (sse1) *sse1 = best;
    if (sse2) *sse2 = second;
}

int orc_fit(int64_t n, int32_t p, const double* X /* p x n */, const double* y, const double* w,
            const uint8_t* val_mask, int32_t K, const orc_learner* bl, const orc_config* cfg,
            orc_result* res)
{
    if (n < 2 || p < 1 || K < 1 || !cfg || cfg->iterations < 0) return ORC_EINVAL;
    if (cfg->opt == 2 && !val_mask) return ORC_EINVAL;
    int hybrid = cfg->opt == 2 && val_mask != NULL;
    int accel = cfg->opt == 1 || cfg->opt == 2;
    uint8_t* train = NULL;          /* fitting rows of the first phase (NULL = all) */
    if (hybrid) {
        train = (uint8_t*)malloc((size_t)n);
        int64_t ntr = 0, nval = 0;
        for (int64_t i = 0; i < n; ++i) { train[i] = val_mask[i] ? 0 : 1; ntr += train[i]; }
        nval = n - ntr;
        if (ntr < 2 || nval < 1) { free(train); return ORC_EINVAL; }
    }
    int dmax = 0;
    for (int32_t k = 0; k < K; ++k) {
        if (bl[k].feature < 0 || bl[k].feature >= p || bl[k].type < 0 || bl[k].type > 3) {
            free(train);
            return ORC_EINVAL;
        }
        int d = learner_d(&bl[k]);
        if (d > dmax) dmax = d;
    }
    res->dmax = dmax;
    bl_state* S = (bl_state*)calloc((size_t)K, sizeof(bl_state));
    int st = ORC_OK;
    for (int32_t k = 0; k < K && st == ORC_OK; ++k) {
        st = setup_design(&bl[k], X + (int64_t)bl[k].feature * n, n, &S[k]);
        if (st == ORC_OK) st = setup_phase(&bl[k], &S[k], n, w, train, 0);
        if (st == ORC_OK && hybrid) st = setup_phase(&bl[k], &S[k], n, w, NULL, 1);
        if (st == ORC_OK) {
            if (res->lambda) res->lambda[k] = S[k].lam[0];
            if (res->lambda_full) res->lambda_full[k] = hybrid ? S[k].lam[1] : S[k].lam[0];
            if (res->nstar) res->nstar[k] = S[k].nstar;
        }
    }
    double offset = 0.0;
    if (st == ORC_OK) {
        if (cfg->use_offset) offset = cfg->offset;
        else st = orc_offset(cfg->loss, y, w, train, n, &offset);
    }
    if (st != ORC_OK) {
        for (int32_t k = 0; k < K; ++k) free_state(&S[k]);
        free(S); free(train);
        return st;
    }
    res->offset = offset;
    res->switch_iter = 0;

    double* f = res->f;
    double* h = (double*)malloc(sizeof(double) * (size_t)n);
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* c = (double*)malloc(sizeof(double) * (size_t)n);
    double* bcor = (double*)malloc(sizeof(double) * (size_t)n);   /* previous correction fit */
    double* theta_all = (double*)malloc(sizeof(double) * (size_t)K * dmax);
    double* theta_cor = (double*)malloc(sizeof(double) * (size_t)K * dmax);
    double* th_h = (double*)calloc((size_t)K * dmax, sizeof(double));
    for (int64_t i = 0; i < n; ++i) { f[i] = offset; h[i] = offset; g[i] = offset; }
    for (int64_t i = 0; i < (int64_t)K * dmax; ++i) res->theta_f[i] = 0.0;

    int32_t counter = 0;
    int switched = 0;
    double risk_prev = 0.0;
    if (hybrid) {                     /* validation risk of the offset model */
        double s = 0.0; int64_t nv = 0;
        for (int64_t i = 0; i < n; ++i) if (val_mask[i]) { s += loss_value(cfg->loss, y[i], f[i]); ++nv; }
        risk_prev = s / (double)nv;
    }

    for (int32_t m = 1; m <= cfg->iterations; ++m) {
        int32_t forced = res->forced_k ? res->forced_k[m - 1] : -1;
        int do_accel = accel && !(hybrid && counter >= cfg->patience);
        if (hybrid && !do_accel && !switched) { switched = 1; res->switch_iter = m; }
        if (res->val_risk) res->val_risk[m - 1] = NAN;
        if (!do_accel) {
            /* CWB step (Algorithm 1) on all rows; phase 1 cache after an HCWB switch. */
            int a = (hybrid && switched) ? 1 : 0;
            for (int64_t i = 0; i < n; ++i) r[i] = pseudo_residual(cfg->loss, y[i], f[i]);
            int32_t kb;
            double s1, s2;
            find_best(K, S, a, n, w, NULL, r, theta_all, dmax, &kb, &s1, &s2, forced);
            const double* th = theta_all + (int64_t)kb * dmax;
            for (int64_t i = 0; i < n; ++i) f[i] += cfg->nu * learner_value(&S[kb], i, th);
            for (int j = 0; j < dmax; ++j) res->theta_f[(int64_t)kb * dmax + j] += cfg->nu * th[j];
            res->k_sel[m - 1] = kb;
            if (res->k_cor) res->k_cor[m - 1] = -1;
            if (res->sse_best) res->sse_best[m - 1] = s1;
            if (res->sse_second) res->sse_second[m - 1] = s2;
            if (res->sse_best_cor) res->sse_best_cor[m - 1] = NAN;
            if (res->sse_second_cor) res->sse_second_cor[m - 1] = NAN;
            continue;
        }
        /* ACWB step (Algorithm 3), fits on the training rows, models updated on all rows. */
        double th_m = 2.0 / ((double)m + 1.0);
        for (int64_t i = 0; i < n; ++i) g[i] = (1.0 - th_m) * f[i] + th_m * h[i];
        for (int64_t i = 0; i < n; ++i) r[i] = pseudo_residual(cfg->loss, y[i], g[i]);
        int32_t kb, kc;
        double s1, s2, c1, c2;
        find_best(K, S, 0, n, w, train, r, theta_all, dmax, &kb, &s1, &s2, forced);
        const double* th = theta_all + (int64_t)kb * dmax;
        for (int64_t i = 0; i < n; ++i) f[i] = g[i] + cfg->nu * learner_value(&S[kb], i, th);
        if (m == 1) {
            for (int64_t i = 0; i < n; ++i) c[i] = r[i];
        } else {
            double a = (double)m / ((double)m + 1.0);
            for (int64_t i = 0; i < n; ++i) c[i] = r[i] + a * (c[i] - bcor[i]);
        }
        find_best(K, S, 0, n, w, train, c, theta_cor, dmax, &kc, &c1, &c2, -1);
        const double* thc = theta_cor + (int64_t)kc * dmax;
        double eta = cfg->gamma * cfg->nu / th_m;
        for (int64_t i = 0; i < n; ++i) {
            bcor[i] = learner_value(&S[kc], i, thc);
            h[i] += eta * bcor[i];
        }
        /* parameter aggregation, Sec. 3.2.1 */
        for (int64_t q = 0; q < (int64_t)K * dmax; ++q)
            res->theta_f[q] = (1.0 - th_m) * res->theta_f[q] + th_m * th_h[q];
        for (int j = 0; j < dmax; ++j) {
            res->theta_f[(int64_t)kb * dmax + j] += cfg->nu * th[j];
            th_h[(int64_t)kc * dmax + j] += eta * thc[j];
        }
        res->k_sel[m - 1] = kb;
        if (res->k_cor) res->k_cor[m - 1] = kc;
        if (res->sse_best) res->sse_best[m - 1] = s1;
        if (res->sse_second) res->sse_second[m - 1] = s2;
        if (res->sse_best_cor) res->sse_best_cor[m - 1] = c1;
        if (res->sse_second_cor) res->sse_second_cor[m - 1] = c2;
        if (hybrid) {               /* Algorithm 4: patience on the validation risk */
            double s = 0.0; int64_t nv = 0;
            for (int64_t i = 0; i < n; ++i) if (val_mask[i]) { s += loss_value(cfg->loss, y[i], f[i]); ++nv; }
            double risk = s / (double)nv;
            if (res->val_risk) res->val_risk[m - 1] = risk;
            if (risk > risk_prev) counter += 1; else counter = 0;
            risk_prev = risk;
        }
    }
    if (res->theta_h) memcpy(res->theta_h, th_h, sizeof(double) * (size_t)K * dmax);

    free(h); free(g); free(r); free(c); free(bcor); free(theta_all); free(theta_cor); free(th_h);
    for (int32_t k = 0; k < K; ++k) free_state(&S[k]);
    free(S); free(train);
    return ORC_OK;
}

/* Prediction of a fitted additive model at new points: offset + sum_k g_k(x)^T theta_k,
 * x clamped to the learner's training range (Sec. 2.3, aggregated coefficients). */
int orc_predict(int64_t n_new, int32_t p, const double* Xnew /* p x n_new */, int32_t K,
                const orc_learner* bl, const double* xmin, const double* xmax,
                const double* theta /* K x dmax */, int32_t dmax, double offset, double* out)
{
    for (int64_t i = 0; i < n_new; ++i) out[i] = offset;
    double* row = (double*)malloc(sizeof(double) * (size_t)(dmax > 2 ? dmax : 2));
    for (int32_t k = 0; k < K; ++k) {
        if (bl[k].feature < 0 || bl[k].feature >= p) { free(row); return ORC_EINVAL; }
        int d = learner_d(&bl[k]);
        for (int64_t i = 0; i < n_new; ++i) {
            double x = Xnew[(int64_t)bl[k].feature * n_new + i];
            if (bl[k].type == 2 || bl[k].type == 3) {
                /* a valid class code contributes its coefficient, anything else (an unknown
                   code, a non-integer) nothing */
                if (x >= 0.0 && x < (double)bl[k].n_knots && x == floor(x)) {
                    if (bl[k].type == 2) out[i] += theta[(int64_t)k * dmax + (int64_t)x];
                    else if ((int32_t)x == bl[k].level) out[i] += theta[(int64_t)k * dmax];
                }
                continue;
            }
            if (x < xmin[k]) x = xmin[k];
            if (x > xmax[k]) x = xmax[k];
            if (bl[k].type == 1) orc_linear_basis(&x, 1, row);
            else orc_bspline_basis(&x, 1, xmin[k], xmax[k], bl[k].degree, bl[k].n_knots, row);
            double v = 0.0;
            for (int j = 0; j < d; ++j) v += row[j] * theta[(int64_t)k * dmax + j];
            out[i] += v;
        }
    }
    free(row);
    return ORC_OK;
}
