"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute force,
a library routine (scipy's B-splines, numpy dense algebra), a closed form, a
hand-computed worked example, or an identity the paper states.  A plausible
slip in the oracle (a dropped term, a wrong index, a transposed operand, a
wrong tie rule) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- binning (Sec. 3.1.1)

def test_isqrt_matches_integer_sqrt():
    for n in list(range(0, 2000)) + [10**6, 2 * 10**6, 2**53 - 1, 999_999, 1_000_001]:
        assert O.isqrt(n) == math.isqrt(n)


def _brute_nearest(x, z):
    """Closest design point by exhaustive search; ties go to the lower point."""
    out = np.empty(x.size, dtype=np.int64)
    for i, v in enumerate(x):
        dist = np.abs(v - z)
        best = dist.min()
        out[i] = int(np.flatnonzero(dist == best)[0])
    return out


def test_binning_brute_force_with_exact_midpoints():
    nstar = 9
    z = np.arange(nstar, dtype=np.float64)          # xmin = 0, xmax = 8 -> h = 1 exactly
    x = np.concatenate([z, z[:-1] + 0.5, [0.25, 7.75, 3.4999, 3.5001, 0.0, 8.0]])
    ind, zo = O.bin_equidistant(x, nstar, 0.0, 8.0)
    np.testing.assert_array_equal(zo, z)
    np.testing.assert_array_equal(ind, _brute_nearest(x, z))
    # half-way values go to the lower design point
    assert ind[nstar + 2] == 2 and ind[nstar] == 0


def test_binning_random_against_brute_force():
    rng = np.random.default_rng(5)
    for nstar in (2, 3, 17, 100):
        x = rng.normal(size=500) * 3 + 1
        ind, z = O.bin_equidistant(x, nstar)
        assert z[0] == x.min() and abs(z[-1] - x.max()) < 1e-12
        np.testing.assert_array_equal(ind, _brute_nearest(x, z))
        assert ind[np.argmin(x)] == 0 and ind[np.argmax(x)] == nstar - 1


def test_exact_binning_matches_unique():
    rng = np.random.default_rng(6)
    x = rng.integers(0, 50, size=400).astype(np.float64) * 0.37
    ind, z = O.bin_exact(x)
    np.testing.assert_array_equal(z, np.unique(x))
    np.testing.assert_array_equal(z[ind], x)


# --------------------------------------------------------------- basis (Sec. 2.2)

def test_bspline_matches_scipy_design_matrix():
    from scipy.interpolate import BSpline
    xmin, xmax, q, nk = -1.3, 2.9, 3, 20
    delta = (xmax - xmin) / (nk + 1)
    t = xmin + (np.arange(nk + 2 * q + 2) - q) * delta
    x = np.linspace(xmin, xmax - 1e-9, 301)
    ref = BSpline.design_matrix(x, t, q).toarray()
    got = O.bspline_basis(x, xmin, xmax, q, nk)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_bspline_partition_of_unity_and_support():
    x = np.linspace(0.0, 1.0, 1001)
    B = O.bspline_basis(x, 0.0, 1.0, 3, 20)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-13)
    assert ((B > 1e-15).sum(1) <= 4).all()
    assert (B >= -1e-15).all()


def test_uniform_cubic_textbook_pieces():
    # inside one knot interval at local position s the four non-zero uniform cubic
    # B-splines are (1-s)^3/6, (3s^3-6s^2+4)/6, (-3s^3+3s^2+3s+1)/6, s^3/6
    nk, q = 20, 3
    delta = 1.0 / (nk + 1)
    for s in (0.0, 0.3, 0.5, 0.9):
        j = 7                                   # interval [t_{j+q}, t_{j+q+1})
        x = j * delta + s * delta
        row = O.bspline_basis(np.array([x]), 0.0, 1.0, q, nk)[0]
        want = [(1 - s) ** 3 / 6, (3 * s**3 - 6 * s**2 + 4) / 6, (-3 * s**3 + 3 * s**2 + 3 * s + 1) / 6, s**3 / 6]
        np.testing.assert_allclose(row[j:j + 4], want, atol=1e-13)


def test_linear_basis():
    np.testing.assert_array_equal(O.linear_basis([2.0, -1.5]), [[1.0, 2.0], [1.0, -1.5]])


def test_penalty_second_order_difference():
    for d in (4, 7, 24):
        D = np.diff(np.eye(d), n=2, axis=0)
        np.testing.assert_allclose(O.penalty(d, 2), D.T @ D, atol=0)
    D1 = np.diff(np.eye(6), n=1, axis=0)
    np.testing.assert_allclose(O.penalty(6, 1), D1.T @ D1, atol=0)


# --------------------------------------------------------------- Algorithm 2

def test_binmatvec_binmatmat_equal_dense_products():
    rng = np.random.default_rng(7)
    n, nstar = 3000, 40
    x = rng.random(n)
    ind, z = O.bin_equidistant(x, nstar)
    Zb = O.bspline_basis(z, x.min(), x.max(), 3, 20)
    Zt = Zb[ind]                                   # discretised dense design (n x d)
    w = rng.random(n) + 0.5
    r = rng.normal(size=n)
    rows = (rng.random(n) < 0.7).astype(np.uint8)
    W = w * rows
    np.testing.assert_allclose(O.bin_matvec(ind, r, Zb, w=w, rows=rows), Zt.T @ (W * r), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.bin_matmat(ind, Zb, w=w, rows=rows), Zt.T @ (W[:, None] * Zt), rtol=1e-12,
                               atol=1e-12)
    u = O.bin_matvec_u(ind, r, nstar)
    np.testing.assert_allclose(u, np.bincount(ind, weights=r, minlength=nstar), atol=1e-12)


# --------------------------------------------------------------- df -> lambda (App. A.2)

def _tiny_design(seed=8, n=60, nstar=12):
    rng = np.random.default_rng(seed)
    x = rng.random(n)
    ind, z = O.bin_equidistant(x, nstar)
    Zb = O.bspline_basis(z, x.min(), x.max(), 3, 4)
    return Zb[ind], Zb, ind


def test_df1_equals_trace_of_explicit_hat_matrix():
    Zt, Zb, ind = _tiny_design()
    d = Zt.shape[1]
    K = O.penalty(d, 2)
    G = Zt.T @ Zt
    for lam in (0.0, 0.1, 3.0, 250.0):
        H = Zt @ np.linalg.solve(G + lam * K, Zt.T)         # n x n hat matrix, Eq. (modelfit)
        assert abs(O.df1(G, K, lam) - np.trace(H)) < 1e-9


def test_lambda_for_df_solves_and_limits():
    Zt, Zb, ind = _tiny_design()
    d = Zt.shape[1]
    K = O.penalty(d, 2)
    G = Zt.T @ Zt
    for df in (2.5, 3.0, 5.0, 7.5):
        lam = O.lambda_for_df(G, K, df)
        H = Zt @ np.linalg.solve(G + lam * K, Zt.T)
        assert abs(np.trace(H) - df) < 1e-8
    # df at or above the full rank gives lambda = 0; df -> 2 is the penalty null space
    assert O.lambda_for_df(G, K, d + 1.0) == 0.0
    assert abs(O.df1(G, K, 1e12) - 2.0) < 1e-3


def test_spd_inverse():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(24, 24))
    A = A @ A.T + 24 * np.eye(24)
    np.testing.assert_allclose(O.spd_inverse(A) @ A, np.eye(24), atol=1e-12)


# --------------------------------------------------------------- losses

def test_offsets_closed_form():
    y = np.array([1.0, 0.0, 1.0, 1.0])
    assert O.offset(O.LOSS_L2, y) == 0.75
    assert abs(O.offset(O.LOSS_BINOMIAL, y) - math.log(3.0)) < 1e-15


@pytest.mark.parametrize("kind", [O.LOSS_L2, O.LOSS_BINOMIAL])
def test_pseudo_residual_is_negative_gradient(kind):
    eps = 1e-6
    for y in (0.0, 1.0):
        for f in (-3.0, -0.2, 0.0, 0.7, 4.0):
            fd = -(O.loss(kind, y, f + eps) - O.loss(kind, y, f - eps)) / (2 * eps)
            assert abs(O.pseudo_residual(kind, y, f) - fd) < 1e-8


# --------------------------------------------------------------- CWB (Algorithm 1)

def _single_feature(seed=10, n=500):
    rng = np.random.default_rng(seed)
    x = rng.random(n)
    y = np.sin(3 * x) + 0.3 * rng.normal(size=n)
    return x, y


def test_single_learner_closed_form():
    """L2, one learner: theta_agg after M steps is sum_{j<M} (I - nu P G)^j nu P Z^T r_0."""
    x, y = _single_feature()
    nstar, nu, M = 22, 0.3, 37
    spec = dict(feature=0, n_bins=nstar, df=5.0)
    res = O.fit(x[None, :], y, [spec], nu=nu, iterations=M)
    ind, z = O.bin_equidistant(x, nstar)
    Zb = O.bspline_basis(z, x.min(), x.max(), 3, 20)
    Zt = Zb[ind]
    G = Zt.T @ Zt
    K = O.penalty(24, 2)
    lam = res.lam[0]
    P = np.linalg.inv(G + lam * K)
    r0 = y - y.mean()
    step = nu * P @ (Zt.T @ r0)
    A = np.eye(24) - nu * P @ G
    acc, Ak = np.zeros(24), np.eye(24)
    for _ in range(M):
        acc += Ak @ step
        Ak = A @ Ak
    np.testing.assert_allclose(res.theta_f[0], acc, rtol=1e-9, atol=1e-9 * np.abs(acc).max())
    # one step with nu = 1 is the penalised least-squares fit (Eq. pen-regr)
    one = O.fit(x[None, :], y, [spec], nu=1.0, iterations=1)
    pls = np.linalg.solve(G + lam * K, Zt.T @ r0)
    np.testing.assert_allclose(one.theta_f[0], pls, rtol=1e-9, atol=1e-10)
    # the fitted vector is the aggregated model evaluated at the binned design
    np.testing.assert_allclose(res.f, y.mean() + Zt @ res.theta_f[0], atol=1e-10)


def test_sse_identity_on_first_iteration():
    """SSE_k (definition) = r^T r - 2 theta^T s + theta^T G theta for the selected learner."""
    x, y = _single_feature(11)
    X = np.stack([x, np.random.default_rng(3).random(x.size)])
    specs = [dict(feature=0, n_bins=30), dict(feature=1, n_bins=30)]
    res = O.fit(X, y, specs, nu=0.1, iterations=1)
    k = res.k_sel[0]
    ind, z = O.bin_equidistant(X[k], 30)
    Zt = O.bspline_basis(z, X[k].min(), X[k].max(), 3, 20)[ind]
    r = y - y.mean()
    theta = res.theta_f[k] / 0.1
    s = Zt.T @ r
    G = Zt.T @ Zt
    assert abs(res.sse_best[0] - (r @ r - 2 * theta @ s + theta @ G @ theta)) < 1e-8 * (r @ r)


def test_argmin_picks_signal_and_breaks_ties_low():
    rng = np.random.default_rng(12)
    n = 800
    X = rng.random((3, n))
    y = np.sin(6 * X[1]) + 0.05 * rng.normal(size=n)
    specs = [dict(feature=0, n_bins=25), dict(feature=1, n_bins=25), dict(feature=1, n_bins=25)]
    res = O.fit(X, y, specs, iterations=5)
    # learners 1 and 2 are identical: SSE ties exactly, the lower index wins
    assert (res.k_sel == 1).all()
    assert (res.sse_best == res.sse_second).all()


def test_exact_binning_reproduces_unbinned():
    """Binning with n* = number of unique values reproduces unbinned CWB (Sec. 3.1)."""
    rng = np.random.default_rng(13)
    n = 300
    X = np.round(rng.random((3, n)) * 60) / 60.0       # repeated values
    y = np.sin(5 * X[0]) + X[2] ** 2 + 0.1 * rng.normal(size=n)
    ex = [dict(feature=j, n_bins=O.BINS_EXACT) for j in range(3)]
    de = [dict(feature=j, n_bins=O.BINS_DENSE) for j in range(3)]
    a = O.fit(X, y, ex, iterations=40)
    b = O.fit(X, y, de, iterations=40)
    np.testing.assert_array_equal(a.k_sel, b.k_sel)
    np.testing.assert_allclose(a.theta_f, b.theta_f, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(a.f, b.f, atol=1e-11)
    np.testing.assert_allclose(a.lam, b.lam, rtol=1e-9)


def test_equidistant_binning_on_grid_data_is_exact():
    """Data on an equidistant grid of G points binned with n* = G equals exact binning."""
    rng = np.random.default_rng(14)
    Gp = 37
    X = rng.integers(0, Gp, size=(2, 500)) / (Gp - 1.0)
    X[:, 0] = 0.0
    X[:, 1] = 1.0
    y = np.cos(4 * X[0]) + 0.1 * rng.normal(size=500)
    a = O.fit(X, y, [dict(feature=j, n_bins=Gp) for j in range(2)], iterations=30)
    b = O.fit(X, y, [dict(feature=j, n_bins=O.BINS_DENSE) for j in range(2)], iterations=30)
    np.testing.assert_array_equal(a.k_sel, b.k_sel)
    np.testing.assert_allclose(a.theta_f, b.theta_f, rtol=1e-9, atol=1e-12)


def test_prediction_at_training_points_equals_fitted_vector():
    rng = np.random.default_rng(15)
    X = rng.random((3, 400))
    y = np.sin(4 * X[0]) - X[1] + 0.1 * rng.normal(size=400)
    specs = [dict(feature=j, n_bins=O.BINS_EXACT) for j in range(3)] + [dict(type=O.BL_LINEAR, feature=1,
                                                                              n_bins=O.BINS_EXACT)]
    for opt in (O.OPT_CWB, O.OPT_ACWB):
        res = O.fit(X, y, specs, opt=opt, gamma=0.01, iterations=30)
        xmin = [X[s["feature"]].min() for s in specs]
        xmax = [X[s["feature"]].max() for s in specs]
        pred = O.predict(X, specs, xmin, xmax, res.theta_f, res.offset)
        np.testing.assert_allclose(pred, res.f, atol=1e-10)



def test_prediction_clamps_to_the_training_range():
    """Prediction outside [min x, max x] evaluates each learner at the nearest end of its training
    range (reading R19): the basis comes from scipy's B-spline design matrix at the clamped point,
    and a linear learner gives theta_0 + theta_1 clamp(x)."""
    from scipy.interpolate import BSpline
    rng = np.random.default_rng(31)
    n = 800
    X = rng.random((3, n)) * np.array([[2.0], [1.0], [3.0]]) - np.array([[0.5], [0.0], [1.0]])
    y = np.sin(3 * X[0]) + 0.7 * X[1] - 0.3 * X[2] ** 2 + 0.1 * rng.normal(size=n)
    specs = [dict(feature=0, n_bins=O.BINS_SQRT), dict(type=O.BL_LINEAR, feature=1, n_bins=O.BINS_SQRT),
             dict(feature=2, n_bins=O.BINS_SQRT, degree=2, n_knots=12)]
    res = O.fit(X, y, specs, iterations=60)
    assert len(set(res.k_sel.tolist())) == 3            # every learner carries coefficients
    xmin = np.array([X[s["feature"]].min() for s in specs])
    xmax = np.array([X[s["feature"]].max() for s in specs])
    span = xmax - xmin
    # rows far below, just below, at, and above the range of every feature at once
    offsets = np.array([-3.0, -1e-3, 0.0, 1.0, 1.0 + 1e-3, 4.0])
    Xnew = np.empty((3, offsets.size))
    for j in range(3):
        Xnew[j] = xmin[j] + offsets * span[j]
    got = O.predict(Xnew, specs, xmin, xmax, res.theta_f, res.offset)
    want = np.full(offsets.size, res.offset)
    for k, sp in enumerate(specs):
        xc = np.clip(Xnew[sp["feature"]], xmin[k], xmax[k])
        th = res.theta_f[k]
        if sp.get("type") == O.BL_LINEAR:
            want += th[0] + th[1] * xc
            continue
        q, nk = sp.get("degree", 3), sp.get("n_knots", 20)
        delta = (xmax[k] - xmin[k]) / (nk + 1)
        t = xmin[k] + (np.arange(nk + 2 * q + 2) - q) * delta
        Bm = BSpline.design_matrix(xc, t, q).toarray()
        want += Bm @ th[: nk + q + 1]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    # outside the range the prediction is flat: equal to the prediction at the nearest end
    np.testing.assert_allclose(got[0], got[2], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(got[5], got[3], rtol=1e-13, atol=1e-13)

# --------------------------------------------------------------- ACWB (Algorithm 3)

def _read_golden_acwb():
    rows = []
    with open(os.path.join(GOLDEN, "acwb_orthogonal_n4.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            m, k, kc, fx1, fx2, hx1, hx2 = line.split()
            rows.append((int(m), int(k), int(kc), *[float(Fraction(v)) for v in (fx1, fx2, hx1, hx2)]))
    return rows


def test_acwb_hand_computed_recursion():
    x1 = np.array([-1.0, -1.0, 1.0, 1.0])
    x2 = np.array([-1.0, 1.0, -1.0, 1.0])
    X = np.stack([x1, x2])
    y = 2 * x1 + x2
    specs = [dict(type=O.BL_LINEAR, feature=0, n_bins=O.BINS_EXACT),
             dict(type=O.BL_LINEAR, feature=1, n_bins=O.BINS_EXACT)]
    for m, k, kc, fx1, fx2, hx1, hx2 in _read_golden_acwb():
        res = O.fit(X, y, specs, opt=O.OPT_ACWB, nu=0.5, gamma=0.5, iterations=m)
        assert res.k_sel[m - 1] == k - 1 and res.k_cor[m - 1] == kc - 1
        np.testing.assert_allclose(res.f, fx1 * x1 + fx2 * x2, atol=1e-14)
        # aggregated parameters (Sec. 3.2.1): intercept 0, slopes equal the coordinates
        np.testing.assert_allclose(res.theta_f, [[0, fx1], [0, fx2]], atol=1e-14)
        np.testing.assert_allclose(res.theta_h, [[0, hx1], [0, hx2]], atol=1e-14)


# --------------------------------------------------------------- HCWB (Algorithm 4)

def _hybrid_data(seed=16, n=600):
    rng = np.random.default_rng(seed)
    X = rng.random((3, n))
    y = np.sin(5 * X[0]) + 0.5 * X[1] + 0.4 * rng.normal(size=n)
    val = (rng.random(n) < 0.25).astype(np.uint8)
    # extremes of every feature in training rows so per-phase binning ranges agree
    for j in range(3):
        val[np.argmin(X[j])] = 0
        val[np.argmax(X[j])] = 0
    return X, y, val


def test_hybrid_patience_zero_is_cwb_on_all_rows():
    X, y, val = _hybrid_data()
    specs = [dict(feature=j, n_bins=20) for j in range(3)]
    off = O.offset(O.LOSS_L2, y, rows=1 - val)
    h = O.fit(X, y, specs, opt=O.OPT_HCWB, val_mask=val, patience=0, gamma=0.05, iterations=25)
    c = O.fit(X, y, specs, opt=O.OPT_CWB, iterations=25, offset_value=off)
    assert h.switch_iter == 1
    np.testing.assert_array_equal(h.k_sel, c.k_sel)
    np.testing.assert_allclose(h.theta_f, c.theta_f, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(h.f, c.f, atol=1e-12)


def test_hybrid_large_patience_is_acwb_on_training_rows():
    X, y, val = _hybrid_data()
    specs = [dict(feature=j, n_bins=20) for j in range(3)]
    M = 30
    h = O.fit(X, y, specs, opt=O.OPT_HCWB, val_mask=val, patience=M + 1, gamma=0.05, iterations=M)
    tr = val == 0
    a = O.fit(X[:, tr], y[tr], specs, opt=O.OPT_ACWB, gamma=0.05, iterations=M)
    assert h.switch_iter == 0
    np.testing.assert_array_equal(h.k_sel, a.k_sel)
    np.testing.assert_array_equal(h.k_cor, a.k_cor)
    np.testing.assert_allclose(h.theta_f, a.theta_f, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(h.theta_h, a.theta_h, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(h.f[tr], a.f, atol=1e-11)


def test_hybrid_switch_follows_patience_rule_on_recorded_risks():
    """Counter += 1 on a strictly larger validation risk, reset otherwise; switch at pat_0."""
    rng = np.random.default_rng(17)
    n = 500
    X = rng.random((2, n))
    y = np.sin(5 * X[0]) + 2.0 * rng.normal(size=n)         # noisy: validation risk turns up
    val = (rng.random(n) < 0.4).astype(np.uint8)
    for j in range(2):
        val[np.argmin(X[j])] = 0
        val[np.argmax(X[j])] = 0
    specs = [dict(feature=j, n_bins=22) for j in range(2)]
    pat = 3
    res = O.fit(X, y, specs, opt=O.OPT_HCWB, val_mask=val, patience=pat, gamma=0.5, nu=0.5, iterations=150)
    assert res.switch_iter > 0
    tr = val == 0
    prev = np.mean([O.loss(0, yy, res.offset) for yy in y[val == 1]])
    counter, expect = 0, 0
    for m in range(1, 151):
        if counter >= pat:
            expect = m
            break
        risk = res.val_risk[m - 1]
        counter = counter + 1 if risk > prev else 0
        prev = risk
    assert res.switch_iter == expect
    assert np.isnan(res.val_risk[res.switch_iter - 1:]).all()
    assert (res.k_cor[res.switch_iter - 1:] == -1).all()
    assert tr.sum() > 0



def _closed_form_loss(kind, y, f):
    """L2: (y - f)^2 / 2; binomial with y in {0, 1}: log(1 + e^f) - y f (reading R17)."""
    if kind == O.LOSS_L2:
        return 0.5 * (y - f) ** 2
    return np.logaddexp(0.0, f) - y * f


@pytest.mark.parametrize("kind", [O.LOSS_L2, O.LOSS_BINOMIAL])
def test_hybrid_validation_risk_is_mean_loss_of_f_on_validation_rows(kind):
    """Algorithm 4's validation risk after iteration m is the empirical risk R_emp(f^[m] | D_val):
    the mean over the validation rows of the loss at the primary model f^[m].  Recomputed here with
    numpy from the f the oracle returns after m iterations (the fit is sequential, so a fit of m
    iterations ends in the state the m-th iteration of a longer fit passes through), and the
    patience rule replayed on these recomputed risks, starting from the offset model's risk."""
    rng = np.random.default_rng(32)
    n = 420
    X = rng.random((2, n))
    eta = 2.0 * np.sin(5 * X[0]) - X[1]
    if kind == O.LOSS_L2:
        y = eta + 1.5 * rng.normal(size=n)
    else:
        y = (rng.random(n) < 1 / (1 + np.exp(-eta))).astype(np.float64)
    val = (rng.random(n) < 0.3).astype(np.uint8)
    for j in range(2):
        val[np.argmin(X[j])] = 0
        val[np.argmax(X[j])] = 0
    specs = [dict(feature=j, n_bins=16) for j in range(2)]
    kw = dict(loss=kind, opt=O.OPT_HCWB, val_mask=val, gamma=0.5, nu=0.5)
    pat = 2
    M = 40
    full = O.fit(X, y, specs, patience=pat, iterations=M, **kw)
    vm = val == 1
    prev = float(np.mean(_closed_form_loss(kind, y[vm], np.full(vm.sum(), full.offset))))
    counter, switch = 0, 0
    for m in range(1, M + 1):
        if counter >= pat:
            switch = m
            break
        f_m = O.fit(X, y, specs, patience=pat, iterations=m, **kw).f
        risk = float(np.mean(_closed_form_loss(kind, y[vm], f_m[vm])))
        np.testing.assert_allclose(full.val_risk[m - 1], risk, rtol=1e-12, atol=0.0)
        # not the training rows' risk (the two differ on this data)
        assert abs(risk - float(np.mean(_closed_form_loss(kind, y[~vm], f_m[~vm])))) > 1e-6 * risk
        counter = counter + 1 if risk > prev else 0
        prev = risk
    assert switch > 0, "the data should make the validation risk turn up"
    assert full.switch_iter == switch

def test_binomial_fit_decreases_risk():
    rng = np.random.default_rng(18)
    n = 1000
    X = rng.random((3, n))
    prob = 1 / (1 + np.exp(-(3 * np.sin(5 * X[0]) - 1.5 * X[2])))
    y = (rng.random(n) < prob).astype(np.float64)
    specs = [dict(feature=j, n_bins=30) for j in range(3)]
    res = O.fit(X, y, specs, loss=O.LOSS_BINOMIAL, iterations=80)
    risk0 = np.mean([O.loss(1, a, res.offset) for a in y])
    risk = np.mean([O.loss(1, a, b) for a, b in zip(y, res.f)])
    assert risk < risk0
    assert set(res.k_sel.tolist()) <= {0, 2}


# --------------------------------------------------------------- categorical learners (App. B.1)

def _categorical_data(seed=21, n=900, c=7):
    rng = np.random.default_rng(seed)
    probs = rng.dirichlet(np.full(c, 0.7))
    codes = rng.choice(c, size=n, p=probs).astype(np.float64)
    codes[:c] = np.arange(c)                        # every class present at least once
    effect = rng.normal(size=c)
    y = effect[codes.astype(int)] + 0.5 * rng.normal(size=n)
    w = rng.uniform(0.5, 2.0, size=n)
    return codes, y, w, c


def test_categorical_ridge_closed_form_over_iterations():
    """Ridge learner: (Z^T W Z + lambda I) is diagonal with entries n_k + lambda (App. B.1), so for
    L2 and one learner theta after M steps is (1 - (1 - nu n_k / (n_k + lambda))^M) u_k / n_k per
    class, with n_k the class weight and u_k the class sum of w r_0."""
    codes, y, w, c = _categorical_data()
    lam, nu = 3.5, 0.3
    spec = dict(type=O.BL_CATEGORICAL, feature=0, n_knots=c, df=0.0, lam=lam)
    r0 = y - np.sum(w * y) / np.sum(w)
    nk = np.bincount(codes.astype(int), weights=w, minlength=c)
    uk = np.bincount(codes.astype(int), weights=w * r0, minlength=c)
    for M in (1, 17):
        res = O.fit(codes[None, :], y, [spec], w=w, nu=nu, iterations=M)
        want = (1.0 - (1.0 - nu * nk / (nk + lam)) ** M) * uk / nk
        np.testing.assert_allclose(res.theta_f[0, :c], want, rtol=1e-10, atol=1e-13)
        assert res.nstar[0] == c and res.lam[0] == lam
        np.testing.assert_allclose(res.f, res.offset + res.theta_f[0, codes.astype(int)], atol=1e-12)


def test_categorical_ridge_df_matches_scalar_closed_form():
    """df1 of the ridge learner is sum_k n_k / (n_k + lambda) (App. B.1); the oracle's lambda, found
    by its general matrix search, must solve that scalar equation."""
    from scipy.optimize import brentq
    codes, y, _, c = _categorical_data(22, n=2000, c=9)
    nk = np.bincount(codes.astype(int), minlength=c).astype(np.float64)
    for df in (1.5, 4.0, 8.5):
        res = O.fit(codes[None, :], y, [dict(type=O.BL_CATEGORICAL, feature=0, n_knots=c, df=df)],
                    iterations=1)
        want = brentq(lambda lam: np.sum(nk / (nk + lam)) - df, 1e-12, 1e12, xtol=1e-14, rtol=1e-15)
        assert abs(res.lam[0] - want) <= 1e-9 * want
    # df at or above c (all classes free) gives the unpenalised fit
    res = O.fit(codes[None, :], y, [dict(type=O.BL_CATEGORICAL, feature=0, n_knots=c, df=c)], iterations=1)
    assert res.lam[0] == 0.0


def test_categorical_binary_learner_is_class_mean_and_selects_largest_reduction():
    """Binary learner of class k: theta = class mean of r (App. B.1); among binary learners of one
    feature the argmin of the SSE is the class with the largest u_k^2 / n_k (brute force)."""
    codes, y, w, c = _categorical_data(23)
    specs = [dict(type=O.BL_CATEGORICAL_BINARY, feature=0, n_knots=c, level=k) for k in range(c)]
    res = O.fit(codes[None, :], y, specs, w=w, nu=1.0, iterations=1)
    r0 = y - np.sum(w * y) / np.sum(w)
    nk = np.bincount(codes.astype(int), weights=w, minlength=c)
    uk = np.bincount(codes.astype(int), weights=w * r0, minlength=c)
    best = int(np.argmax(uk ** 2 / nk))
    assert res.k_sel[0] == best
    assert abs(res.theta_f[best, 0] - uk[best] / nk[best]) <= 1e-12 * abs(uk[best] / nk[best])
    assert (res.theta_f[np.arange(c) != best, 0] == 0.0).all()
    assert (res.lam == 0.0).all()
    # a binary learner's SSE is sum w r^2 - u_k^2 / n_k
    assert abs(res.sse_best[0] - (np.sum(w * r0 ** 2) - uk[best] ** 2 / nk[best])) <= 1e-9 * np.sum(w * r0 ** 2)


def test_categorical_ridge_unpenalised_equals_sum_of_binary_steps():
    """With lambda = 0 and nu = 1, one ridge step fits every class mean at once, i.e. the sum of the
    c binary learners' one-step fits (they touch disjoint rows)."""
    codes, y, w, c = _categorical_data(24)
    ridge = O.fit(codes[None, :], y, [dict(type=O.BL_CATEGORICAL, feature=0, n_knots=c, df=0.0, lam=0.0)],
                  w=w, nu=1.0, iterations=1)
    specs = [dict(type=O.BL_CATEGORICAL_BINARY, feature=0, n_knots=c, level=k) for k in range(c)]
    binary = O.fit(codes[None, :], y, specs, w=w, nu=1.0, iterations=c)
    assert sorted(binary.k_sel.tolist()) == list(range(c))     # each class once, then done
    np.testing.assert_allclose(binary.theta_f[:, 0], ridge.theta_f[0, :c], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(binary.f, ridge.f, atol=1e-12)


def test_categorical_prediction_of_unknown_codes_is_offset_only():
    codes, y, w, c = _categorical_data(25)
    specs = [dict(type=O.BL_CATEGORICAL, feature=0, n_knots=c, df=3.0),
             dict(type=O.BL_CATEGORICAL_BINARY, feature=0, n_knots=c, level=2)]
    res = O.fit(codes[None, :], y, specs, w=w, iterations=20)
    Xn = np.array([[0.0, 2.0, c - 1.0, -1.0, float(c), 2.5, np.nan]])
    pred = O.predict(Xn, specs, [0.0, 0.0], [c - 1.0, c - 1.0], res.theta_f, res.offset)
    want = res.offset + np.array([res.theta_f[0, 0], res.theta_f[0, 2] + res.theta_f[1, 0], res.theta_f[0, c - 1],
                                  0.0, 0.0, 0.0, 0.0])
    np.testing.assert_allclose(pred, want, atol=1e-14)
    # at the training rows the prediction is the fitted vector
    np.testing.assert_allclose(O.predict(codes[None, :], specs, [0.0, 0.0], [c - 1.0, c - 1.0], res.theta_f,
                                         res.offset), res.f, atol=1e-12)


@pytest.mark.parametrize("bad", [2.5, -1.0, 7.0])
def test_categorical_rejects_codes_outside_the_classes(bad):
    codes, y, _, c = _categorical_data(26)
    codes = codes.copy()
    codes[5] = bad
    with pytest.raises(RuntimeError):
        O.fit(codes[None, :], y, [dict(type=O.BL_CATEGORICAL, feature=0, n_knots=c)], iterations=1)
    with pytest.raises(RuntimeError):
        O.fit(np.arange(900.0)[None, :] % 7, y, [dict(type=O.BL_CATEGORICAL_BINARY, feature=0, n_knots=7,
                                                        level=7)], iterations=1)


def test_learner_loop_on_several_threads_is_bit_identical():
    import synthetic_inputs as S
    """The OpenMP learner loop of the oracle changes only who computes each learner's fit: the
    selections, coefficients, criteria and fitted values equal the one-thread run bit for bit."""
    data = S.additive_regression(3000, 6, 3, seed=17, dtype=np.float64)
    specs = [dict(feature=j) for j in range(6)] + [dict(feature=j, type=O.BL_LINEAR) for j in range(3)]
    O.set_threads(1)
    one = O.fit(data.X, data.y, specs, iterations=25)
    got = O.set_threads(4)
    try:
        many = O.fit(data.X, data.y, specs, iterations=25)
    finally:
        O.set_threads(1)
    np.testing.assert_array_equal(one.k_sel, many.k_sel)
    np.testing.assert_array_equal(one.theta_f, many.theta_f)
    np.testing.assert_array_equal(one.sse_best, many.sse_best)
    np.testing.assert_array_equal(one.f, many.f)
    assert got in (1, 4)
