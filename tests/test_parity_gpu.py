"""Parity of the CUDA library (through the C ABI) with the FP64 oracle, on the GPU.

Inputs are seeded and synthetic; sizes span several scatter tiles, ragged row
counts, both index widths (uint8 for n* <= 256, uint16 otherwise), exact and
equidistant binning, both losses, weights, all three optimisers.
"""
import numpy as np
import pytest

import synthetic_inputs as S
from oracle import oracle as O
from parity_util import REL_TOL, check_coefficients, check_sequences, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cwb():
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as pkg
    return pkg


def _specs_to_gpu(cwb, specs):
    out = []
    for s in specs:
        out.append(cwb.learner(s["feature"], type=s.get("type", 0), degree=s.get("degree", 3),
                               n_knots=s.get("n_knots", 20), diff_order=s.get("diff_order", 2),
                               df=s.get("df", 5.0), lam=s.get("lam", 0.0), n_bins=s.get("n_bins", -1),
                               level=s.get("level", 0)))
    return out


def run_pair(cwb, X, y, specs, *, M, loss=0, opt=0, nu=0.1, gamma=0.0, patience=5, w=None, val_mask=None,
             check_predict=True):
    """Fit on the GPU and in the oracle, compare everything; returns (model, oracle result)."""
    X = np.ascontiguousarray(X)
    model = cwb.Model(X, y, _specs_to_gpu(cwb, specs), loss=loss, opt=opt, nu=nu, gamma=gamma, iterations=M,
                      patience=patience, w=w, val_mask=val_mask, device=0)
    model.fit(M)
    ref = O.fit(X.astype(np.float64), np.asarray(y, dtype=np.float64), specs, loss=loss, opt=opt, nu=nu,
                gamma=gamma, iterations=M, patience=patience, w=w, val_mask=val_mask)
    k_sel, k_cor, sw = model.trace()
    assert k_sel.size == M
    tie = check_sequences(k_sel, ref, k_cor if opt != 0 else None)
    if tie >= 0:
        # an oracle near-tie: replay the GPU with the oracle's choices forced and compare the rest
        model.free()
        model = cwb.Model(X, y, _specs_to_gpu(cwb, specs), loss=loss, opt=opt, nu=nu, gamma=gamma, iterations=M,
                          patience=patience, w=w, val_mask=val_mask, device=0)
        model.force_selection(ref.k_sel)
        model.fit(M)
        k_sel, k_cor, sw = model.trace()
    if opt == 2:
        assert sw == ref.switch_iter
    theta = model.all_coefficients(0, dmax=ref.dmax)
    check_coefficients(theta, ref.theta_f)
    if opt != 0:
        check_coefficients(model.all_coefficients(1, dmax=ref.dmax), ref.theta_h)
    f = model.fitted()
    assert rel_err(f, ref.f) <= REL_TOL, rel_err(f, ref.f)
    assert abs(model.offset - ref.offset) <= 1e-12 * max(1.0, abs(ref.offset))
    if check_predict:
        rng = np.random.default_rng(99)
        p, n = X.shape
        idx = rng.integers(0, n, size=min(n, 3000))
        Xn = X[:, idx].astype(np.float64) + rng.normal(scale=0.01, size=(p, idx.size))
        for sp in specs:
            if sp.get("type", 0) in (O.BL_CATEGORICAL, O.BL_CATEGORICAL_BINARY):
                # class codes, a few replaced by an unseen code, a negative one or a non-integer
                row = X[sp["feature"], idx].astype(np.float64)
                odd = rng.random(idx.size) < 0.05
                row[odd] = rng.choice([float(sp["n_knots"]), -1.0, 1.5], size=int(odd.sum()))
                Xn[sp["feature"]] = row
        xmin = [X[s["feature"]].min() for s in specs]
        xmax = [X[s["feature"]].max() for s in specs]
        pred_ref = O.predict(Xn, specs, xmin, xmax, ref.theta_f, ref.offset)
        pred = model.predict(np.ascontiguousarray(Xn))
        assert rel_err(pred, pred_ref) <= REL_TOL, rel_err(pred, pred_ref)
    return model, ref


# ------------------------------------------------------------------ setup

@pytest.mark.parametrize("n_bins,n", [(-1, 5000), (300, 4099), (2, 777)])
def test_setup_matches_oracle(cwb, n_bins, n):
    data = S.additive_regression(n, 4, 3, seed=21, dtype=np.float32)
    specs = [dict(feature=j, n_bins=n_bins) for j in range(4)]
    if n_bins == 2:
        specs = [dict(feature=j, n_bins=2, type=1) for j in range(4)]
    model = cwb.Model(data.X, data.y, _specs_to_gpu(cwb, specs), iterations=1, device=0)
    for k, s in enumerate(specs):
        x = data.X[s["feature"]].astype(np.float64)
        nstar = O.isqrt(n) if n_bins == -1 else n_bins
        ind_ref, z = O.bin_equidistant(x, nstar)
        ind = model.bin_index(k)
        np.testing.assert_array_equal(ind, ind_ref)          # integer work: bit-exact
        info = model.learner_info(k)
        assert info.nstar == nstar and info.xmin == x.min() and info.xmax == x.max()
        if s.get("type", 0) == 1:
            Zb = O.linear_basis(z)
        else:
            Zb = O.bspline_basis(z, x.min(), x.max(), 3, 20)
        G_ref = O.bin_matmat(ind_ref, Zb)
        G, P = model.matrices(k)
        assert rel_err(G, G_ref) < 1e-12
        if s.get("type", 0) == 1:
            lam = 0.0
        else:
            lam = O.lambda_for_df(G_ref, O.penalty(24, 2), 5.0)
        assert abs(info.lam - lam) <= 1e-8 * max(lam, 1e-300)
        K = O.penalty(Zb.shape[1], 2) if s.get("type", 0) == 0 else np.zeros((2, 2))
        P_ref = O.spd_inverse(G_ref + lam * K)
        assert rel_err(P, P_ref) < 1e-7
    model.free()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("nstar", [7, 1000, 60000])
def test_binning_at_half_way_points_is_bit_exact(cwb, dtype, nstar):
    """Values on, and a few ulps around, the half-way points between design points (where the
    rule sends ties to the lower point) and on the design points themselves: the device index
    equals the oracle's bit for bit, for FP32 and FP64 features (Sec. 3.1.1)."""
    rng = np.random.default_rng(nstar)
    lo, hi = -3.7, 11.3
    h = (hi - lo) / (nstar - 1)
    l = rng.integers(0, nstar - 1, size=20_000)
    mids = lo + (l + 0.5) * h
    pts = lo + l * h
    vals = [np.array([lo, hi]), mids, pts]
    for k in (1, 2, 3):
        vals += [np.nextafter(mids, np.inf) if k == 1 else mids + k * np.spacing(mids),
                 mids - k * np.spacing(mids)]
    x = np.concatenate(vals).astype(dtype)
    x[0], x[1] = dtype(lo), dtype(hi)
    y = rng.normal(size=x.size).astype(dtype)
    X = np.stack([x, rng.random(x.size).astype(dtype)])
    m = cwb.Model(X, y, [cwb.learner(0, n_bins=nstar, type=1)], iterations=1, device=0)
    ind_ref, _ = O.bin_equidistant(x.astype(np.float64), nstar)
    np.testing.assert_array_equal(m.bin_index(0), ind_ref)
    m.free()


def test_lambda_on_sparse_tail_bins(cwb):
    """N(0,1) features: nearly empty tail bins make Z^T Z ill conditioned; lambda must still match."""
    data = S.sim_binomial_hybrid(seed=30, n=40_000, p=8, n_informative=3)
    specs = [dict(feature=j, n_bins=-1) for j in range(8)]
    model = cwb.Model(data.X, data.y, _specs_to_gpu(cwb, specs), loss=1, iterations=1, device=0)
    for k in range(8):
        x = data.X[k].astype(np.float64)
        ind, z = O.bin_equidistant(x, O.isqrt(x.size))
        G_ref = O.bin_matmat(ind, O.bspline_basis(z, x.min(), x.max(), 3, 20))
        lam = O.lambda_for_df(G_ref, O.penalty(24, 2), 5.0)
        info = model.learner_info(k)
        assert abs(info.lam - lam) <= 1e-9 * lam, (k, info.lam, lam)
        G, P = model.matrices(k)
        P_ref = O.spd_inverse(G_ref + lam * O.penalty(24, 2))
        assert rel_err(P, P_ref) < 1e-8
    model.free()


def test_exact_binning_setup(cwb):
    data = S.sim_small_exact(seed=0, n=3000, p=3)
    X = np.round(data.X * 400) / 400          # repeated values
    specs = [dict(feature=j, n_bins=0) for j in range(3)]
    model = cwb.Model(X, data.y, _specs_to_gpu(cwb, specs), iterations=1, device=0)
    for k in range(3):
        ind_ref, z = O.bin_exact(X[k])
        np.testing.assert_array_equal(model.bin_index(k), ind_ref)
        assert model.learner_info(k).nstar == z.size
    model.free()


# ------------------------------------------------------------------ CWB

def test_cwb_l2_binned_uint8(cwb):
    data = S.additive_regression(20_011, 6, 4, seed=22, dtype=np.float32)   # n* = 141, ragged n
    specs = [dict(feature=j, n_bins=-1) for j in range(6)]
    run_pair(cwb, data.X, data.y, specs, M=120)


def test_cwb_l2_binned_uint16_many_tiles(cwb):
    data = S.additive_regression(100_003, 40, 10, seed=23, dtype=np.float32)
    specs = [dict(feature=j, n_bins=400) for j in range(40)]
    run_pair(cwb, data.X, data.y, specs, M=150)


def test_cwb_signal_in_the_second_binning_group(cwb):
    """p = 40 splits into two scatter groups of 20 binnings; the informative features are the
    last ten columns, so every selection comes from the second group's histograms."""
    data = S.additive_regression(60_013, 40, 10, seed=27, dtype=np.float32)
    X = np.ascontiguousarray(data.X[::-1])
    specs = [dict(feature=j, n_bins=-1) for j in range(40)]
    model, ref = run_pair(cwb, X, data.y, specs, M=80)
    assert model.scatter_plan()["groups"] >= 2
    assert np.mean(np.asarray(ref.k_sel) >= 20) > 0.9


def test_cwb_bins_split_over_ranges(cwb):
    """n* = 60,000 does not fit one CTA's shared memory: the scatter splits the bins over
    ranges (slots) and the solve gathers each learner's histogram from both."""
    data = S.additive_regression(150_001, 3, 3, seed=28, dtype=np.float32)
    specs = [dict(feature=0, n_bins=60_000), dict(feature=1, n_bins=-1), dict(feature=2, n_bins=5000)]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=60)
    assert model.scatter_plan()["bin_ranges"] >= 2


def test_cwb_exact_binning_small_config(cwb):
    """n = 10,000, p = 10 FP64, exact binning (n* = number of unique values), M = 500."""
    data = S.sim_small_exact(seed=0)
    specs = [dict(feature=j, n_bins=0) for j in range(10)]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=500)
    assert model.learner_info(0).nstar == 10_000


def test_cwb_binomial(cwb):
    data = S.sim_binomial_hybrid(seed=24, n=30_000, p=8, n_informative=4)
    specs = [dict(feature=j, n_bins=-1) for j in range(8)]
    run_pair(cwb, data.X, data.y, specs, M=150, loss=1)


def test_cwb_weights_and_mixed_learners(cwb):
    data = S.additive_regression(12_345, 5, 3, seed=25, dtype=np.float64)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.2, 3.0, size=data.n)
    specs = [dict(feature=j, n_bins=-1) for j in range(5)] + [dict(feature=j, n_bins=-1, type=1) for j in range(5)]
    specs += [dict(feature=1, n_bins=50, degree=2, n_knots=10, df=4.0)]
    run_pair(cwb, data.X, data.y, specs, M=120, w=w)


def _categorical_specs(p_num, classes, *, binary_of=()):
    specs = [dict(feature=j, n_bins=-1) for j in range(p_num)]
    for t, c in enumerate(classes):
        specs.append(dict(type=O.BL_CATEGORICAL, feature=p_num + t, n_knots=c, df=min(5.0, c - 0.5)))
    for t in binary_of:
        specs += [dict(type=O.BL_CATEGORICAL_BINARY, feature=p_num + t, n_knots=classes[t], level=k)
                  for k in range(classes[t])]
    return specs


def test_categorical_ridge_and_binary_l2(cwb):
    """Ridge and binary categorical learners (App. B.1) beside P-splines, L2, uint8 bins."""
    classes = [6, 13, 40, 3]
    data = S.mixed_categorical(20_011, 3, classes, seed=31, n_informative_cat=2)
    specs = _categorical_specs(3, classes, binary_of=(1,))
    model, ref = run_pair(cwb, data.X, data.y, specs, M=150)
    # a ridge learner and the binary learners of one feature share that feature's class binning
    info = [model.learner_info(k) for k in range(len(specs))]
    assert info[4].nstar == 13 and info[4].d == 13
    assert {info[k].binning for k in range(7, 7 + 13)} == {info[4].binning}
    assert all(info[k].d == 1 for k in range(7, 7 + 13))


def test_categorical_fixed_lambda_binomial_uint16(cwb):
    """Binomial loss, a ridge learner with a fixed lambda, and P-splines at n* = 1500 (uint16)."""
    classes = [9, 64]
    data = S.mixed_categorical(60_000, 4, classes, seed=32, binomial=True)
    specs = [dict(feature=j, n_bins=1500) for j in range(4)]
    specs += [dict(type=O.BL_CATEGORICAL, feature=4, n_knots=9, df=0.0, lam=250.0),
              dict(type=O.BL_CATEGORICAL, feature=5, n_knots=64, df=12.0)]
    run_pair(cwb, data.X, data.y, specs, M=120, loss=1)


def test_categorical_acwb_and_hcwb(cwb):
    classes = [7, 20]
    data = S.mixed_categorical(30_000, 3, classes, seed=33, binomial=True)
    rng = np.random.default_rng(5)
    val = (rng.random(data.n) < 0.25).astype(np.uint8)
    specs = _categorical_specs(3, classes, binary_of=(0,))
    run_pair(cwb, data.X, data.y, specs, M=100, loss=1, opt=1, gamma=0.01)
    run_pair(cwb, data.X, data.y, specs, M=160, loss=1, opt=2, gamma=0.01, patience=3, val_mask=val)


def test_categorical_lookup_is_the_class_code(cwb):
    """Each class is one design point: the bin index of a categorical learner is the code itself
    (in the caller's row order, also with HCWB's train-first row permutation), and the learner's
    design is the dummy matrix (ridge) or the class indicator (binary)."""
    data = S.mixed_categorical(5_000, 1, [11], seed=35)
    codes = data.X[1].astype(np.int32)
    val = (np.random.default_rng(2).random(data.n) < 0.3).astype(np.uint8)
    for opt, vm in ((cwb.OPT_CWB, None), (cwb.OPT_HCWB, val)):
        m = cwb.Model(data.X, data.y, [cwb.learner(1, type=cwb.BL_CATEGORICAL, n_knots=11, df=4.0),
                                       cwb.learner(1, type=cwb.BL_CATEGORICAL_BINARY, n_knots=11, level=7)],
                      opt=opt, val_mask=vm, device=0)
        for k in (0, 1):
            assert np.array_equal(m.bin_index(k), codes)
        info = m.learner_info(0)
        assert (info.nstar, info.d, info.xmin, info.xmax) == (11, 11, 0.0, 10.0)
        assert m.learner_info(1).d == 1 and m.learner_info(1).binning == info.binning
        # Z^T W Z = diag(n_k) on the fitting rows, P = diag(1 / (n_k + lambda)) (App. B.1)
        rows = codes if vm is None else codes[vm == 0]
        nk = np.bincount(rows, minlength=11).astype(np.float64)
        G, P = m.matrices(0)
        np.testing.assert_array_equal(G, np.diag(nk))
        np.testing.assert_allclose(P, np.diag(1.0 / (nk + info.lam)), rtol=1e-13)
        assert abs(np.sum(nk / (nk + info.lam)) - 4.0) < 1e-9      # df1 closed form
        G1, P1 = m.matrices(1)
        np.testing.assert_allclose(P1, np.diag([1.0 / G1[0, 0]]), rtol=1e-13)
        m.free()


def test_categorical_invalid_codes_are_rejected(cwb):
    data = S.mixed_categorical(2_000, 1, [5], seed=34)
    for bad in (2.5, -1.0, 5.0):
        X = data.X.copy()
        X[1, 17] = bad
        with pytest.raises(cwb.CwbError) as e:
            cwb.Model(X, data.y, [cwb.learner(1, type=cwb.BL_CATEGORICAL, n_knots=5)], device=0)
        assert e.value.status == 1 and "class code" in str(e.value)
    with pytest.raises(cwb.CwbError):
        cwb.Model(data.X, data.y, [cwb.learner(1, type=cwb.BL_CATEGORICAL_BINARY, n_knots=5, level=5)], device=0)
    with pytest.raises(cwb.CwbError):
        cwb.Model(data.X, data.y, [cwb.learner(1, type=cwb.BL_CATEGORICAL, n_knots=65)], device=0)


def test_duplicate_learners_tie_to_lowest_index(cwb):
    data = S.additive_regression(9_000, 3, 3, seed=26, dtype=np.float32)
    specs = [dict(feature=0, n_bins=-1), dict(feature=1, n_bins=-1), dict(feature=1, n_bins=-1),
             dict(feature=2, n_bins=-1)]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=60)
    k_sel, _, _ = model.trace()
    assert not np.any(k_sel == 2)


def test_resumed_fit_equals_single_fit(cwb):
    data = S.additive_regression(15_000, 5, 4, seed=27, dtype=np.float32)
    specs = [dict(feature=j, n_bins=-1) for j in range(5)]
    a = cwb.Model(data.X, data.y, _specs_to_gpu(cwb, specs), iterations=80, device=0)
    a.fit(30)
    a.fit(17)
    a.fit(33)
    ref = O.fit(data.X.astype(np.float64), data.y.astype(np.float64), specs, iterations=80)
    k_sel, _, _ = a.trace()
    check_sequences(k_sel, ref)
    check_coefficients(a.all_coefficients(0, dmax=ref.dmax), ref.theta_f)
    assert rel_err(a.fitted(), ref.f) <= REL_TOL


def test_fit_resumes_after_reading_fitted_values(cwb):
    """Reading the fitted values applies the last update without forming residuals; the next row
    pass must still take a valid fixed-point scale (the bound grows by that update), for the L2 and
    the binomial loss, with and without observation weights."""
    for loss, w_on in [(0, False), (0, True), (1, False)]:
        data = S.additive_regression(20_000, 5, 4, seed=41 + loss, dtype=np.float32)
        y = data.y if loss == 0 else (data.eta > np.median(data.eta)).astype(np.float32)
        w = np.random.default_rng(5).uniform(0.5, 2.0, size=data.n) if w_on else None
        specs = [dict(feature=j, n_bins=-1) for j in range(5)]
        a = cwb.Model(data.X, y, _specs_to_gpu(cwb, specs), loss=loss, w=w, iterations=60, device=0)
        for chunk in (7, 13, 20, 20):
            a.fit(chunk)
            a.fitted()
            a.all_coefficients(0)
        ref = O.fit(data.X.astype(np.float64), y.astype(np.float64), specs, loss=loss, w=w, iterations=60)
        k_sel, _, _ = a.trace()
        if check_sequences(k_sel, ref) < 0:
            check_coefficients(a.all_coefficients(0, dmax=ref.dmax), ref.theta_f)
            assert rel_err(a.fitted(), ref.f) <= REL_TOL
        a.free()


@pytest.mark.parametrize("direct", ["1", "0"])
def test_residual_getter_matches_oracle(cwb, monkeypatch, direct):
    """cwb_get_residuals returns w r of the last iteration: with the row pass writing fixed point
    (the default for plain CWB) and with the conversion inside the scatter (CWB_DIRECT_Q=0), it equals
    the oracle's y - f after M - 1 iterations; the fit itself matches the oracle either way."""
    monkeypatch.setenv("CWB_DIRECT_Q", direct)
    data = S.additive_regression(30_001, 6, 4, seed=43, dtype=np.float32)
    specs = [dict(feature=j, n_bins=-1) for j in range(6)]
    M = 25
    model, ref = run_pair(cwb, data.X, data.y, specs, M=M, check_predict=False)
    r = model.residuals(0)
    prev = O.fit(data.X.astype(np.float64), data.y.astype(np.float64), specs, iterations=M - 1)
    r_ref = data.y.astype(np.float64) - prev.f
    assert rel_err(r, r_ref) <= REL_TOL, rel_err(r, r_ref)
    model.free()


# ------------------------------------------------------------------ ACWB / HCWB

def test_acwb_l2(cwb):
    data = S.additive_regression(25_000, 6, 4, seed=28, dtype=np.float32)
    specs = [dict(feature=j, n_bins=-1) for j in range(6)]
    run_pair(cwb, data.X, data.y, specs, M=120, opt=1, gamma=0.05)


def test_acwb_binomial_uint16(cwb):
    data = S.sim_binomial_hybrid(seed=29, n=70_000, p=10, n_informative=4)
    specs = [dict(feature=j, n_bins=300) for j in range(10)]
    run_pair(cwb, data.X, data.y, specs, M=100, opt=1, loss=1, gamma=0.01)


def test_hcwb_binomial_switches_like_oracle(cwb):
    data = S.sim_binomial_hybrid(seed=30, n=40_000, p=8, n_informative=3)
    specs = [dict(feature=j, n_bins=-1) for j in range(8)]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=200, opt=2, loss=1, gamma=0.3, nu=0.3, patience=3,
                          val_mask=data.val_mask)
    assert ref.switch_iter > 0


def test_hcwb_patience_zero_starts_with_cwb(cwb):
    data = S.sim_binomial_hybrid(seed=31, n=20_000, p=5, n_informative=3)
    specs = [dict(feature=j, n_bins=-1) for j in range(5)]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=40, opt=2, loss=1, gamma=0.05, patience=0,
                          val_mask=data.val_mask)
    assert ref.switch_iter == 1


# ------------------------------------------------------------------ edge cases and errors

def test_many_learners_argmin_over_several_passes(cwb):
    """K = 300 learners (P-spline and linear per feature): the argmin's per-lane passes over the
    criteria (128 per pass) and the solve grid of K CTAs; ACWB puts a second channel through it."""
    data = S.additive_regression(3_001, 150, 6, seed=41, dtype=np.float32)
    # informative features last, so the winners sit in the argmin's second pass (128..255)
    specs = [dict(feature=j, n_bins=40, n_knots=6, df=4.0) for j in reversed(range(150))]
    specs += [dict(feature=j, n_bins=40, type=1) for j in reversed(range(150))]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=30)
    assert ref.k_sel.min() >= 128
    run_pair(cwb, data.X, data.y, specs, M=20, opt=1, gamma=0.01)


def test_heavily_skewed_bins_use_fp32_histograms(cwb):
    """A feature with 40 % of its rows at one value puts more than 8192 rows of one cluster into one
    bin: the plan drops the fixed-point histograms for FP32 atomics with compensated cross-cluster
    sums, which must meet the same parity bar."""
    data = S.additive_regression(2_000_000, 4, 3, seed=43, dtype=np.float32)
    X = data.X.copy()
    spike = np.random.default_rng(7).random(X.shape[1]) < 0.4
    X[0, spike] = 0.5
    specs = [dict(feature=j, n_bins=-1) for j in range(4)]
    model, _ = run_pair(cwb, X, data.y, specs, M=15)
    assert model.scatter_plan()["int_fixed_point"] == 0


def test_tiny_problem_linear_learners(cwb):
    X = np.array([[0.0, 1.0, 2.0, 3.0, 5.0], [1.0, -1.0, 0.5, 0.25, 2.0]])
    y = np.array([1.0, 2.0, 2.5, 4.0, 7.0])
    specs = [dict(feature=0, type=1, n_bins=0), dict(feature=1, type=1, n_bins=0)]
    run_pair(cwb, X, y, specs, M=25, nu=0.5)


def test_invalid_inputs_are_rejected(cwb):
    X = np.ones((2, 100), dtype=np.float32)
    y = np.zeros(100, dtype=np.float32)
    with pytest.raises(cwb.CwbError) as e:
        cwb.Model(X, y, [cwb.learner(0)], device=0)
    assert e.value.status == 1 and "constant" in str(e.value)
    Xr = np.random.default_rng(0).random((2, 100)).astype(np.float32)
    with pytest.raises(cwb.CwbError):
        cwb.Model(Xr, y + 2, [cwb.learner(0)], loss=cwb.LOSS_BINOMIAL, device=0)
    with pytest.raises(cwb.CwbError):
        cwb.Model(Xr, y, [cwb.learner(0)], opt=cwb.OPT_HCWB, device=0)
    with pytest.raises(cwb.CwbError):
        cwb.Model(Xr, y, [cwb.learner(5)], device=0)


# ------------------------------------------------------------------ full-size workload, sampled

def test_full_size_binned_l2_first_iterations(cwb):
    """n = 1,000,000, p = 50, n* = 1000 (uint16): the first 12 iterations against the oracle."""
    data = S.sim_binned_l2(seed=1)
    specs = [dict(feature=j, n_bins=-1) for j in range(50)]
    run_pair(cwb, data.X, data.y, specs, M=12, check_predict=False)


def test_full_size_hcwb_binomial_first_iterations(cwb):
    """n = 2,000,000, p = 200 (U[0,1] and N(0,1)), binomial, ACWB with the hybrid switch, 20 % validation
    rows, n* = 1414 (uint16): the first 6 iterations (two fits each) against the oracle."""
    data = S.sim_binomial_hybrid(seed=2)
    specs = [dict(feature=j, n_bins=1414) for j in range(200)]
    run_pair(cwb, data.X, data.y, specs, M=6, loss=1, opt=2, nu=0.1, gamma=0.001, patience=5,
             val_mask=data.val_mask, check_predict=False)


def test_full_size_hcwb_switch_at_first_iteration(cwb):
    """n = 2,000,000, p = 200, n* = 1414, binomial HCWB with patience 0: the switch to CWB on all rows
    happens at iteration 1, so the CWB phase (all-row caches, one-channel plan) runs at full size."""
    data = S.sim_binomial_hybrid(seed=2)
    specs = [dict(feature=j, n_bins=1414) for j in range(200)]
    model, ref = run_pair(cwb, data.X, data.y, specs, M=4, loss=1, opt=2, nu=0.1, gamma=0.001, patience=0,
                          val_mask=data.val_mask, check_predict=False)
    assert ref.switch_iter == 1
    model.free()


# ------------------------------------------------------------------ criterion precision at near ties

def _near_tie_data(n, moved, seed):
    """Feature 1 is a copy of feature 0 with `moved` rows shifted by one bin width (the grid and the
    range stay the same), so the two learners' SSEs differ by a tiny relative amount while the
    winner explains most of r^T r; feature 2 is noise."""
    rng = np.random.default_rng(seed)
    x0 = rng.random(n)
    y = 2.0 * np.sin(2 * np.pi * x0) + rng.normal(size=n)
    nstar = int(np.floor(np.sqrt(n)))
    h = (x0.max() - x0.min()) / (nstar - 1)
    x1 = x0.copy()
    idx = rng.choice(np.flatnonzero((x0 > x0.min() + 2 * h) & (x0 < x0.max() - 2 * h)), size=moved, replace=False)
    x1[idx] += h * np.where(rng.random(moved) < 0.5, -1.0, 1.0)
    return np.stack([x0, x1, rng.random(n)]), y


@pytest.mark.parametrize("moved,seed", [(1, 0), (1, 1), (1, 3), (2, 2), (4, 0), (8, 1)])
def test_near_tie_picks_the_oracle_learner(cwb, moved, seed):
    """The criterion separates learners whose first-iteration SSE gap, relative to the SSE, lies between
    1e-9 and 1e-6 while the winner explains about twice r^T r minus its SSE (|Q| / SSE ~ 1.9): the
    GPU's sequence must equal the oracle's with no teacher forcing."""
    X, y = _near_tie_data(200_000, moved, seed)
    specs = [dict(feature=j, n_bins=-1, df=5.0) for j in range(3)]
    M = 6
    ref = O.fit(X, y, specs, iterations=M)
    gaps = (ref.sse_second - ref.sse_best) / ref.sse_best
    r0 = y - ref.offset
    assert 1e-9 < gaps[0] < 1e-6 and (r0 @ r0 - ref.sse_best[0]) / ref.sse_best[0] > 0.05
    model = cwb.Model(np.ascontiguousarray(X.astype(np.float32)), y.astype(np.float32), _specs_to_gpu(cwb, specs),
                      nu=0.1, iterations=M, device=0)
    model.fit(M)
    k_sel, _, _ = model.trace()
    above = gaps > 1e-9
    np.testing.assert_array_equal(k_sel[above], ref.k_sel[above])
    model.free()


# ------------------------------------------------------------------ the persistent iteration kernel (opt-in)

@pytest.mark.parametrize("case", ["l2_uint16", "l2_weights_f64_uint8", "binomial", "two_groups"])
def test_persistent_path_matches_oracle(cwb, monkeypatch, case):
    """CWB_ITER_MODE=persistent runs plain CWB as one cooperative kernel (row pass folded into the
    scatter, fixed-point scale from a bound, exact int64 sums, float-float solve); same oracle
    tolerances as the kernel path."""
    monkeypatch.setenv("CWB_ITER_MODE", "persistent")
    w = None
    if case == "l2_uint16":
        data = S.additive_regression(150_001, 8, 5, seed=71, dtype=np.float32)
        specs = [dict(feature=j, n_bins=-1) for j in range(8)]
        kw = dict(M=50)
    elif case == "l2_weights_f64_uint8":
        data = S.additive_regression(40_000, 6, 4, seed=72, dtype=np.float64)
        specs = [dict(feature=j, n_bins=200, df=4.0) for j in range(6)]
        w = np.random.default_rng(3).uniform(0.5, 2.0, size=40_000)
        kw = dict(M=40, nu=0.3)
    elif case == "binomial":
        data = S.sim_binomial_hybrid(seed=73, n=120_000, p=7, n_informative=4)
        specs = [dict(feature=j, n_bins=-1) for j in range(7)]
        kw = dict(M=40, loss=1)
    else:
        data = S.additive_regression(90_000, 40, 6, seed=74, dtype=np.float32)
        specs = [dict(feature=j, n_bins=-1) for j in range(40)]
        kw = dict(M=30)
    model, ref = run_pair(cwb, data.X, data.y, specs, w=w, **kw)
    assert model.scatter_plan()["persistent"] == 1
    model.free()
