"""Many fits on one GPU: the autotuner, batched graphs and the fit server (GPU).

Every fit must give the same result however it is scheduled: alone through cwb_fit, as one branch of a
batch graph, or interleaved with other requests in the server; and it must match the FP64 oracle.
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


def _fit_specs():
    """Uneven fits: uint8 and uint16 indices, different p, df and nu (a small CV x grid)."""
    out = []
    for i, (n, p, df, nu) in enumerate([(9_001, 7, 5.0, 0.1), (40_000, 12, 4.0, 0.3), (3_000, 5, 6.0, 0.05),
                                        (120_001, 20, 5.0, 0.2), (70_000, 3, 8.0, 0.1), (20_000, 30, 5.0, 0.1)]):
        data = S.additive_regression(n, p, min(p, 5), seed=100 + i, dtype=np.float32)
        out.append((data, [dict(feature=j, n_bins=-1, df=df) for j in range(p)], nu))
    return out


def _learners(cwb, specs):
    return [cwb.learner(s["feature"], n_bins=s["n_bins"], df=s["df"]) for s in specs]


def _state(model, K):
    k_sel, _, _ = model.trace()
    return np.asarray(k_sel), model.all_coefficients(0, dmax=24), model.fitted()


def test_autotuned_plan_keeps_parity(cwb):
    data = S.additive_regression(60_007, 12, 6, seed=31, dtype=np.float32)
    specs = [dict(feature=j, n_bins=-1) for j in range(12)]
    M = 60
    for objective in (0, 1):
        model = cwb.Model(data.X, data.y, _learners(cwb, [dict(s, df=5.0) for s in specs]), nu=0.1, iterations=M,
                          device=0)
        us = model.autotune(objective=objective, trials=3)
        assert us > 0
        model.fit(M)
        ref = O.fit(data.X.astype(np.float64), data.y.astype(np.float64), specs, nu=0.1, iterations=M)
        k_sel, _, _ = model.trace()
        assert check_sequences(k_sel, ref) < 0
        check_coefficients(model.all_coefficients(0, dmax=ref.dmax), ref.theta_f)
        assert rel_err(model.fitted(), ref.f) <= REL_TOL
        model.free()


def test_batch_equals_individual_fits(cwb, monkeypatch):
    M = 70                                  # two graph launches of 32 and six single iterations
    fits = _fit_specs()
    alone, alone_persistent = [], []
    for data, specs, nu in fits:
        # the batch runs the three-kernel path: alone on the same path it must agree bit for bit;
        # alone on the persistent path (opt-in for plain CWB) within the parity tolerance
        m = cwb.Model(data.X, data.y, _learners(cwb, specs), nu=nu, iterations=M, device=0)
        m.fit(M)
        alone.append(_state(m, M))
        m.free()
        monkeypatch.setenv("CWB_ITER_MODE", "persistent")
        m = cwb.Model(data.X, data.y, _learners(cwb, specs), nu=nu, iterations=M, device=0)
        monkeypatch.delenv("CWB_ITER_MODE")
        m.fit(M)
        alone_persistent.append(_state(m, M))
        m.free()
    for (k_a, th_a, f_a), (k_p, th_p, f_p) in zip(alone, alone_persistent):
        np.testing.assert_array_equal(k_a, k_p)
        assert rel_err(th_p, th_a) <= REL_TOL
        assert rel_err(f_p, f_a) <= REL_TOL
    models = [cwb.Model(data.X, data.y, _learners(cwb, specs), nu=nu, iterations=M, device=0) for data, specs, nu in fits]
    batch = cwb.Batch(models, iters_per_launch=32)
    batch.fit(M)
    batch.synchronize()
    for m, (k_ref, th_ref, f_ref) in zip(models, alone):
        k, th, f = _state(m, M)
        np.testing.assert_array_equal(k, k_ref)
        assert rel_err(th, th_ref) <= 1e-12
        assert rel_err(f, f_ref) <= 1e-12
    # a batch keeps going: 10 more iterations equal a single 80-iteration fit
    batch.fit(10)
    batch.synchronize()
    data, specs, nu = fits[1]
    m80 = cwb.Model(data.X, data.y, _learners(cwb, specs), nu=nu, iterations=80, device=0)
    m80.fit(80)
    k, th, f = _state(models[1], 80)
    k_ref, th_ref, f_ref = _state(m80, 80)
    np.testing.assert_array_equal(k, k_ref)
    assert rel_err(th, th_ref) <= 1e-12
    batch.free()
    for m in models:
        m.free()


def test_server_results_equal_alone_and_oracle(cwb):
    M = 45
    fits = _fit_specs()
    alone = []
    for data, specs, nu in fits:
        m = cwb.Model(data.X, data.y, _learners(cwb, specs), nu=nu, iterations=M, device=0)
        m.fit(M)
        alone.append(_state(m, M))
        m.free()
    # a budget that holds about two of these fits at a time: requests queue and are admitted as memory frees
    srv = cwb.Server(hbm_budget_bytes=320 << 20, device=0, max_active=8, slice_iterations=8)
    ids = [srv.submit(data.X, data.y, _learners(cwb, specs), nu=nu, iterations=M) for data, specs, nu in fits]
    peak_active, done = 0, []
    while len(done) < len(ids):
        done += srv.poll(wait=True)
        st = srv.stats()
        peak_active = max(peak_active, st["active"])
        assert st["bytes_in_use"] <= st["budget"]
    assert sorted(done) == sorted(ids)
    assert 1 <= peak_active < len(ids)      # admission by footprint kept some requests waiting
    st = srv.stats()
    assert st["admitted"] == len(ids) and st["completed"] == len(ids) and st["active"] == 0
    for rid, (k_ref, th_ref, f_ref), (data, specs, nu) in zip(ids, alone, fits):
        m = srv.take(rid)
        k, th, f = _state(m, M)
        np.testing.assert_array_equal(k, k_ref)
        assert rel_err(th, th_ref) <= REL_TOL
        assert rel_err(f, f_ref) <= REL_TOL
        if rid == ids[3]:                   # one of them also against the FP64 oracle
            ref = O.fit(data.X.astype(np.float64), data.y.astype(np.float64), specs, nu=nu, iterations=M)
            assert check_sequences(k, ref) < 0
            check_coefficients(m.all_coefficients(0, dmax=ref.dmax), ref.theta_f)
        m.free()
    srv.free()


def test_server_rejects_requests_above_the_budget(cwb):
    data = S.additive_regression(50_000, 10, 3, seed=7, dtype=np.float32)
    srv = cwb.Server(hbm_budget_bytes=1 << 20, device=0)
    with pytest.raises(cwb.CwbError):
        srv.submit(data.X, data.y, [cwb.learner(j) for j in range(10)], iterations=10)
    srv.free()


def test_batched_fit_specs_match_the_oracle(cwb):
    """Fits drawn from the batched workload's seeded specs (the smaller ones), advanced as one batch with
    autotuned plans, each against the FP64 oracle."""
    specs = [s for s in S.batched_fit_specs(count=512) if s["n"] <= 20_000][:4]
    assert len(specs) == 4
    M = 150
    models, refs = [], []
    for sp in specs:
        d = S.request_dataset(sp)
        lspecs = [dict(feature=j, n_bins=-1, df=sp["df"]) for j in range(sp["p"])]
        m = cwb.Model(d.X, d.y, _learners(cwb, lspecs), nu=sp["nu"], iterations=M, device=0)
        m.autotune(objective=1, trials=2)
        models.append(m)
        refs.append((O.fit(d.X.astype(np.float64), d.y.astype(np.float64), lspecs, nu=sp["nu"], iterations=M), d))
    batch = cwb.Batch(models, iters_per_launch=32)
    batch.fit(M)
    batch.synchronize()
    for m, (ref, d) in zip(models, refs):
        k_sel, _, _ = m.trace()
        assert check_sequences(k_sel, ref) < 0
        check_coefficients(m.all_coefficients(0, dmax=ref.dmax), ref.theta_f)
        assert rel_err(m.fitted(), ref.f) <= REL_TOL
    batch.free()
    for m in models:
        m.free()


def test_create_many_equals_single_creates(cwb):
    """cwb_create_many (the setups of several fits overlapped on host threads and streams) returns the
    models that separate cwb_create calls return: the same fits, bit for bit; a bad request is reported
    by its index and leaves no model behind."""
    M = 40
    fits = _fit_specs()
    reqs = [dict(X=d.X, y=d.y, learners=_learners(cwb, specs), nu=nu, iterations=M) for d, specs, nu in fits]
    many = cwb.Model.create_many(reqs, threads=4)
    for (d, specs, nu), m in zip(fits, many):
        one = cwb.Model(d.X, d.y, _learners(cwb, specs), nu=nu, iterations=M, device=0)
        one.fit(M)
        m.fit(M)
        np.testing.assert_array_equal(m.trace()[0], one.trace()[0])
        np.testing.assert_array_equal(m.all_coefficients(0, dmax=24), one.all_coefficients(0, dmax=24))
        np.testing.assert_array_equal(m.fitted(), one.fitted())
        one.free()
        m.free()
    bad = list(reqs[:3])
    bad[1] = dict(bad[1], learners=[cwb.learner(99)])          # a feature that does not exist
    with pytest.raises(cwb.CwbError, match="request 1"):
        cwb.Model.create_many(bad, threads=2)
