"""Row-sharded fits (cwb_shard_*) on one GPU: shards of one fit emulated in one process.

binMatVec sums over rows (Algorithm 2), so a fit whose rows are split into shards, with the
histograms added across shards, is the same fit as the unsharded one.  Checks: every shard selects
the same learners and holds bit-identical coefficients (they solve on the same integer totals); the
selections, coefficients and fitted values match the FP64 oracle on all rows; the sharded and the
unsharded GPU fits pick the same learners.
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


def _gpu_specs(cwb, specs):
    return [cwb.learner(s["feature"], type=s.get("type", 0), n_bins=s.get("n_bins", -1), df=s.get("df", 5.0))
            for s in specs]


def _sharded(cwb, X, y, specs, parts, M, loss):
    ranges = cwb.split_rows(X.shape[1], parts)
    fit = cwb.ShardedFit([(X[:, a:b], y[a:b]) for a, b in ranges], _gpu_specs(cwb, specs), loss=loss, nu=0.1,
                         iterations=M)
    fit.fit(M)
    return fit, ranges


@pytest.mark.parametrize("loss", [0, 1])
@pytest.mark.parametrize("parts,n,n_bins", [(2, 60_000, -1), (3, 60_001, -1), (3, 40_003, 200)])
def test_shards_match_the_oracle_and_each_other(cwb, loss, parts, n, n_bins):
    M = 50
    data = S.additive_regression(n, 5, 3, seed=31 + parts, dtype=np.float32)
    y = data.y
    if loss == 1:
        y = (data.eta > np.median(data.eta)).astype(np.float32)
    specs = [dict(feature=j, n_bins=n_bins) for j in range(5)] + [dict(feature=0, type=1, n_bins=n_bins)]
    fit, ranges = _sharded(cwb, data.X, y, specs, parts, M, loss)
    ref = O.fit(data.X.astype(np.float64), y.astype(np.float64), specs, loss=loss, nu=0.1, iterations=M, patience=0)
    traces = [s.model.trace()[0] for s in fit.shards]
    thetas = [s.model.all_coefficients(0, dmax=ref.dmax) for s in fit.shards]
    for t, th in zip(traces[1:], thetas[1:]):
        np.testing.assert_array_equal(t, traces[0])
        np.testing.assert_array_equal(th, thetas[0])
    assert check_sequences(traces[0], ref) == -1
    check_coefficients(thetas[0], ref.theta_f)
    f = np.concatenate([s.model.fitted() for s in fit.shards])
    assert rel_err(f, ref.f) <= REL_TOL, rel_err(f, ref.f)
    for s in fit.shards:
        assert abs(s.model.offset - ref.offset) <= 1e-12 * max(1.0, abs(ref.offset))
    # the unsharded GPU fit of the same rows picks the same learners
    whole = cwb.Model(data.X, y, _gpu_specs(cwb, specs), loss=loss, nu=0.1, iterations=M, patience=0, device=0)
    whole.fit(M)
    np.testing.assert_array_equal(whole.trace()[0], traces[0])
    # predictions of any shard are the model's predictions
    Xn = np.ascontiguousarray(data.X[:, :2000])
    pred_ref = O.predict(Xn.astype(np.float64), specs, [data.X[s["feature"]].min() for s in specs],
                         [data.X[s["feature"]].max() for s in specs], ref.theta_f, ref.offset)
    assert rel_err(fit.shards[-1].model.predict(Xn), pred_ref) <= REL_TOL
    whole.free()
    fit.free()


def test_shard_rejects_rows_outside_the_global_range_and_cwb_fit(cwb):
    data = S.additive_regression(4000, 2, 2, seed=5, dtype=np.float32)
    specs = [cwb.learner(0), cwb.learner(1)]
    X0 = np.ascontiguousarray(data.X[:, :2000])
    lo = X0.min(axis=1).astype(np.float64)
    hi = X0.max(axis=1).astype(np.float64)
    cfg = cwb.binding.cwb_config(loss=0, opt=0, nu=0.1, gamma=0.0, iterations=5, patience=0, val_mask=None,
                                 stream=None, device=0)
    y0 = np.ascontiguousarray(data.y[:2000])
    with pytest.raises(cwb.CwbError):
        cwb.cwb_shard_create(cfg, X0, 0, 2000, 2, y0, specs, 0, 4000, lo + 0.01, hi)
    with pytest.raises(cwb.CwbError):          # the global row count cannot be below the shard's own
        cwb.cwb_shard_create(cfg, X0, 0, 2000, 2, y0, specs, 0, 1999, lo, hi)
    h = cwb.cwb_shard_create(cfg, X0, 0, 2000, 2, y0, specs, 0, 4000, lo, hi)
    m = cwb.Model._adopt(h, 2000, 2, specs)
    with pytest.raises(cwb.CwbError):
        m.fit(3)
    m.free()


def test_device_exchange_equals_host_exchange(cwb):
    """The exchange through device buffers (CUDA tensors on the current stream, what a NCCL all-reduce
    moves) gives the same fit as the exchange through host arrays, bit for bit."""
    M = 30
    data = S.additive_regression(50_001, 4, 3, seed=37, dtype=np.float32)
    specs = [dict(feature=j, n_bins=-1) for j in range(4)]
    parts = [(data.X[:, a:b], data.y[a:b]) for a, b in cwb.split_rows(data.n, 2)]
    fits = []
    for dev in (False, True):
        fit = cwb.ShardedFit(parts, _gpu_specs(cwb, specs), nu=0.1, iterations=M, device_exchange=dev)
        fit.fit(M)
        fits.append(fit)
    for a, b in zip(fits[0].shards, fits[1].shards):
        np.testing.assert_array_equal(a.model.trace()[0], b.model.trace()[0])
        np.testing.assert_array_equal(a.model.all_coefficients(0), b.model.all_coefficients(0))
        np.testing.assert_array_equal(a.model.fitted(), b.model.fitted())
    for f in fits:
        f.free()
