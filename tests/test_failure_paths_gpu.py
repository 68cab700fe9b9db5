"""Failure paths on the GPU without faulting it: a device-side wait that runs out returns an error
status (the kernel ends normally and the GPU stays usable), a diverging fit reports CWB_ENUMERIC,
non-finite targets are rejected at create."""
import numpy as np
import pytest

import synthetic_inputs as S
from oracle import oracle as O
from parity_util import REL_TOL, rel_err

pytestmark = pytest.mark.gpu

CWB_ENUMERIC, CWB_ETIMEOUT, CWB_EINVAL = 4, 5, 1


@pytest.fixture(scope="module")
def cwb():
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as pkg
    return pkg


def test_ring_wait_that_runs_out_reports_timeout_and_the_gpu_stays_usable(cwb, monkeypatch):
    """A scatter tile whose copies are never issued (CWB_WITHHOLD_TILE) leaves its ring stage's barrier
    incomplete: the waits on it run out after CWB_WAIT_CYCLES, the kernel drains the copies it did
    issue and returns, and the next synchronising call reports CWB_ETIMEOUT."""
    data = S.additive_regression(60_000, 6, 4, seed=81, dtype=np.float32)
    learners = [cwb.learner(j) for j in range(6)]
    monkeypatch.setenv("CWB_WAIT_CYCLES", str(200_000_000))      # about 0.1 s
    monkeypatch.setenv("CWB_WITHHOLD_TILE", "3")
    monkeypatch.setenv("CWB_ITER_MODE", "kernels")
    bad = cwb.Model(data.X, data.y, learners, iterations=5, device=0)     # setup waits keep the default limit
    for v in ("CWB_WAIT_CYCLES", "CWB_WITHHOLD_TILE", "CWB_ITER_MODE"):
        monkeypatch.delenv(v)
    bad.fit(2)
    with pytest.raises(cwb.CwbError) as info:
        bad.synchronize()
    assert info.value.status == CWB_ETIMEOUT
    bad.free()
    # the next model on the same GPU fits correctly
    M = 30
    good = cwb.Model(data.X, data.y, learners, iterations=M, device=0)
    good.fit(M)
    good.synchronize()
    ref = O.fit(data.X.astype(np.float64), data.y.astype(np.float64), [dict(feature=j, n_bins=-1) for j in range(6)],
                iterations=M)
    k_sel, _, _ = good.trace()
    np.testing.assert_array_equal(k_sel, ref.k_sel)
    assert rel_err(good.fitted(), ref.f) <= REL_TOL
    good.free()


def test_diverging_fit_reports_enumeric(cwb):
    data = S.additive_regression(20_000, 4, 3, seed=82, dtype=np.float32)
    # a step of 1e38 overflows FP32 at the first update
    model = cwb.Model(data.X, data.y, [cwb.learner(j) for j in range(4)], nu=1e38, iterations=4, device=0)
    model.fit(4)
    with pytest.raises(cwb.CwbError) as info:
        model.synchronize()
    assert info.value.status == CWB_ENUMERIC
    model.free()


def test_non_finite_targets_are_rejected(cwb):
    data = S.additive_regression(5_000, 3, 2, seed=83, dtype=np.float32)
    y = data.y.copy()
    y[17] = np.inf
    with pytest.raises(cwb.CwbError) as info:
        cwb.Model(data.X, y, [cwb.learner(j) for j in range(3)], device=0)
    assert info.value.status == CWB_EINVAL and "finite" in str(info.value)
