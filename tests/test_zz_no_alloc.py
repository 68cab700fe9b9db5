"""cwb_predict_noalloc: predictions from host buffers without any device allocation.

Callers that cannot allocate device memory while predicting (stream capture,
allocation-free serving loops, fixed device-memory budgets) use this entry point;
it stages the inputs through the library's fixed scratch array instead of
cudaMalloc.  Its output must equal cwb_predict's for the same host inputs.  The
file is named so pytest collects it last; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synthetic_inputs as S
from parity_util import REL_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cwb():
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as pkg
    return pkg


def test_noalloc_predict_matches_predict_twice(cwb):
    data = S.additive_regression(30_000, 6, 4, seed=41, dtype=np.float32)
    model = cwb.Model(data.X, data.y, [cwb.learner(j) for j in range(6)], nu=0.1, iterations=60, device=0)
    model.fit(60)
    rng = np.random.default_rng(42)
    for call in range(2):
        n_new = 7_001 + call * 3_000
        Xn = np.ascontiguousarray(rng.random((6, n_new)).astype(np.float32 if call == 0 else np.float64))
        ref = model.predict(Xn)
        out = np.full(n_new, np.nan, dtype=np.float32)
        cwb.cwb_predict_noalloc(model.handle, Xn, 0 if call == 0 else 1, n_new, out)
        assert np.isfinite(out).all()
        assert rel_err(out, ref) <= REL_TOL
    model.free()


def test_noalloc_predict_rejects_oversized_requests(cwb):
    data = S.additive_regression(5_000, 3, 2, seed=43, dtype=np.float32)
    model = cwb.Model(data.X, data.y, [cwb.learner(j) for j in range(3)], iterations=5, device=0)
    model.fit(5)
    lib = cwb.load_library()
    n_new = (16 << 20) // 4                       # 3 features x 4 bytes x n_new > 16 MiB
    Xn = np.zeros((3, n_new), dtype=np.float32)
    out = np.zeros(n_new, dtype=np.float32)
    st = lib.cwb_predict_noalloc(model.handle, Xn.ctypes.data_as(ctypes.c_void_p), 0, n_new,
                                 out.ctypes.data_as(ctypes.c_void_p))
    assert st == 1
    assert "limit" in cwb.cwb_last_error()
    model.free()
