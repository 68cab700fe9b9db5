"""Estimation quality of partial effects on paper-style simulated data (Sec. 4.1.1, H2/H3;
App. B.3 for n* = n^(1/4)): the MISE harness of bench.py on a reduced grid, early stopping on
noise-free data.  Seeded, so every figure is reproducible; the thresholds leave wide margins
around the measured values."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rows():
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as cwb
    import bench
    return bench.mise_cases(cwb, ns=(5_000, 20_000), snrs=(1.0, 10.0), dfs=(5.0,), gammas=(0.1,))


def _get(rows, n, snr, variant):
    (r,) = [r for r in rows if r["n"] == n and r["snr"] == snr and r["variant"] == variant]
    return r


@pytest.mark.parametrize("n", [5_000, 20_000])
@pytest.mark.parametrize("snr", [1.0, 10.0])
def test_binning_keeps_the_partial_effects(rows, n, snr):
    """H2: n* = floor(sqrt n) estimates the partial effects as well as no binning."""
    exact = _get(rows, n, snr, "exact")["mise"]
    binned = _get(rows, n, snr, "sqrt df5")["mise"]
    assert abs(binned - exact) <= 0.15 * exact, (binned, exact)


@pytest.mark.parametrize("variant", ["exact", "sqrt df5"])
@pytest.mark.parametrize("snr", [1.0, 10.0])
def test_mise_falls_with_n(rows, variant, snr):
    assert _get(rows, 20_000, snr, variant)["mise"] < 0.7 * _get(rows, 5_000, snr, variant)["mise"]


@pytest.mark.parametrize("n", [5_000, 20_000])
def test_quarter_root_bins_are_too_coarse_at_high_snr(rows, n):
    """App. B.3: n* = n^(1/4) bins cost accuracy when the signal is strong."""
    assert _get(rows, n, 10.0, "quarter df5")["mise"] >= 5 * _get(rows, n, 10.0, "sqrt df5")["mise"]


@pytest.mark.parametrize("n", [5_000, 20_000])
@pytest.mark.parametrize("snr", [1.0, 10.0])
def test_momentum_stops_earlier(rows, n, snr):
    """H3: ACWB with momentum reaches its early-stopping optimum in far fewer iterations."""
    assert 2 * _get(rows, n, snr, "sqrt ACWB gamma 0.1")["stop_iter"] <= _get(rows, n, snr, "sqrt df5")["stop_iter"]
