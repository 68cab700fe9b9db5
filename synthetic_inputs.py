"""Seeded synthetic inputs for componentwise boosting workloads.

This module only draws data (features, targets, validation masks, request
streams).  It holds none of the boosting arithmetic: no binning, no basis, no
fitting.  Both the FP64 CPU oracle and the CUDA library consume what it
produces, which is the only thing they share.

Every generator takes an explicit integer seed and uses numpy's PCG64, so a
workload is reproducible from (name, seed).  The shapes follow the paper's
simulation setting (Sec. 4.1.1: additive non-linear effects of numerical
features plus Gaussian noise at a given signal-to-noise ratio) scaled to the
sizes of the named workloads below.  The paper's own simulation draws and its
OpenML benchmark data are not available; these inputs stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Dataset",
    "additive_regression",
    "mixed_categorical",
    "sim_small_exact",
    "sim_binned_l2",
    "sim_binomial_hybrid",
    "batched_fit_specs",
    "served_request_stream",
    "request_dataset",
    "request_dataset_f32",
    "paper_style_simulation",
    "paper_style_effect",
    "paper_style_sample",
]


@dataclasses.dataclass
class Dataset:
    """Column-major features X[p][n], target y[n], optional validation mask."""

    X: np.ndarray            # shape (p, n); float32 or float64; feature-major
    y: np.ndarray            # shape (n,), same dtype as X
    val_mask: np.ndarray | None = None   # shape (n,), uint8 (1 = validation row)
    eta: np.ndarray | None = None        # noise-free additive signal (float64)
    truth: list | None = None            # generator parameters of the true effects (paper-style data)
    description: str = ""

    @property
    def n(self) -> int:
        return int(self.X.shape[1])

    @property
    def p(self) -> int:
        return int(self.X.shape[0])


def _effect(kind: int, x: np.ndarray) -> np.ndarray:
    """Effect family for informative feature number ``kind`` (1-based)."""
    if kind <= 5:
        return np.sin(2.0 * math.pi * kind * x / 3.0)
    if kind % 2 == 0:
        return 4.0 * (x - 0.5) ** 2
    return 8.0 * (x - 0.5) ** 3


def additive_regression(n: int, p: int, n_informative: int, seed: int, *,
                        dtype=np.float32, snr: float = 1.0,
                        normal_features: int = 0) -> Dataset:
    """Additive regression data: y = sum_j e_j(x_j) + N(0, (sd(eta)/snr)^2).

    The first ``p - normal_features`` features are U[0, 1]; the remaining
    ``normal_features`` are N(0, 1).  Informative features are the first
    ``n_informative`` columns; effect families cycle through five sine waves
    sin(2 pi j x / 3) and alternating quadratic / cubic polynomials.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.empty((p, n), dtype=np.float64)
    n_unif = p - normal_features
    X[:n_unif] = rng.random((n_unif, n))
    if normal_features:
        X[n_unif:] = rng.standard_normal((normal_features, n))
    eta = np.zeros(n, dtype=np.float64)
    for j in range(min(n_informative, p)):
        kind = (j % 10) + 1
        eta += _effect(kind, X[j])
    sd = float(np.std(eta)) if n > 1 else 1.0
    noise = rng.standard_normal(n) * (sd / snr if snr > 0 else 0.0)
    y = eta + noise
    return Dataset(X=X.astype(dtype), y=y.astype(dtype), eta=eta,
                   description=f"additive regression n={n} p={p} inf={n_informative} seed={seed}")


def mixed_categorical(n: int, p_num: int, classes: list[int], seed: int, *, n_informative_num: int = 2,
                      n_informative_cat: int = 1, dtype=np.float32, snr: float = 1.0,
                      binomial: bool = False) -> Dataset:
    """Numerical plus categorical features (the setting of the paper's categorical simulation,
    App. B.2, with the numerical effects of Sec. 4.1.1 added).

    Rows 0..p_num-1 of X are U[0, 1] features, the first ``n_informative_num`` with the effects of
    :func:`additive_regression`.  Then one row per entry of ``classes``: integer class codes
    0..c-1 stored as floats, class frequencies drawn from a Dirichlet(0.7) (so some classes are
    rare), every class present at least once.  The first ``n_informative_cat`` categorical features
    carry class effects drawn from N(0, 1); the others are noise.  ``binomial`` turns the linear
    predictor into y ~ Bernoulli(sigmoid(eta)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = p_num + len(classes)
    X = np.empty((p, n), dtype=np.float64)
    X[:p_num] = rng.random((p_num, n))
    eta = np.zeros(n, dtype=np.float64)
    for j in range(min(n_informative_num, p_num)):
        eta += _effect((j % 10) + 1, X[j])
    for t, c in enumerate(classes):
        probs = rng.dirichlet(np.full(c, 0.7))
        codes = rng.choice(c, size=n, p=probs)
        codes[rng.choice(n, size=c, replace=False)] = np.arange(c)
        X[p_num + t] = codes
        if t < n_informative_cat:
            eta += rng.standard_normal(c)[codes]
    if binomial:
        y = (rng.random(n) < 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
    else:
        sd = float(np.std(eta)) if n > 1 else 1.0
        y = eta + rng.standard_normal(n) * (sd / snr if snr > 0 else 0.0)
    return Dataset(X=X.astype(dtype), y=y.astype(dtype), eta=eta,
                   description=f"numerical + categorical n={n} p_num={p_num} classes={classes} seed={seed}")


def sim_small_exact(seed: int = 0, n: int = 10_000, p: int = 10) -> Dataset:
    """n=10,000, p=10, x ~ U[0,1] in FP64, y = sum_{j<=5} sin(2 pi j x_j / 3) + noise, SNR 1."""
    return additive_regression(n, p, 5, seed, dtype=np.float64)


def sim_binned_l2(seed: int = 1, n: int = 1_000_000, p: int = 50) -> Dataset:
    """n=1,000,000, p=50 U[0,1] FP32 features, 10 informative, SNR 1 (L2 loss)."""
    return additive_regression(n, p, 10, seed, dtype=np.float32)


def sim_binomial_hybrid(seed: int = 2, n: int = 2_000_000, p: int = 200,
                        n_informative: int = 20, val_fraction: float = 0.2) -> Dataset:
    """Binary classification: half U[0,1], half N(0,1) features, y ~ Bernoulli(sigmoid(eta)).

    The additive signal eta (20 informative features, same effect families)
    is centred and scaled to unit standard deviation.  A seeded 20% validation
    mask is drawn for the hybrid optimizer.  Informative features alternate
    between the uniform and the normal block so both kinds carry signal.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_norm = p // 2
    n_unif = p - n_norm
    X = np.empty((p, n), dtype=np.float64)
    X[:n_unif] = rng.random((n_unif, n))
    X[n_unif:] = rng.standard_normal((n_norm, n))
    eta = np.zeros(n, dtype=np.float64)
    for j in range(n_informative):
        col = (j // 2) if j % 2 == 0 else n_unif + (j // 2)
        x = X[col]
        if col >= n_unif:           # map N(0,1) into the unit interval for the effect shape
            x = 1.0 / (1.0 + np.exp(-x))
        eta += _effect((j % 10) + 1, x)
    eta -= eta.mean()
    eta /= max(float(eta.std()), 1e-12)
    prob = 1.0 / (1.0 + np.exp(-eta))
    y = (rng.random(n) < prob).astype(np.float64)
    val = (rng.random(n) < val_fraction).astype(np.uint8)
    return Dataset(X=X.astype(np.float32), y=y.astype(np.float32), val_mask=val, eta=eta,
                   description=f"binomial hybrid n={n} p={p} seed={seed}")


def batched_fit_specs(count: int = 512, seed: int = 3, n_lo: int = 5_000, n_hi: int = 500_000,
                      p_lo: int = 5, p_hi: int = 100) -> list[dict]:
    """Specs for many independent fits shaped like CV folds x a df/nu grid.

    n is log-uniform in [n_lo, n_hi], p uniform in [p_lo, p_hi]; each spec
    carries its own data seed, df in {4, 5, 6, 8} and nu in {0.05, 0.1, 0.2, 0.3}
    cycling like a grid over folds.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dfs = (4.0, 5.0, 6.0, 8.0)
    nus = (0.05, 0.1, 0.2, 0.3)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p = int(rng.integers(p_lo, p_hi + 1))
        out.append(dict(index=i, n=n, p=p, seed=int(rng.integers(0, 2**31 - 1)),
                        df=dfs[(i // 4) % 4], nu=nus[i % 4], fold=i % 5))
    return out


def served_request_stream(count: int = 10_000, seed: int = 4, rate_per_s: float = 10.0,
                          n_lo: int = 10_000, n_hi: int = 5_000_000, p_lo: int = 10,
                          p_hi: int = 500, m_lo: int = 500, m_hi: int = 5_000) -> list[dict]:
    """Poisson stream of fit requests: variant, loss, n, p, M, per-request seed, arrival time."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        out.append(dict(index=i, arrival_s=t, variant=int(rng.integers(0, 3)),
                        loss=int(rng.integers(0, 2)), n=n, p=p,
                        iterations=int(rng.integers(m_lo, m_hi + 1)),
                        seed=int(rng.integers(0, 2**31 - 1))))
    return out


def request_dataset(spec: dict, dtype=np.float32) -> Dataset:
    """Data of one fit request (served or batched workloads): ``spec`` carries n, p and seed, and
    optionally loss (0 L2, 1 binomial) and variant (2 = hybrid, which draws a 20% validation mask).

    Features are U[0, 1]; min(p, 10) of them carry the additive effects of ``additive_regression``.
    For the binomial loss the signal is centred, scaled to unit standard deviation and y is drawn as
    Bernoulli(sigmoid(signal)).
    """
    n, p, seed = int(spec["n"]), int(spec["p"]), int(spec["seed"])
    d = additive_regression(n, p, min(p, 10), seed, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    y = d.y
    if int(spec.get("loss", 0)) == 1:
        eta = d.eta - d.eta.mean()
        eta /= max(float(eta.std()), 1e-12)
        y = (rng.random(n) < 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
    val = (rng.random(n) < 0.2).astype(np.uint8) if int(spec.get("variant", 0)) == 2 else None
    return Dataset(X=d.X.astype(dtype), y=y.astype(dtype), val_mask=val, eta=d.eta,
                   description=f"request n={n} p={p} seed={seed}")


def request_dataset_f32(spec: dict) -> Dataset:
    """Data of one full-size fit request (n up to 5M, p up to 500), drawn straight in FP32 so that the
    largest requests (billions of feature values) are generated without FP64 copies.

    Features are U[0, 1) FP32 from PCG64(seed); the first min(p, 10) carry the additive effects of
    ``additive_regression`` evaluated in FP64 on the FP32 values; Gaussian noise at SNR 1 (PCG64(seed ^
    0x5EED)).  Binomial requests (loss 1) centre and scale the signal to unit standard deviation and draw
    y ~ Bernoulli(sigmoid(signal)); hybrid requests (variant 2) draw a 20% validation mask.
    """
    n, p, seed = int(spec["n"]), int(spec["p"]), int(spec["seed"])
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.random((p, n), dtype=np.float32)
    eta = np.zeros(n, dtype=np.float64)
    for j in range(min(p, 10)):
        eta += _effect((j % 10) + 1, X[j].astype(np.float64))
    rng2 = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    if int(spec.get("loss", 0)) == 1:
        z = eta - eta.mean()
        z /= max(float(z.std()), 1e-12)
        y = (rng2.random(n) < 1.0 / (1.0 + np.exp(-z))).astype(np.float32)
    else:
        sd = float(np.std(eta)) if n > 1 else 1.0
        y = (eta + rng2.standard_normal(n) * sd).astype(np.float32)
    val = (rng2.random(n) < 0.2).astype(np.uint8) if int(spec.get("variant", 0)) == 2 else None
    return Dataset(X=X, y=y, val_mask=val, eta=eta, description=f"full-size request n={n} p={p} seed={seed}")


def paper_style_effect(truth_j: tuple, x: np.ndarray) -> np.ndarray:
    """True effect of one informative feature of :func:`paper_style_simulation` at x.

    ``truth_j = (lo, hi, tau)``: a cubic spline on [lo, hi] with 10 equidistant inner knots in the
    truncated-power basis (1, u, u^2, u^3, ((x - kappa_i)_+ / (hi - lo))^3), u = (x - lo) / (hi - lo).
    """
    lo, hi, tau = truth_j
    width = max(hi - lo, 1e-12)
    knots = np.linspace(lo, hi, 12)[1:-1]
    u = (x - lo) / width
    cols = [np.ones_like(x), u, u ** 2, u ** 3] + [np.clip((x - k) / width, 0, None) ** 3 for k in knots]
    return np.stack(cols, 1) @ tau


def paper_style_simulation(n: int, p: int, p_noise: int, snr: float, seed: int) -> Dataset:
    """Variant following Sec. 4.1.1 literally: feature ranges drawn from U[0,100],
    effects are random splines (cubic, 10 inner knots, coefficients N(0, 9)),
    noise features N(0,1), Gaussian target noise with sd(eta)/snr.

    The spline effects are drawn with a truncated-power cubic basis on the
    feature's own range, which spans the same function space as the paper's
    order-4 B-spline basis with 10 inner knots (14 coefficients).  ``truth``
    holds (lo, hi, tau) per informative feature (see :func:`paper_style_effect`).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    truth = []
    for j in range(p):             # the truth first: the same seed gives the same effects at every n
        lo = rng.uniform(0, 100)
        hi = lo + rng.uniform(0, 100)
        truth.append((lo, hi, rng.normal(0.0, 3.0, 14)))
    X = np.empty((p + p_noise, n), dtype=np.float64)
    eta = np.zeros(n)
    for j, (lo, hi, tau) in enumerate(truth):
        X[j] = rng.uniform(lo, hi, n)
        eta += paper_style_effect(truth[j], X[j])
    if p_noise:
        X[p:] = rng.standard_normal((p_noise, n))
    y = eta + rng.standard_normal(n) * (float(np.std(eta)) / snr)
    return Dataset(X=X, y=y, eta=eta, truth=truth,
                   description=f"paper-style sim n={n} p={p} noise={p_noise} snr={snr}")


def paper_style_sample(truth: list, p_noise: int, n: int, seed: int) -> Dataset:
    """Fresh noise-free rows from the truth of :func:`paper_style_simulation` (y = eta): the large
    validation set of the paper's early stopping (Sec. 4.1.1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = len(truth)
    X = np.empty((p + p_noise, n), dtype=np.float64)
    eta = np.zeros(n)
    for j, (lo, hi, tau) in enumerate(truth):
        X[j] = rng.uniform(lo, hi, n)
        eta += paper_style_effect(truth[j], X[j])
    if p_noise:
        X[p:] = rng.standard_normal((p_noise, n))
    return Dataset(X=X, y=eta.copy(), eta=eta, truth=truth, description=f"paper-style noise-free sample n={n}")
