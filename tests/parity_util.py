"""Helpers for comparing the CUDA library with the FP64 oracle.

Tolerances: relative 1e-5 (max |a - b| / max |b|) on aggregated coefficients
per learner, on fitted values and on predictions; the selected learner
sequence must be identical wherever the oracle's best-vs-second SSE gap,
relative to the best SSE, exceeds 1e-9.  At a closer tie either choice is
correct, so the comparison re-runs the GPU with the oracle's choices forced
(the oracle decides, nothing flows from the GPU into the oracle).
"""
from __future__ import annotations

import numpy as np

REL_TOL = 1e-5
GAP_TOL = 1e-9


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max() if b.size else 0.0
    if den == 0.0:
        return float(np.abs(a).max()) if a.size else 0.0
    return float(np.abs(a - b).max() / den)


def first_divergence(k_gpu, k_ref):
    k_gpu = np.asarray(k_gpu)
    k_ref = np.asarray(k_ref)
    bad = np.flatnonzero(k_gpu != k_ref)
    return int(bad[0]) if bad.size else -1


def oracle_gap(ref, t: int, corr: bool = False) -> float:
    b = ref.sse_best_cor[t] if corr else ref.sse_best[t]
    s = ref.sse_second_cor[t] if corr else ref.sse_second[t]
    return float((s - b) / abs(b)) if b != 0 else float("inf")


def check_sequences(k_gpu, ref, corr_gpu=None):
    """Identical selections except at oracle near-ties; returns the first near-tie index or -1."""
    t = first_divergence(k_gpu, ref.k_sel)
    tc = -1 if corr_gpu is None else first_divergence(corr_gpu, ref.k_cor)
    firsts = [x for x in (t, tc) if x >= 0]
    if not firsts:
        return -1
    t0 = min(firsts)
    gap = min(oracle_gap(ref, t0), oracle_gap(ref, t0, corr=True) if corr_gpu is not None and
              np.isfinite(ref.sse_best_cor[t0]) else np.inf)
    assert gap <= GAP_TOL, (f"learner sequence diverges at iteration {t0 + 1} with oracle gap {gap:.3e} > {GAP_TOL}: "
                            f"gpu {k_gpu[t0]} vs oracle {ref.k_sel[t0]}")
    return t0


def check_coefficients(theta_gpu, theta_ref, tol=REL_TOL):
    worst = 0.0
    for k in range(theta_ref.shape[0]):
        if not np.any(theta_ref[k]) and not np.any(theta_gpu[k]):
            continue
        e = rel_err(theta_gpu[k, : theta_ref.shape[1]], theta_ref[k])
        worst = max(worst, e)
        assert e <= tol, f"learner {k}: coefficient relative error {e:.3e} > {tol}"
    return worst
