"""ctypes wrapper around the FP64 CPU oracle (cwb_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the CUDA library and its
Python binding never import it.  The oracle is compiled from source with gcc
on first use (``build()``), FMA contraction off so x86 and Arm hosts give the
same bits.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwb_oracle.c")
_LIB = os.path.join(_HERE, "libcwb_oracle.so")
_lock = threading.Lock()
_lib = None

LOSS_L2, LOSS_BINOMIAL = 0, 1
OPT_CWB, OPT_ACWB, OPT_HCWB = 0, 1, 2
BL_PSPLINE, BL_LINEAR, BL_CATEGORICAL, BL_CATEGORICAL_BINARY = 0, 1, 2, 3
BINS_EXACT, BINS_SQRT, BINS_DENSE = 0, -1, -2


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC]
        try:      # OpenMP over learners where the compiler has it; the arithmetic is the same either way
            subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Learner(C.Structure):
    _fields_ = [("type", C.c_int32), ("feature", C.c_int32), ("degree", C.c_int32),
                ("n_knots", C.c_int32), ("diff_order", C.c_int32), ("df", C.c_double),
                ("lam", C.c_double), ("n_bins", C.c_int32), ("level", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("loss", C.c_int32), ("opt", C.c_int32), ("nu", C.c_double), ("gamma", C.c_double),
                ("iterations", C.c_int32), ("patience", C.c_int32), ("use_offset", C.c_int32),
                ("offset", C.c_double)]


class Result(C.Structure):
    _fields_ = [("offset", C.c_double), ("dmax", C.c_int32), ("switch_iter", C.c_int32),
                ("theta_f", C.c_void_p), ("theta_h", C.c_void_p), ("f", C.c_void_p),
                ("k_sel", C.c_void_p), ("k_cor", C.c_void_p), ("sse_best", C.c_void_p),
                ("sse_second", C.c_void_p), ("sse_best_cor", C.c_void_p),
                ("sse_second_cor", C.c_void_p), ("val_risk", C.c_void_p), ("lam", C.c_void_p),
                ("lam_full", C.c_void_p), ("nstar", C.c_void_p), ("forced_k", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_isqrt.restype = C.c_int64
            L.orc_isqrt.argtypes = [C.c_int64]
            L.orc_loss.restype = C.c_double
            L.orc_loss.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_pseudo_residual.restype = C.c_double
            L.orc_pseudo_residual.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_set_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
        return _lib


def set_threads(t: int) -> int:
    """Threads of the learner loop (1 by default); returns the count in effect (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(t)))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def learner_d(spec: dict) -> int:
    t = spec.get("type", BL_PSPLINE)
    if t == BL_CATEGORICAL:
        return spec["n_knots"]
    if t == BL_CATEGORICAL_BINARY:
        return 1
    return 2 if t == BL_LINEAR else spec.get("n_knots", 20) + spec.get("degree", 3) + 1


# --- building blocks -------------------------------------------------------

def isqrt(n: int) -> int:
    return int(lib().orc_isqrt(int(n)))


def bin_equidistant(x, nstar, xmin=None, xmax=None):
    x = _f64(x)
    xmin = float(x.min()) if xmin is None else float(xmin)
    xmax = float(x.max()) if xmax is None else float(xmax)
    ind = np.empty(x.size, dtype=np.int32)
    z = np.empty(nstar, dtype=np.float64)
    _check(lib().orc_bin_equidistant(_p(x), C.c_int64(x.size), C.c_int32(nstar), C.c_double(xmin),
                                     C.c_double(xmax), _p(ind), _p(z)), "bin_equidistant")
    return ind, z


def bin_exact(x):
    x = _f64(x)
    z = np.empty(max(x.size, 1), dtype=np.float64)
    ind = np.empty(x.size, dtype=np.int32)
    ns = C.c_int32(0)
    _check(lib().orc_bin_exact(_p(x), C.c_int64(x.size), _p(z), _p(ind), C.byref(ns)), "bin_exact")
    return ind, z[: ns.value].copy()


def bspline_basis(x, xmin, xmax, degree=3, n_knots=20):
    x = _f64(np.atleast_1d(x))
    d = n_knots + degree + 1
    out = np.empty((x.size, d), dtype=np.float64)
    _check(lib().orc_bspline_basis(_p(x), C.c_int64(x.size), C.c_double(xmin), C.c_double(xmax),
                                   C.c_int32(degree), C.c_int32(n_knots), _p(out)), "bspline_basis")
    return out


def linear_basis(x):
    x = _f64(np.atleast_1d(x))
    out = np.empty((x.size, 2), dtype=np.float64)
    lib().orc_linear_basis(_p(x), C.c_int64(x.size), _p(out))
    return out


def penalty(d, order=2):
    K = np.empty((d, d), dtype=np.float64)
    _check(lib().orc_penalty(C.c_int32(d), C.c_int32(order), _p(K)), "penalty")
    return K


def bin_matvec_u(ind, r, nstar, w=None, rows=None):
    ind = np.ascontiguousarray(ind, dtype=np.int32)
    r = _f64(r)
    w = None if w is None else _f64(w)
    rows = None if rows is None else np.ascontiguousarray(rows, dtype=np.uint8)
    u = np.empty(nstar, dtype=np.float64)
    lib().orc_bin_matvec_u(_p(ind), C.c_int64(ind.size), _p(w), _p(r), _p(rows), C.c_int32(nstar), _p(u))
    return u


def bin_matvec(ind, r, Zb, w=None, rows=None):
    ind = np.ascontiguousarray(ind, dtype=np.int32)
    Zb = _f64(Zb)
    nstar, d = Zb.shape
    r = _f64(r)
    w = None if w is None else _f64(w)
    rows = None if rows is None else np.ascontiguousarray(rows, dtype=np.uint8)
    out = np.empty(d, dtype=np.float64)
    lib().orc_bin_matvec(_p(ind), C.c_int64(ind.size), _p(w), _p(r), _p(rows), C.c_int32(nstar),
                         _p(Zb), C.c_int32(d), _p(out))
    return out


def bin_matmat(ind, Zb, w=None, rows=None):
    ind = np.ascontiguousarray(ind, dtype=np.int32)
    Zb = _f64(Zb)
    nstar, d = Zb.shape
    w = None if w is None else _f64(w)
    rows = None if rows is None else np.ascontiguousarray(rows, dtype=np.uint8)
    out = np.empty((d, d), dtype=np.float64)
    lib().orc_bin_matmat(_p(ind), C.c_int64(ind.size), _p(w), _p(rows), C.c_int32(nstar), _p(Zb),
                         C.c_int32(d), _p(out))
    return out


def df1(G, K, lam):
    G, K = _f64(G), _f64(K)
    v = C.c_double(0.0)
    _check(lib().orc_df1(_p(G), _p(K), C.c_int32(G.shape[0]), C.c_double(lam), C.byref(v)), "df1")
    return v.value


def lambda_for_df(G, K, df):
    G, K = _f64(G), _f64(K)
    v = C.c_double(0.0)
    _check(lib().orc_lambda_for_df(_p(G), _p(K), C.c_int32(G.shape[0]), C.c_double(df), C.byref(v)),
           "lambda_for_df")
    return v.value


def spd_inverse(A):
    A = _f64(A)
    out = np.empty_like(A)
    _check(lib().orc_spd_inverse(_p(A), C.c_int32(A.shape[0]), _p(out)), "spd_inverse")
    return out


def offset(loss, y, w=None, rows=None):
    y = _f64(y)
    w = None if w is None else _f64(w)
    rows = None if rows is None else np.ascontiguousarray(rows, dtype=np.uint8)
    v = C.c_double(0.0)
    _check(lib().orc_offset(C.c_int(loss), _p(y), _p(w), _p(rows), C.c_int64(y.size), C.byref(v)), "offset")
    return v.value


def loss(kind, y, f):
    return lib().orc_loss(kind, float(y), float(f))


def pseudo_residual(kind, y, f):
    return lib().orc_pseudo_residual(kind, float(y), float(f))


# --- whole fits ------------------------------------------------------------

def make_learner(spec: dict) -> Learner:
    return Learner(type=spec.get("type", BL_PSPLINE), feature=spec["feature"], degree=spec.get("degree", 3),
                   n_knots=spec.get("n_knots", 20), diff_order=spec.get("diff_order", 2),
                   df=spec.get("df", 5.0), lam=spec.get("lam", 0.0), n_bins=spec.get("n_bins", BINS_SQRT),
                   level=spec.get("level", 0))


@dataclasses.dataclass
class FitResult:
    offset: float
    theta_f: np.ndarray      # (K, dmax)
    theta_h: np.ndarray      # (K, dmax)
    f: np.ndarray            # (n,)
    k_sel: np.ndarray
    k_cor: np.ndarray
    sse_best: np.ndarray
    sse_second: np.ndarray
    sse_best_cor: np.ndarray
    sse_second_cor: np.ndarray
    val_risk: np.ndarray
    switch_iter: int
    lam: np.ndarray
    lam_full: np.ndarray
    nstar: np.ndarray
    dmax: int


def fit(X, y, learners: list[dict], *, loss=LOSS_L2, opt=OPT_CWB, nu=0.1, gamma=0.0, iterations=100,
        patience=5, w=None, val_mask=None, offset_value=None, forced_k=None) -> FitResult:
    """Run CWB / ACWB / HCWB in FP64 on X (p x n, column-major features)."""
    X = _f64(X)
    if X.ndim == 1:
        X = X[None, :]
    p, n = X.shape
    y = _f64(y)
    w = None if w is None else _f64(w)
    vm = None if val_mask is None else np.ascontiguousarray(val_mask, dtype=np.uint8)
    K = len(learners)
    arr = (Learner * K)(*[make_learner(s) for s in learners])
    dmax = max(learner_d(s) for s in learners)
    M = int(iterations)
    cfg = Config(loss=loss, opt=opt, nu=nu, gamma=gamma, iterations=M, patience=patience,
                 use_offset=0 if offset_value is None else 1,
                 offset=0.0 if offset_value is None else float(offset_value))
    out = dict(theta_f=np.zeros((K, dmax)), theta_h=np.zeros((K, dmax)), f=np.zeros(n),
               k_sel=np.zeros(M, np.int32), k_cor=np.zeros(M, np.int32), sse_best=np.zeros(M),
               sse_second=np.zeros(M), sse_best_cor=np.zeros(M), sse_second_cor=np.zeros(M),
               val_risk=np.zeros(M), lam=np.zeros(K), lam_full=np.zeros(K), nstar=np.zeros(K, np.int32))
    fk = None if forced_k is None else np.ascontiguousarray(forced_k, dtype=np.int32)
    res = Result(**{k: _p(v) for k, v in out.items()}, forced_k=_p(fk))
    st = lib().orc_fit(C.c_int64(n), C.c_int32(p), _p(X), _p(y), _p(w), _p(vm), C.c_int32(K), arr,
                       C.byref(cfg), C.byref(res))
    _check(st, "fit")
    return FitResult(offset=res.offset, switch_iter=res.switch_iter, dmax=res.dmax, **out)


def predict(Xnew, learners: list[dict], xmin, xmax, theta, offset_value):
    Xnew = _f64(Xnew)
    if Xnew.ndim == 1:
        Xnew = Xnew[None, :]
    p, m = Xnew.shape
    K = len(learners)
    arr = (Learner * K)(*[make_learner(s) for s in learners])
    theta = _f64(theta)
    out = np.empty(m)
    _check(lib().orc_predict(C.c_int64(m), C.c_int32(p), _p(Xnew), C.c_int32(K), arr, _p(_f64(xmin)),
                             _p(_f64(xmax)), _p(theta), C.c_int32(theta.shape[1]), C.c_double(offset_value),
                             _p(out)), "predict")
    return out
