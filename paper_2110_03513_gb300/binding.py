"""ctypes binding of libcwb.so (include/cwb.h).

Arrays may be numpy arrays (host memory, device_ptrs = 0) or CUDA tensors /
objects exposing ``data_ptr()`` (device memory, device_ptrs = 1).  Nothing
here computes any part of the method.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcwb.so")

LOSS_L2, LOSS_BINOMIAL = 0, 1
OPT_CWB, OPT_ACWB, OPT_HCWB = 0, 1, 2
BL_PSPLINE, BL_LINEAR, BL_CATEGORICAL, BL_CATEGORICAL_BINARY = 0, 1, 2, 3
F32, F64 = 0, 1
BINS_EXACT, BINS_SQRT = 0, -1
PROF_ALL = 1
_PROF_BITS = {"rows": 0x10, "scatter": 0x20, "solve": 0x40}

_STATUS = {0: "CWB_OK", 1: "CWB_EINVAL", 2: "CWB_ENOMEM", 3: "CWB_ECUDA", 4: "CWB_ENUMERIC", 5: "CWB_ETIMEOUT",
           6: "CWB_ESTATE"}


class CwbError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {message}")
        self.status = status


class cwb_learner(C.Structure):
    _fields_ = [("type", C.c_int32), ("feature", C.c_int32), ("degree", C.c_int32), ("n_knots", C.c_int32),
                ("diff_order", C.c_int32), ("df", C.c_double), ("lam", C.c_double), ("n_bins", C.c_int32),
                ("level", C.c_int32)]


class cwb_config(C.Structure):
    _fields_ = [("loss", C.c_int32), ("opt", C.c_int32), ("nu", C.c_double), ("gamma", C.c_double),
                ("iterations", C.c_int32), ("patience", C.c_int32), ("val_mask", C.c_void_p),
                ("stream", C.c_void_p), ("device", C.c_int32)]


class cwb_server_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget_bytes", C.c_uint64), ("max_active", C.c_int32),
                ("slice_iterations", C.c_int32)]


class cwb_fit_request(C.Structure):
    _fields_ = [("cfg", cwb_config), ("X", C.c_void_p), ("x_dtype", C.c_int32), ("n", C.c_int64), ("p", C.c_int32),
                ("y", C.c_void_p), ("w", C.c_void_p), ("bl", C.POINTER(cwb_learner)), ("K", C.c_int32)]


class cwb_shard_config(C.Structure):
    _fields_ = [("n_global", C.c_int64), ("xmin", C.c_void_p), ("xmax", C.c_void_p)]


class cwb_learner_info(C.Structure):
    _fields_ = [("d", C.c_int32), ("nstar", C.c_int32), ("binning", C.c_int32), ("reserved", C.c_int32),
                ("xmin", C.c_double), ("xmax", C.c_double), ("lam", C.c_double), ("lam_full", C.c_double)]


_lib = None

_SIGS = {
    "cwb_create": (C.c_int, [C.POINTER(cwb_config), C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_void_p,
                             C.c_void_p, C.POINTER(cwb_learner), C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "cwb_fit": (C.c_int, [C.c_void_p, C.c_int32]),
    "cwb_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_int32]),
    "cwb_get_coefficients": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    "cwb_get_trace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "cwb_get_criteria": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_get_fitted": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_get_learner_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(cwb_learner_info)]),
    "cwb_get_learner_matrices": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "cwb_get_bin_index": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "cwb_force_selection": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_get_residuals": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "cwb_get_scatter_plan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_predict_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_void_p]),
    "cwb_synchronize": (C.c_int, [C.c_void_p]),
    "cwb_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "cwb_get_profile": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "cwb_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "cwb_batch_fit": (C.c_int, [C.c_void_p, C.c_int32]),
    "cwb_batch_synchronize": (C.c_int, [C.c_void_p]),
    "cwb_batch_free": (None, [C.c_void_p]),
    "cwb_server_create": (C.c_int, [C.POINTER(cwb_server_config), C.POINTER(C.c_void_p)]),
    "cwb_server_submit": (C.c_int, [C.c_void_p, C.POINTER(cwb_config), C.c_void_p, C.c_int32, C.c_int64, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.POINTER(cwb_learner), C.c_int32, C.c_void_p]),
    "cwb_server_poll": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    "cwb_server_take": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_void_p)]),
    "cwb_server_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_server_free": (None, [C.c_void_p]),
    "cwb_create_many": (C.c_int, [C.POINTER(cwb_fit_request), C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p),
                                  C.c_void_p]),
    "cwb_shard_create": (C.c_int, [C.POINTER(cwb_config), C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_void_p,
                                   C.POINTER(cwb_learner), C.c_int32, C.c_int32, C.POINTER(cwb_shard_config),
                                   C.POINTER(C.c_void_p)]),
    "cwb_shard_sizes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "cwb_shard_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cwb_shard_finish": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_shard_rows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_shard_scatter": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_shard_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cwb_last_error": (C.c_char_p, []),
    "cwb_free": (None, [C.c_void_p]),
}


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libcwb.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def cwb_last_error() -> str:
    return load_library().cwb_last_error().decode()


def _check(st: int, where: str):
    if st != 0:
        raise CwbError(st, where, cwb_last_error())


def _is_device(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _ptr(a):
    if a is None:
        return None
    if _is_device(a):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _dtype_code(a) -> int:
    name = str(a.dtype)
    if name.endswith("float64"):
        return F64
    if name.endswith("float32"):
        return F32
    raise TypeError(f"unsupported dtype {a.dtype}; use float32 or float64")


def learner(feature: int, *, type: int = BL_PSPLINE, degree: int = 3, n_knots: int = 20, diff_order: int = 2,
            df: float = 5.0, lam: float = 0.0, n_bins: int = BINS_SQRT, level: int = 0) -> cwb_learner:
    """One base learner; for the categorical types n_knots is the number of classes c."""
    return cwb_learner(type=type, feature=feature, degree=degree, n_knots=n_knots, diff_order=diff_order, df=df,
                       lam=lam, n_bins=n_bins, level=level)


# ---- one wrapper per C entry point -------------------------------------------------

def cwb_create(cfg: cwb_config, X, x_dtype: int, n: int, p: int, y, w, learners, device_ptrs: int) -> C.c_void_p:
    arr = (cwb_learner * len(learners))(*learners)
    out = C.c_void_p()
    st = load_library().cwb_create(C.byref(cfg), _ptr(X), x_dtype, n, p, _ptr(y), _ptr(w), arr, len(learners),
                                   device_ptrs, C.byref(out))
    _check(st, "cwb_create")
    return out


def cwb_create_many(reqs, device_ptrs: int = 0, threads: int = 0):
    """Create len(reqs) models (a list of cwb_fit_request); returns (handles, statuses)."""
    count = len(reqs)
    arr = (cwb_fit_request * count)(*reqs)
    out = (C.c_void_p * count)()
    st = np.zeros(count, dtype=np.int32)
    rc = load_library().cwb_create_many(arr, count, device_ptrs, threads, out, _ptr(st))
    handles = [C.c_void_p(h) if h else None for h in out]
    if rc != 0:
        for h in handles:
            if h:
                cwb_free(h)
        _check(rc, "cwb_create_many")
    return handles, st


def cwb_fit(model, iterations: int):
    _check(load_library().cwb_fit(model, iterations), "cwb_fit")


def cwb_predict(model, Xnew, x_dtype: int, n_new: int, out, device_ptrs: int):
    _check(load_library().cwb_predict(model, _ptr(Xnew), x_dtype, n_new, _ptr(out), device_ptrs), "cwb_predict")


def cwb_predict_noalloc(model, Xnew: np.ndarray, x_dtype: int, n_new: int, out: np.ndarray):
    _check(load_library().cwb_predict_noalloc(model, _ptr(Xnew), x_dtype, n_new, _ptr(out)), "cwb_predict_noalloc")


def cwb_get_coefficients(model, k: int, which: int, theta: np.ndarray, offset: np.ndarray | None = None):
    _check(load_library().cwb_get_coefficients(model, k, which, _ptr(theta), theta.size, _ptr(offset)),
           "cwb_get_coefficients")


def cwb_get_trace(model, k_sel: np.ndarray, k_cor: np.ndarray | None, switch_iter: np.ndarray | None,
                  done: np.ndarray | None):
    _check(load_library().cwb_get_trace(model, _ptr(k_sel), _ptr(k_cor), k_sel.size, _ptr(switch_iter),
                                        _ptr(done)), "cwb_get_trace")


def cwb_get_criteria(model, q_best: np.ndarray, q_second: np.ndarray):
    _check(load_library().cwb_get_criteria(model, _ptr(q_best), _ptr(q_second), q_best.size), "cwb_get_criteria")


def cwb_get_fitted(model, f, device_ptrs: int):
    _check(load_library().cwb_get_fitted(model, _ptr(f), device_ptrs), "cwb_get_fitted")


def cwb_get_learner_info(model, k: int) -> cwb_learner_info:
    info = cwb_learner_info()
    _check(load_library().cwb_get_learner_info(model, k, C.byref(info)), "cwb_get_learner_info")
    return info


def cwb_get_learner_matrices(model, k: int, phase: int, G: np.ndarray | None, P: np.ndarray | None):
    _check(load_library().cwb_get_learner_matrices(model, k, phase, _ptr(G), _ptr(P)), "cwb_get_learner_matrices")


def cwb_get_bin_index(model, k: int, ind: np.ndarray):
    _check(load_library().cwb_get_bin_index(model, k, _ptr(ind)), "cwb_get_bin_index")


def cwb_force_selection(model, k_forced: np.ndarray):
    _check(load_library().cwb_force_selection(model, _ptr(k_forced), k_forced.size), "cwb_force_selection")


def cwb_shard_create(cfg: cwb_config, X, x_dtype: int, n: int, p: int, y, learners, device_ptrs: int,
                     n_global: int, xmin: np.ndarray, xmax: np.ndarray) -> C.c_void_p:
    arr = (cwb_learner * len(learners))(*learners)
    xmin = np.ascontiguousarray(xmin, dtype=np.float64)
    xmax = np.ascontiguousarray(xmax, dtype=np.float64)
    sc = cwb_shard_config(n_global=n_global, xmin=_ptr(xmin).value, xmax=_ptr(xmax).value)
    out = C.c_void_p()
    st = load_library().cwb_shard_create(C.byref(cfg), _ptr(X), x_dtype, n, p, _ptr(y), arr, len(learners), device_ptrs,
                                         C.byref(sc), C.byref(out))
    _check(st, "cwb_shard_create")
    return out


def cwb_shard_sizes(model) -> tuple[int, int]:
    b, s = C.c_int32(0), C.c_int32(0)
    _check(load_library().cwb_shard_sizes(model, C.byref(b), C.byref(s)), "cwb_shard_sizes")
    return b.value, s.value


def cwb_shard_stats(model, counts: np.ndarray, sums: np.ndarray) -> int:
    c = C.c_int32(0)
    _check(load_library().cwb_shard_stats(model, _ptr(counts), _ptr(sums), C.byref(c)), "cwb_shard_stats")
    return c.value


def cwb_shard_finish(model, counts: np.ndarray, sums: np.ndarray, cnt_log2: int):
    _check(load_library().cwb_shard_finish(model, _ptr(counts), _ptr(sums), cnt_log2), "cwb_shard_finish")


def cwb_shard_rows(model, rmax, device_ptrs: int = 0):
    _check(load_library().cwb_shard_rows(model, _ptr(rmax), device_ptrs), "cwb_shard_rows")


def cwb_shard_scatter(model, rmax, u, device_ptrs: int = 0):
    _check(load_library().cwb_shard_scatter(model, _ptr(rmax), _ptr(u), device_ptrs), "cwb_shard_scatter")


def cwb_shard_solve(model, u, device_ptrs: int = 0):
    _check(load_library().cwb_shard_solve(model, _ptr(u), device_ptrs), "cwb_shard_solve")


def cwb_get_residuals(model, channel: int, out: np.ndarray):
    _check(load_library().cwb_get_residuals(model, channel, _ptr(out)), "cwb_get_residuals")


_PLAN_KEYS = ("f_lane", "binnings_per_group", "groups", "bin_ranges", "bins_per_cta", "cluster_size", "clusters",
              "stages", "threads", "smem_bytes", "int_fixed_point", "resident_ctas_cs1", "resident_ctas_cs2",
              "resident_ctas_cs4", "resident_ctas_cs8", "persistent", "persistent_stages", "persistent_ctas",
              "persistent_smem_bytes")


def cwb_get_scatter_plan(model) -> dict:
    vals = np.zeros(len(_PLAN_KEYS), dtype=np.int32)
    _check(load_library().cwb_get_scatter_plan(model, _ptr(vals), vals.size), "cwb_get_scatter_plan")
    return {k: int(v) for k, v in zip(_PLAN_KEYS, vals)}


def cwb_synchronize(model):
    _check(load_library().cwb_synchronize(model), "cwb_synchronize")


def cwb_profile(model, enable: int):
    _check(load_library().cwb_profile(model, enable), "cwb_profile")


def cwb_get_profile(model, ms: np.ndarray, launches: np.ndarray):
    _check(load_library().cwb_get_profile(model, _ptr(ms), _ptr(launches), ms.size), "cwb_get_profile")


def cwb_free(model):
    if model:
        load_library().cwb_free(model)


# ---- convenience wrapper --------------------------------------------------------

def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Model:
    """A fitted (or fitting) componentwise boosting model on one GPU.

    X is p x n feature-major (numpy on the host, or a CUDA tensor); y has n
    entries of the same dtype; learners is a list of ``learner(...)`` specs.
    """

    def __init__(self, X, y, learners, *, loss=LOSS_L2, opt=OPT_CWB, nu=0.1, gamma=0.0, iterations=100,
                 patience=5, val_mask=None, w=None, stream=None, device=-1):
        dev = _is_device(X)
        if not dev:
            X = np.ascontiguousarray(X)
            y = np.ascontiguousarray(y, dtype=X.dtype)
            w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
            val_mask = None if val_mask is None else np.ascontiguousarray(val_mask, dtype=np.uint8)
        if X.ndim == 1:
            X = X.reshape(1, -1)
        p, n = int(X.shape[0]), int(X.shape[1])
        self.p, self.n = p, n
        self.learners = list(learners)
        self._keep = (X, y, w, val_mask)
        sh = _stream_handle(stream)
        cfg = cwb_config(loss=loss, opt=opt, nu=nu, gamma=gamma, iterations=iterations, patience=patience,
                         val_mask=None if val_mask is None else _ptr(val_mask).value,
                         stream=sh, device=device)
        self.handle = cwb_create(cfg, X, _dtype_code(X), n, p, y, w, self.learners, 1 if dev else 0)
        self._keep = None

    @classmethod
    def create_many(cls, requests, threads: int = 0) -> list:
        """Models for many fits at once (cwb_create_many: their setups overlap on the GPU).  Each request
        is a dict with X, y, learners and the keyword arguments of Model (loss, opt, nu, gamma,
        iterations, patience, val_mask, w; host arrays)."""
        keep, reqs = [], []
        for r in requests:
            X = np.ascontiguousarray(r["X"])
            if X.ndim == 1:
                X = X.reshape(1, -1)
            y = np.ascontiguousarray(r["y"], dtype=X.dtype)
            w = None if r.get("w") is None else np.ascontiguousarray(r["w"], dtype=np.float64)
            vm = None if r.get("val_mask") is None else np.ascontiguousarray(r["val_mask"], dtype=np.uint8)
            lrn = list(r["learners"])
            arr = (cwb_learner * len(lrn))(*lrn)
            cfg = cwb_config(loss=r.get("loss", LOSS_L2), opt=r.get("opt", OPT_CWB), nu=r.get("nu", 0.1),
                             gamma=r.get("gamma", 0.0), iterations=r.get("iterations", 100),
                             patience=r.get("patience", 5), val_mask=None if vm is None else _ptr(vm).value,
                             stream=None, device=r.get("device", -1))
            p, n = int(X.shape[0]), int(X.shape[1])
            reqs.append(cwb_fit_request(cfg=cfg, X=_ptr(X).value, x_dtype=_dtype_code(X), n=n, p=p, y=_ptr(y).value,
                                        w=None if w is None else _ptr(w).value, bl=arr, K=len(lrn)))
            keep.append((X, y, w, vm, arr, lrn, n, p))
        handles, _ = cwb_create_many(reqs, 0, threads)
        return [cls._adopt(h, n, p, lrn) for h, (_, _, _, _, _, lrn, n, p) in zip(handles, keep)]

    @classmethod
    def _adopt(cls, handle, n: int, p: int, learners):
        """Wrap a model handle created elsewhere (a server's finished request); takes ownership."""
        m = cls.__new__(cls)
        m.handle, m.n, m.p, m.learners, m._keep = handle, n, p, list(learners), None
        return m

    def __del__(self):
        self.free()

    def autotune(self, objective: int = 0, trials: int = 5) -> float:
        """Pick the scatter's grid and cluster size by timing candidates; returns us per scatter."""
        t = C.c_double(0.0)
        _check(load_library().cwb_autotune(self.handle, objective, trials, C.byref(t)), "cwb_autotune")
        return t.value

    def free(self):
        h = getattr(self, "handle", None)
        if h:
            cwb_free(h)
            self.handle = None

    def fit(self, iterations: int = 0):
        cwb_fit(self.handle, iterations)
        return self

    def synchronize(self):
        cwb_synchronize(self.handle)

    def predict(self, Xnew, out=None):
        dev = _is_device(Xnew)
        if not dev:
            Xnew = np.ascontiguousarray(Xnew)
            if Xnew.ndim == 1:
                Xnew = Xnew.reshape(1, -1)
        n_new = int(Xnew.shape[1])
        if out is None:
            if dev:
                import torch
                out = torch.empty(n_new, dtype=torch.float32, device=Xnew.device)
            else:
                out = np.empty(n_new, dtype=np.float32)
        cwb_predict(self.handle, Xnew, _dtype_code(Xnew), n_new, out, 1 if dev else 0)
        return out

    def coefficients(self, k: int, which: int = 0) -> np.ndarray:
        info = cwb_get_learner_info(self.handle, k)
        theta = np.zeros(info.d, dtype=np.float64)
        cwb_get_coefficients(self.handle, k, which, theta)
        return theta

    def all_coefficients(self, which: int = 0, dmax: int | None = None) -> np.ndarray:
        ds = [cwb_get_learner_info(self.handle, k).d for k in range(len(self.learners))]
        D = dmax or max(ds)
        out = np.zeros((len(ds), D))
        for k, d in enumerate(ds):
            th = np.zeros(d)
            cwb_get_coefficients(self.handle, k, which, th)
            out[k, :d] = th
        return out

    @property
    def offset(self) -> float:
        theta = np.zeros(1, dtype=np.float64)
        off = np.zeros(1, dtype=np.float64)
        cwb_get_coefficients(self.handle, 0, 0, theta, off)
        return float(off[0])

    def trace(self):
        done = np.zeros(1, dtype=np.int32)
        sw = np.zeros(1, dtype=np.int32)
        probe = np.zeros(0, dtype=np.int32)
        cwb_get_trace(self.handle, probe, None, sw, done)
        M = int(done[0])
        k_sel = np.zeros(M, dtype=np.int32)
        k_cor = np.zeros(M, dtype=np.int32)
        cwb_get_trace(self.handle, k_sel, k_cor, sw, done)
        return k_sel, k_cor, int(sw[0])

    def criteria(self):
        k_sel, _, _ = self.trace()
        qb = np.zeros(k_sel.size)
        qs = np.zeros(k_sel.size)
        cwb_get_criteria(self.handle, qb, qs)
        return qb, qs

    def fitted(self, out=None):
        if out is None:
            out = np.empty(self.n, dtype=np.float32)
        cwb_get_fitted(self.handle, out, 1 if _is_device(out) else 0)
        return out

    def learner_info(self, k: int) -> cwb_learner_info:
        return cwb_get_learner_info(self.handle, k)

    def matrices(self, k: int, phase: int = 0):
        d = cwb_get_learner_info(self.handle, k).d
        G = np.zeros((d, d))
        P = np.zeros((d, d))
        cwb_get_learner_matrices(self.handle, k, phase, G, P)
        return G, P

    def bin_index(self, k: int) -> np.ndarray:
        ind = np.zeros(self.n, dtype=np.int32)
        cwb_get_bin_index(self.handle, k, ind)
        return ind

    def profile(self, enable: bool = True, classes=None):
        """Per-kernel event timing; `classes` picks kernel classes ("rows", "scatter", "solve"), None = all."""
        if not enable:
            code = 0
        elif classes is None:
            code = PROF_ALL
        else:
            code = 0
            for c in classes:
                code |= _PROF_BITS[c]
        cwb_profile(self.handle, code)

    def get_profile(self):
        ms = np.zeros(4)
        launches = np.zeros(4, dtype=np.int64)
        cwb_get_profile(self.handle, ms, launches)
        return {name: (float(ms[i]), int(launches[i])) for i, name in enumerate(("rows", "scatter", "solve"))}

    def residuals(self, channel: int = 0) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.float32)
        cwb_get_residuals(self.handle, channel, out)
        return out

    def scatter_plan(self) -> dict:
        return cwb_get_scatter_plan(self.handle)

    def force_selection(self, ks):
        cwb_force_selection(self.handle, np.ascontiguousarray(ks, dtype=np.int32))


class Batch:
    """Models advanced together: each batch step is one CUDA graph launch over all of them."""

    def __init__(self, models, iters_per_launch: int = 32):
        self.models = list(models)
        arr = (C.c_void_p * len(self.models))(*[m.handle for m in self.models])
        out = C.c_void_p()
        _check(load_library().cwb_batch_create(arr, len(self.models), iters_per_launch, C.byref(out)),
               "cwb_batch_create")
        self.handle = out

    def fit(self, iterations: int):
        _check(load_library().cwb_batch_fit(self.handle, iterations), "cwb_batch_fit")
        return self

    def synchronize(self):
        _check(load_library().cwb_batch_synchronize(self.handle), "cwb_batch_synchronize")

    def free(self):
        h = getattr(self, "handle", None)
        if h:
            load_library().cwb_batch_free(h)
            self.handle = None

    def __del__(self):
        self.free()


SERVER_STATS = ("pending", "active", "admitted", "completed", "bytes_in_use", "budget")


class Server:
    """Continuous-batching fit server on one GPU (admission by device footprint)."""

    def __init__(self, hbm_budget_bytes: int, device: int = 0, max_active: int = 64, slice_iterations: int = 32):
        cfg = cwb_server_config(device=device, hbm_budget_bytes=hbm_budget_bytes, max_active=max_active,
                                slice_iterations=slice_iterations)
        out = C.c_void_p()
        _check(load_library().cwb_server_create(C.byref(cfg), C.byref(out)), "cwb_server_create")
        self.handle = out
        self._requests = {}

    def submit(self, X, y, learners, *, loss=LOSS_L2, opt=OPT_CWB, nu=0.1, gamma=0.0, iterations=100, patience=5,
               val_mask=None, w=None) -> int:
        X = np.ascontiguousarray(X)
        if X.ndim == 1:
            X = X.reshape(1, -1)
        y = np.ascontiguousarray(y, dtype=X.dtype)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        vm = None if val_mask is None else np.ascontiguousarray(val_mask, dtype=np.uint8)
        p, n = int(X.shape[0]), int(X.shape[1])
        cfg = cwb_config(loss=loss, opt=opt, nu=nu, gamma=gamma, iterations=iterations, patience=patience,
                         val_mask=None if vm is None else _ptr(vm).value, stream=None, device=0)
        arr = (cwb_learner * len(learners))(*learners)
        rid = C.c_int64(0)
        _check(load_library().cwb_server_submit(self.handle, C.byref(cfg), _ptr(X), _dtype_code(X), n, p, _ptr(y),
                                                _ptr(w), arr, len(learners), C.byref(rid)), "cwb_server_submit")
        self._requests[rid.value] = (X, y, w, n, p, list(learners))     # buffers stay alive until done
        return rid.value

    def poll(self, wait: bool = False, cap: int = 1024) -> list:
        ids = np.zeros(cap, dtype=np.int64)
        got = C.c_int32(0)
        _check(load_library().cwb_server_poll(self.handle, 1 if wait else 0, _ptr(ids), cap, C.byref(got)),
               "cwb_server_poll")
        return [int(i) for i in ids[: got.value]]

    def take(self, rid: int) -> "Model":
        out = C.c_void_p()
        st = load_library().cwb_server_take(self.handle, rid, C.byref(out))
        X, y, w, n, p, learners = self._requests.pop(rid, (None, None, None, 0, 0, []))
        _check(st, "cwb_server_take")
        return Model._adopt(out, n, p, learners)

    def stats(self) -> dict:
        v = np.zeros(len(SERVER_STATS), dtype=np.int64)
        _check(load_library().cwb_server_stats(self.handle, _ptr(v), v.size), "cwb_server_stats")
        return {k: int(x) for k, x in zip(SERVER_STATS, v)}

    def free(self):
        h = getattr(self, "handle", None)
        if h:
            load_library().cwb_server_free(h)
            self.handle = None

    def __del__(self):
        self.free()
