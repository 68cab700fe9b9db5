"""Row-sharded fits: one fit's rows split over several GPUs (cwb_shard_* in include/cwb.h).

binMatVec sums over rows (Algorithm 2), so each shard scatters its own rows and only the
per-bin sums travel: per iteration one MAX of a scalar (the largest |r|, which fixes the common
fixed-point scale) and one SUM of the exact int64 histograms [B][S]; every shard then runs the
same solve and argmin on the same totals.  Setup exchanges the feature ranges (MIN / MAX), the
row count, the bin counts and the target sum (SUM) and the scatter's bin-count bound (MAX).

`ShardedFit` drives the shards one process owns (several in one process emulate several GPUs;
one per process with an `allreduce` across processes, e.g. :func:`torch_allreduce`).  The shard
operations go through a backend object (default: the CUDA library), so the exchange logic can
be exercised without a GPU.  With `device_exchange=True` the per-iteration buffers stay on the GPU
(torch CUDA tensors, all work on the current torch stream), so a NCCL all-reduce
(:func:`torch_allreduce_tensor`) moves them without host copies.  Nothing here computes any part
of the method.
"""
from __future__ import annotations

import numpy as np

from . import binding as _b

_OPS = {"sum": np.add, "max": np.maximum, "min": np.minimum}


def split_rows(n: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [start, stop) of `parts` shards covering 0..n-1 once, sizes within one."""
    if parts < 1 or n < parts:
        raise ValueError("need 1 <= parts <= n")
    edges = [n * i // parts for i in range(parts + 1)]
    return [(edges[i], edges[i + 1]) for i in range(parts)]


def torch_allreduce(group=None):
    """An `allreduce(array, op)` over the processes of a torch.distributed group (gloo on CPU tensors)."""
    import torch
    import torch.distributed as dist
    ops = {"sum": dist.ReduceOp.SUM, "max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN}

    def allreduce(a: np.ndarray, op: str) -> np.ndarray:
        t = torch.from_numpy(np.ascontiguousarray(a).copy())
        dist.all_reduce(t, op=ops[op], group=group)
        return t.numpy()
    return allreduce


def torch_allreduce_tensor(group=None):
    """An in-place `allreduce(tensor, op)` of torch tensors over a torch.distributed group (NCCL for
    CUDA tensors); returns the tensor."""
    import torch.distributed as dist
    ops = {"sum": dist.ReduceOp.SUM, "max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN}

    def allreduce(t, op: str):
        dist.all_reduce(t, op=ops[op], group=group)
        return t
    return allreduce


class GpuShard:
    """The CUDA library's row shard (one cwb_shard_* model).  With `device_exchange` the model runs on
    the current torch stream and rows / scatter / solve take and return CUDA tensors."""

    def __init__(self, X, y, learners, *, n_global, xmin, xmax, loss, nu, iterations, device,
                 device_exchange=False):
        X = np.ascontiguousarray(X)
        y = np.ascontiguousarray(y, dtype=X.dtype)
        self.p, self.n = int(X.shape[0]), int(X.shape[1])
        self.learners = list(learners)
        self.device_exchange = device_exchange
        stream = None
        if device_exchange:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
            if not stream:
                # the legacy default stream (handle 0) would leave the model on a stream of its own,
                # unordered with the exchange's tensor operations
                raise ValueError("device exchange needs a created torch stream as the current stream")
        cfg = _b.cwb_config(loss=loss, opt=_b.OPT_CWB, nu=nu, gamma=0.0, iterations=iterations, patience=0,
                            val_mask=None, stream=stream, device=device)
        self.handle = _b.cwb_shard_create(cfg, X, _b._dtype_code(X), self.n, self.p, y, self.learners, 0, n_global,
                                          xmin, xmax)
        self.B, self.S = _b.cwb_shard_sizes(self.handle)
        self.model = _b.Model._adopt(self.handle, self.n, self.p, self.learners)

    def stats(self):
        counts = np.zeros(self.B * self.S, dtype=np.float64)
        sums = np.zeros(2, dtype=np.float64)
        c = _b.cwb_shard_stats(self.handle, counts, sums)
        return counts, sums, c

    def finish(self, counts, sums, cnt_log2):
        _b.cwb_shard_finish(self.handle, np.ascontiguousarray(counts, dtype=np.float64),
                            np.ascontiguousarray(sums, dtype=np.float64), int(cnt_log2))

    def rows(self):
        if self.device_exchange:
            import torch
            r = torch.zeros(1, dtype=torch.float32, device="cuda")
            _b.cwb_shard_rows(self.handle, r, 1)
            return r
        r = np.zeros(1, dtype=np.float32)
        _b.cwb_shard_rows(self.handle, r, 0)
        return float(r[0])

    def scatter(self, rmax):
        if self.device_exchange:
            import torch
            u = torch.empty(self.B * self.S, dtype=torch.int64, device="cuda")
            _b.cwb_shard_scatter(self.handle, rmax, u, 1)
            return u
        r = np.array([rmax], dtype=np.float32)
        u = np.zeros(self.B * self.S, dtype=np.int64)
        _b.cwb_shard_scatter(self.handle, r, u, 0)
        return u

    def solve(self, u):
        if self.device_exchange:
            _b.cwb_shard_solve(self.handle, u.contiguous(), 1)
            return
        _b.cwb_shard_solve(self.handle, np.ascontiguousarray(u, dtype=np.int64), 0)

    def free(self):
        self.model.free()


class ShardedFit:
    """The shards of one fit that this process owns, stepped in lock step with the others.

    parts: list of (X_part, y_part) (p x n_i feature-major, n_i targets) of this process's shards.
    allreduce: reduction across processes, or None when this process holds every shard.
    """

    def __init__(self, parts, learners, *, loss=_b.LOSS_L2, nu=0.1, iterations=100, device=0, allreduce=None,
                 backend=GpuShard, device_exchange=False):
        self.allreduce = allreduce
        self.device_exchange = device_exchange
        X0 = np.asarray(parts[0][0])
        p = X0.shape[0] if X0.ndim > 1 else 1
        mins = np.min([np.asarray(X).reshape(p, -1).min(axis=1) for X, _ in parts], axis=0).astype(np.float64)
        maxs = np.max([np.asarray(X).reshape(p, -1).max(axis=1) for X, _ in parts], axis=0).astype(np.float64)
        n_local = np.array([sum(np.asarray(y).size for _, y in parts)], dtype=np.int64)
        self.xmin = self._reduce(mins, "min")
        self.xmax = self._reduce(maxs, "max")
        self.n_global = int(self._reduce(n_local, "sum")[0])
        kw = {"device_exchange": True} if device_exchange else {}
        self.stream = None
        if device_exchange:
            # one stream for the shards' work and the exchange's tensor operations, in issue order
            import torch
            self.stream = torch.cuda.Stream(device=device)
        with self._on_stream():
            self.shards = [backend(X, y, learners, n_global=self.n_global, xmin=self.xmin, xmax=self.xmax, loss=loss,
                                   nu=nu, iterations=iterations, device=device, **kw) for X, y in parts]
        # setup exchange: bin counts and target sums (SUM), the scatter's bin-count bound (MAX)
        st = [s.stats() for s in self.shards]
        counts = self._reduce(self._local(np.stack([c for c, _, _ in st]), "sum"), "sum")
        sums = self._reduce(self._local(np.stack([q for _, q, _ in st]), "sum"), "sum")
        clog = int(self._reduce(np.array([max(c for _, _, c in st)], dtype=np.int64), "max")[0])
        for s in self.shards:
            s.finish(counts, sums, clog)
        self.iterations_done = 0

    def _on_stream(self):
        import contextlib
        if self.stream is None:
            return contextlib.nullcontext()
        import torch
        return torch.cuda.stream(self.stream)

    def _local(self, stacked: np.ndarray, op: str) -> np.ndarray:
        return _OPS[op].reduce(stacked, axis=0)

    def _reduce(self, a: np.ndarray, op: str) -> np.ndarray:
        return a if self.allreduce is None else self.allreduce(a, op)

    def step(self):
        """One iteration: rows -> MAX of |r| -> scatter -> SUM of the histograms -> solve."""
        if self.device_exchange:
            import torch
            with torch.cuda.stream(self.stream):
                rmax = torch.stack([s.rows() for s in self.shards]).amax(dim=0)      # [1] float32 on the GPU
                rmax = self._reduce(rmax, "max")
                u = torch.stack([s.scatter(rmax) for s in self.shards]).sum(dim=0)  # exact int64 sums
                u = self._reduce(u, "sum")
                for s in self.shards:
                    s.solve(u)
            self.iterations_done += 1
            return
        rmax = np.array([max(s.rows() for s in self.shards)], dtype=np.float32)
        rmax = self._reduce(rmax, "max")
        u = self._local(np.stack([s.scatter(float(rmax[0])) for s in self.shards]), "sum")
        u = self._reduce(u.astype(np.int64), "sum")
        for s in self.shards:
            s.solve(u)
        self.iterations_done += 1

    def fit(self, iterations: int):
        for _ in range(iterations):
            self.step()

    def free(self):
        for s in self.shards:
            s.free()
