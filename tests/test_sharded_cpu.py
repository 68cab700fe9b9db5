"""Exchange logic of row-sharded fits (paper_2110_03513_gb300.sharded) on CPU, gloo ranks.

The shard backend is a small numpy stand-in with the same interface as the CUDA shard: integer
(fixed-point) bin sums under a common scale taken from the MAX of the shards' largest |r|, a
learner picked from the summed histograms, a per-bin update of the shard's rows.  Whatever the
split over processes and shards, every shard must see the same exchanged values as one shard
holding all rows, and the rows' fitted values must come out bit for bit the same.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2110_03513_gb300.sharded import ShardedFit, split_rows, torch_allreduce

S_BINS = 16


class FakeShard:
    def __init__(self, X, y, learners, *, n_global, xmin, xmax, loss, nu, iterations, device):
        self.X = np.asarray(X, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.B, self.S = self.X.shape[0], S_BINS
        self.n_global, self.xmin, self.xmax, self.nu = n_global, np.array(xmin), np.array(xmax), nu
        t = (self.X - self.xmin[:, None]) / (self.xmax - self.xmin)[:, None]
        self.ind = np.minimum(np.floor(t * (S_BINS - 1) + 0.5).astype(np.int64), S_BINS - 1)
        self.log = []

    def stats(self):
        counts = np.stack([np.bincount(self.ind[b], minlength=self.S) for b in range(self.B)]).astype(np.float64)
        return counts.ravel(), np.array([self.y.sum(), self.y.size], dtype=np.float64), int(np.log2(self.y.size))

    def finish(self, counts, sums, cnt_log2):
        self.counts = np.asarray(counts).reshape(self.B, self.S)
        self.cnt_log2 = cnt_log2
        self.f = np.full(self.y.size, sums[0] / sums[1])

    def rows(self):
        self.r = self.y - self.f
        return float(np.abs(self.r).max())

    def scatter(self, rmax):
        self.log.append(("rmax", rmax))
        q = np.rint(self.r / rmax * 2.0 ** 20).astype(np.int64)
        return np.stack([np.bincount(self.ind[b], weights=q.astype(np.float64), minlength=self.S).astype(np.int64)
                         for b in range(self.B)]).ravel()

    def solve(self, u):
        u = np.asarray(u, dtype=np.int64).reshape(self.B, self.S)
        self.log.append(("u", u.copy()))
        rmax = self.log[-2][1]
        mean = u / np.maximum(self.counts, 1.0) * (rmax / 2.0 ** 20)
        k = int(np.argmax((mean * mean * self.counts).sum(axis=1)))
        self.f = self.f + self.nu * mean[k][self.ind[k]]


def _data(n=1_001, p=3, seed=7):
    rng = np.random.default_rng(seed)
    X = rng.random((p, n))
    y = np.sin(6 * X[0]) + X[1] ** 2 + 0.1 * rng.standard_normal(n)
    # targets on a 2^-20 grid: their FP64 sums are exact in any order, so the offset does not
    # depend on how the rows are split (floating-point sums of general targets differ in the last ulps)
    return X, np.rint(y * 2.0 ** 20) / 2.0 ** 20


def _whole(X, y, M):
    fit = ShardedFit([(X, y)], learners=[], iterations=M, backend=FakeShard)
    fit.fit(M)
    return fit


def test_split_rows_covers_every_row_once():
    for n, parts in [(10, 3), (1_000_001, 7), (5, 5)]:
        r = split_rows(n, parts)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [b - a for a, b in r]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        split_rows(3, 4)


def test_in_process_shards_equal_one_shard():
    X, y = _data()
    M = 12
    whole = _whole(X, y, M)
    parts = [(X[:, a:b], y[a:b]) for a, b in split_rows(X.shape[1], 3)]
    fit = ShardedFit(parts, learners=[], iterations=M, backend=FakeShard)
    fit.fit(M)
    assert fit.n_global == X.shape[1]
    np.testing.assert_array_equal(np.concatenate([s.f for s in fit.shards]), whole.shards[0].f)
    for s in fit.shards:
        for (ka, va), (kb, vb) in zip(s.log, whole.shards[0].log):
            assert ka == kb
            np.testing.assert_array_equal(va, vb)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, M, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, y = _data()
        ranges = split_rows(X.shape[1], 2 * world)[2 * rank: 2 * rank + 2]     # two shards per rank
        fit = ShardedFit([(X[:, a:b], y[a:b]) for a, b in ranges], learners=[], iterations=M,
                         allreduce=torch_allreduce(), backend=FakeShard)
        fit.fit(M)
        out[rank] = dict(f=np.concatenate([s.f for s in fit.shards]), xmin=fit.xmin, xmax=fit.xmax,
                         n_global=fit.n_global, log=[[(k, np.asarray(v)) for k, v in s.log] for s in fit.shards])
    finally:
        dist.destroy_process_group()


def test_gloo_ranks_equal_one_shard():
    world, M = 2, 12
    X, y = _data()
    whole = _whole(X, y, M)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), M, out), nprocs=world, join=True, start_method="spawn")
    f = np.concatenate([out[r]["f"] for r in range(world)])
    np.testing.assert_array_equal(f, whole.shards[0].f)
    for r in range(world):
        np.testing.assert_array_equal(out[r]["xmin"], X.min(axis=1))
        np.testing.assert_array_equal(out[r]["xmax"], X.max(axis=1))
        assert out[r]["n_global"] == X.shape[1]
        for log in out[r]["log"]:
            for (ka, va), (kb, vb) in zip(log, whole.shards[0].log):
                assert ka == kb
                np.testing.assert_array_equal(va, vb)


def _tensor_rank_main(rank, world, port, out):
    import torch
    from paper_2110_03513_gb300.sharded import torch_allreduce_tensor
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ar = torch_allreduce_tensor()
        u = torch.arange(6, dtype=torch.int64) * (rank + 1) + (1 << 40)
        r = torch.tensor([0.5 + rank], dtype=torch.float32)
        out[rank] = (ar(u, "sum").tolist(), ar(r, "max").tolist())
    finally:
        dist.destroy_process_group()


def test_tensor_allreduce_sums_int64_exactly_and_takes_the_max():
    """The in-place tensor all-reduce of the device exchange (gloo on CPU tensors here, NCCL on CUDA
    tensors on GPUs): int64 histogram sums stay exact integers, the scale takes the maximum."""
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_tensor_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    want = [3 * i + 2 * (1 << 40) for i in range(6)]
    for rank in range(world):
        u, r = out[rank]
        assert u == want
        assert r == [1.5]
