#!/usr/bin/env python3
"""Benchmark of the binned CWB iteration on GB300.

Workload (the headline configuration): binned componentwise boosting, L2
loss, n = 1,000,000 rows, p = 50 U[0,1] FP32 features (10 informative,
SNR 1), n* = floor(sqrt(n)) = 1000 equidistant bins per feature (uint16
index vectors), one cubic P-spline learner per feature (d = 24, df = 5),
nu = 0.1.  Seeded synthetic data stands in for the paper's simulation data.

A step is one boosting iteration through the public C ABI (cwb_fit(model, 1)):
pseudo residuals, binMatVec scatter of every feature, Z^T u, the solve with
the cached inverse, the SSE criterion, the argmin and the model update.  The
L2 cache is flushed before every timed step (a 256 MiB buffer is written and
then read back, so the timed step starts with no dirty lines of the flush to
write back) and each step is timed with CUDA events on the model's stream; the
flush is not timed.  The iteration's kernels overlap through programmatic
dependent launch, so the scatter's own duration is taken in a second pass of
the same K steps in which event-record nodes of the iteration graph bracket
it (serialising it against its neighbours); its average gives the roofline
figure.  A third pass brackets every kernel for the per-kernel breakdown.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "binned CWB iters/s & HBM GB/s at n=1M,p=50; served fits/s, p50/p99 latency"
UNIT = "iters/s"
N_ROWS, N_FEAT, NSTAR, M_FIT = 1_000_000, 50, 1000, 2000
NU = 0.1
# Algorithmic bytes (FP32 vectors, uint16 indices): the index stream of every feature
# plus y (read), f (read + write) and the update gather of the selected feature.
ALG_BYTES_ITER = N_FEAT * N_ROWS * 2 + N_ROWS * (4 + 8 + 2)
# Per launch of the scatter kernel: the index stream plus the residual vector.
ALG_BYTES_SCATTER = N_FEAT * N_ROWS * 2 + N_ROWS * 4
FLUSH_BYTES = 256 << 20
WORKLOAD = ("binned CWB, L2 loss, n=1,000,000, p=50 U[0,1] FP32 features (10 informative, SNR 1), "
            "n*=1000 equidistant bins per feature (uint16 index), cubic P-splines d=24 df=5, nu=0.1")

# DRAM traffic of one scatter launch from the committed ncu capture, valid for the
# scatter kernel source with this SHA-256 prefix (null once the kernel changes).
SCATTER_TRAFFIC = {"sha256": "ae8e411dae40ef75", "bytes": 104056064 + 3881216}   # one ncu capture of this kernel
# the same kernel on the HCWB workload (ACWB phase: 200 binnings x 1.6M training rows, two channels)
HCWB_SCATTER_TRAFFIC = {"sha256": "ae8e411dae40ef75", "bytes": 663198464 + 3175936}


def scatter_source_hash() -> str:
    """Hash of the scatter kernel's source and of the device helpers it uses (a recorded ncu traffic
    figure is reported only while both are unchanged)."""
    csrc = os.path.join(ROOT, "paper_2110_03513_gb300", "csrc")
    text = open(os.path.join(csrc, "cwb_iter.cu")).read()
    start = text.find("// binMatVec scatter")
    end = text.find("// Per-learner fit, criterion and argmin")
    helpers = open(os.path.join(csrc, "cwb_device.cuh")).read()
    # comments and blank lines do not change the kernel
    code = [ln.split("//", 1)[0].rstrip() for ln in (text[start:end] + helpers).splitlines()]
    return hashlib.sha256("\n".join(ln for ln in code if ln).encode()).hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--skip-cpu-baseline", action="store_true", help="do not time the CPU oracle")
    ap.add_argument("--skip-e2e", action="store_true", help="do not run the end-to-end fit")
    ap.add_argument("--skip-batched", action="store_true", help="do not run the batched-fits measurement")
    ap.add_argument("--skip-served", action="store_true", help="do not run the served-requests measurement")
    ap.add_argument("--skip-hcwb", action="store_true", help="do not add the HCWB workload's figures")
    ap.add_argument("--skip-small", action="store_true", help="do not add the small exact-binning fit's figures")
    ap.add_argument("--batched-fits", type=int, default=512,
                    help="fits in the batched measurement (the first of the 512 seeded specs)")
    ap.add_argument("--served-requests", type=int, default=96, help="requests in the served measurement")
    ap.add_argument("--served-full-requests", type=int, default=16,
                    help="requests of the full-size served measurement (--workload served_full)")
    ap.add_argument("--workload", choices=["binned_l2", "hcwb_binomial", "mise", "served_full"], default="binned_l2",
                    help="binned_l2: the headline line (n=1M, p=50); hcwb_binomial: ACWB with the hybrid "
                         "switch, binomial loss, n=2M, p=200, n*=1414 (a separate line); mise: estimation "
                         "quality of partial effects on paper-style simulated data (a separate line)")
    return ap.parse_args()


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- CPU oracle

def time_oracle(X, y, specs, iters: int):
    """Seconds per oracle iteration (setup timed separately and subtracted)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.fit(X, y, specs, nu=NU, iterations=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.fit(X, y, specs, nu=NU, iterations=iters)
    t_all = time.perf_counter() - t0
    return max(t_all - t_setup, 1e-9) / iters, t_setup


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline_full(data, iters: int = 6):
    """The FP64 oracle as it stands on one thread, and with its learner loop on every host core
    (OpenMP; the per-learner sums keep their order, so the results are bit-identical)."""
    import numpy as np
    from oracle import oracle as O
    specs = [dict(feature=j, n_bins=-1, df=5.0) for j in range(N_FEAT)]
    X = data.X.astype(np.float64)
    y = data.y.astype(np.float64)
    O.set_threads(1)
    per_iter, t_setup = time_oracle(X, y, specs, iters)
    nproc = os.cpu_count() or 1
    threads = O.set_threads(nproc)
    try:
        per_iter_mt, _ = time_oracle(X, y, specs, iters)
    finally:
        O.set_threads(1)
    return {"value": 1.0 / per_iter, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 C oracle, single thread, {iters} iterations of the full n=1,000,000 p=50 workload "
                      f"(setup {t_setup:.1f} s timed separately and excluded)",
            "cpu": cpu_model(), "nproc": nproc,
            "openmp": {"value": 1.0 / per_iter_mt, "unit": UNIT, "cores": threads,
                       "sample": f"the same {iters} iterations with the oracle's learner loop on {threads} threads"}}


def run_reference(args):
    """The FP64 CPU oracle timed as the reference arm (rank 0 only)."""
    import numpy as np
    import synthetic_inputs as S
    from oracle import oracle as O
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    O.build()
    data = S.sim_binned_l2(seed=args.seed)
    # bounded sample: the first n' rows, one iteration per step; the iteration is linear in n
    budget_s = 150.0
    per_row = 1.6e-6              # rough oracle seconds per row and iteration at p = 50
    steps = max(args.steps, 1) + max(args.warmup, 0)
    n_s = int(min(N_ROWS, max(20_000, budget_s / steps / per_row)))
    X = data.X[:, :n_s].astype(np.float64)
    y = data.y[:n_s].astype(np.float64)
    specs = [dict(feature=j, n_bins=NSTAR, df=5.0) for j in range(N_FEAT)]
    t0 = time.perf_counter()
    O.fit(X, y, specs, nu=NU, iterations=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.fit(X, y, specs, nu=NU, iterations=steps)
    per_step = max(time.perf_counter() - t0 - t_setup, 1e-9) / steps
    value = 1.0 / (per_step * N_ROWS / n_s)
    sample = (f"FP64 C oracle, single thread: {steps} iterations on the first {n_s} rows of the n=1,000,000 p=50 "
              f"workload (n*=1000 bins), time per iteration scaled by n/n' = {N_ROWS / n_s:.2f}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * N_ROWS / n_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_ROWS, "p": N_FEAT, "nstar": NSTAR,
                                            "index": "uint16", "learners": N_FEAT},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm

def replica_throughput(local_ms: float, steps: int, world: int, dist=None, device=None):
    """Whole-job iterations/s of `world` independent replicas that each timed `steps` steps.

    The job's time is the slowest rank's (max over ranks, one all-reduce of a scalar; the data
    path has no collective).  Returns (iterations/s over all ranks, ms per step of the slowest rank).
    """
    import torch
    total_ms = float(local_ms)
    if dist is not None and world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms / steps


def run_ours(args):
    import numpy as np
    import torch
    import synthetic_inputs as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as cwb

    data = S.sim_binned_l2(seed=args.seed + rank)
    stream = torch.cuda.Stream(device=dev)
    learners = [cwb.learner(j, n_bins=NSTAR, df=5.0) for j in range(N_FEAT)]
    with torch.cuda.stream(stream):
        Xd = torch.from_numpy(data.X).to(dev)
        yd = torch.from_numpy(data.y).to(dev)
        stream.synchronize()
        t_setup = time.perf_counter()
        model = cwb.Model(Xd, yd, learners, nu=NU, iterations=M_FIT, stream=stream, device=local)
        stream.synchronize()
        t_setup = time.perf_counter() - t_setup
        del Xd, yd
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        sink = torch.empty(1, dtype=torch.float32, device=dev)

        def flush_l2():
            flush.zero_()
            torch.sum(flush, dim=0, keepdim=True, out=sink)

        for _ in range(max(args.warmup, 3)):
            flush_l2()
            model.fit(1)
        stream.synchronize()
        K = args.steps
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        props = torch.cuda.get_device_properties(dev)
        gpu_id = str(getattr(props, "uuid", local))
        if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
            gpu_id = "GPU-" + gpu_id
        sampler = ClockSampler(gpu_id if rank == 0 else str(local))
        if rank == 0:
            sampler.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for i in range(K):
            flush_l2()
            starts[i].record(stream)
            model.fit(1)
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = sampler.stop() if rank == 0 else None
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        # roofline pass: the same K steps with the scatter bracketed by event-record nodes of the
        # iteration graph (this serialises it against its neighbours, so it is not the value pass)
        model.profile(True, classes=["scatter"])
        for i in range(K):
            flush_l2()
            model.fit(1)
        prof = model.get_profile()
        # breakdown pass: every kernel bracketed by events
        model.profile(True)
        for i in range(min(K, 200)):
            flush_l2()
            model.fit(1)
        breakdown = model.get_profile()
        model.profile(False)
        plan = model.scatter_plan()
    value, ms_per_step = replica_throughput(sum(step_ms), K, world, dist, dev)
    launches = K * 3              # rows, scatter and solve per CWB iteration

    # roofline of the dominant kernel (the scatter), from its own events on the model's stream
    sc_ms, sc_n = prof["scatter"]
    sc_avg = sc_ms / max(sc_n, 1) / 1e3
    peak, peak_kind = measured_peaks()
    achieved = ALG_BYTES_SCATTER / sc_avg / 1e9
    traffic = SCATTER_TRAFFIC["bytes"] if SCATTER_TRAFFIC["sha256"] == scatter_source_hash() else None

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_ROWS, "p": N_FEAT, "nstar": NSTAR, "index": "uint16",
                       "learners": N_FEAT,
                       "l2": "flushed before every timed step (256 MiB written, then read; untimed)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "hbm_gbs": ALG_BYTES_ITER / (ms_per_step / 1e3) / 1e9,
            "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in breakdown.items()},
            "kernel_ms_note": "separate pass with every kernel bracketed by graph event nodes (no kernel overlap)",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_scatter",
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "timing": f"CUDA events around the scatter node, {K} steps, second pass"},
            "gpu_launches": launches, "clocks": clocks, "scatter_plan": plan,
            "setup_ms": t_setup * 1e3}

    if not args.skip_e2e:
        line["e2e"] = run_e2e(cwb, data, stream, dev, local)
    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_full(data)
    if rank == 0 and world == 1:
        del data
        if not args.skip_batched:
            line["batched"] = run_batched(cwb, args)
        if not args.skip_served:
            line["served"] = run_served(cwb, args)
    model.free()
    if rank == 0 and world == 1 and not args.skip_hcwb:
        h = measure_hcwb(cwb, min(args.steps, 40), 3, args.seed)
        line["hcwb"] = {k: h[k] for k in ("metric", "value", "unit", "ms_per_step", "hbm_gbs", "roofline",
                                          "scatter_us", "config", "clocks")}
    if rank == 0 and world == 1 and not args.skip_small:
        line["small_exact"] = measure_small(cwb)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_small(cwb, M: int = 500):
    """The small configuration: n = 10,000, p = 10 U[0,1] FP64 features, exact binning (n* = number of
    unique values, about 10,000, uint16), cubic P-splines df = 5, nu = 0.1, M = 500 (L2).  One whole
    fit of M iterations per step (its iteration graphs replayed), three steps after one warm-up fit;
    at this size an iteration is bound by kernel latency, not by memory."""
    import numpy as np
    import synthetic_inputs as S
    d = S.sim_small_exact()
    learners = [cwb.learner(j, n_bins=cwb.BINS_EXACT, df=5.0) for j in range(d.p)]
    times = []
    for rep in range(4):
        model = cwb.Model(d.X, d.y, learners, nu=NU, iterations=M, device=0)
        model.synchronize()
        t0 = time.perf_counter()
        model.fit(M)
        model.synchronize()
        if rep:
            times.append(time.perf_counter() - t0)
        model.free()
    t = float(np.median(times))
    return {"workload": "binned CWB, L2, n=10,000, p=10 U[0,1] FP64, exact binning (n* = unique values), "
                        "P-splines d=24 df=5, nu=0.1, M=500", "value": M / t, "unit": "iters/s",
            "ms_per_fit": t * 1e3, "timing": "host clock around cwb_fit(M) and a synchronize, median of 3 fits"}


def _percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if xs else None


def run_batched(cwb, args):
    """Uneven fits shaped like CV folds x a df/nu grid: n log-uniform 5k-500k, p uniform 5-100,
    n* = floor(sqrt(n)), L2, M = 1000.  Arm 1 (sequential): each fit alone, one after another,
    through cwb_fit (its own graphs).  Arm 2 (batched): every model autotuned for SM-time, then all
    advanced together by cwb_batch_fit (one graph launch per 32 iterations of all fits).  Setup
    (data, create, autotune) is not timed; both arms start from identical models."""
    import numpy as np
    import torch
    import synthetic_inputs as S
    M = 1000
    specs = S.batched_fit_specs(count=512)[: max(1, args.batched_fits)]
    datasets = [S.request_dataset(sp) for sp in specs]
    learner_sets = [[cwb.learner(j, n_bins=-1, df=sp["df"]) for j in range(sp["p"])] for sp in specs]
    # setup of every fit: one create after another, and all at once (cwb_create_many)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_models = [cwb.Model(d.X, d.y, lrn, nu=sp["nu"], iterations=M, device=0)
                  for sp, d, lrn in zip(specs, datasets, learner_sets)]
    torch.cuda.synchronize()
    t_create_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    bat_models = cwb.Model.create_many([dict(X=d.X, y=d.y, learners=lrn, nu=sp["nu"], iterations=M, device=0)
                                        for sp, d, lrn in zip(specs, datasets, learner_sets)])
    torch.cuda.synchronize()
    t_create_many = time.perf_counter() - t0
    del datasets
    # sequential arm
    t_seq, coef_seq = 0.0, []
    for m in seq_models:
        m.synchronize()
        t0 = time.perf_counter()
        m.fit(M)
        m.synchronize()
        t_seq += time.perf_counter() - t0
        coef_seq.append(m.all_coefficients(0, dmax=24))
        m.free()
    # batched arm
    t0 = time.perf_counter()
    for m in bat_models:
        m.autotune(objective=1, trials=2)
    t_tune = time.perf_counter() - t0
    batch = cwb.Batch(bat_models, iters_per_launch=32)
    batch.synchronize()
    t0 = time.perf_counter()
    batch.fit(M)
    batch.synchronize()
    t_bat = time.perf_counter() - t0
    worst = 0.0
    for m, ref in zip(bat_models, coef_seq):
        th = m.all_coefficients(0, dmax=24)
        den = float(np.abs(ref).max()) or 1.0
        worst = max(worst, float(np.abs(th - ref).max()) / den)
    batch.free()
    for m in bat_models:
        m.free()
    nf = len(specs)
    return {"fits": nf, "iterations": M, "fits_per_s": nf / t_bat, "sequential_fits_per_s": nf / t_seq,
            "speedup_vs_sequential": t_seq / t_bat, "batched_s": t_bat, "sequential_s": t_seq,
            "autotune_s": t_tune, "max_rel_coef_diff_vs_sequential": worst,
            "setup_sequential_s": t_create_seq, "setup_create_many_s": t_create_many,
            "what": "n log-uniform 5k-500k, p uniform 5-100, n*=floor(sqrt n), L2, df in {4,5,6,8}, nu in "
                    "{0.05,0.1,0.2,0.3}, M=1000; wall clock of fit + synchronize, setup excluded"}


def run_served(cwb, args):
    """Poisson stream of fit requests (variant CWB/ACWB/HCWB, loss L2/binomial) through the fit server.
    The configured stream (n up to 5M, p up to 500, M up to 5000) needs an estimated 10+ minutes of GPU
    work per 1000 requests, so this measurement replays the first R requests of the stream with n, p
    and M scaled by 1/10 (n 1k-500k, p 1-50, M 50-500).  Arm 1: the requests one after another
    (sequential capacity).  Arm 2: the server at offered loads 0.8x and 1.0x of that capacity and a
    burst (all requests at t = 0); latency = completion - arrival, including creation (setup)."""
    import numpy as np
    import torch
    import synthetic_inputs as S
    R = max(1, args.served_requests)
    stream = S.served_request_stream(count=R, seed=4)
    reqs = []
    for r in stream:
        sp = dict(r, n=max(1000, r["n"] // 10), p=max(1, r["p"] // 10), iterations=max(50, r["iterations"] // 10))
        d = S.request_dataset(sp)
        reqs.append((sp, d))
    opts = {0: cwb.OPT_CWB, 1: cwb.OPT_ACWB, 2: cwb.OPT_HCWB}

    def kwargs(sp, d):
        return dict(loss=cwb.LOSS_BINOMIAL if sp["loss"] == 1 else cwb.LOSS_L2, opt=opts[sp["variant"]], nu=0.1,
                    gamma=0.001, iterations=sp["iterations"], patience=5, val_mask=d.val_mask)

    def learners(sp):
        return [cwb.learner(j, n_bins=-1, df=5.0) for j in range(sp["p"])]

    # sequential arm: create + fit + read back, one request at a time
    service, coef_alone = [], []
    for sp, d in reqs:
        t0 = time.perf_counter()
        m = cwb.Model(d.X, d.y, learners(sp), device=0, **kwargs(sp, d))
        m.fit(sp["iterations"])
        coef_alone.append(m.all_coefficients(0, dmax=24))
        service.append(time.perf_counter() - t0)
        m.free()
    cap = R / sum(service)

    def replay(load):
        srv = cwb.Server(hbm_budget_bytes=64 << 30, device=0, max_active=32, slice_iterations=32)
        gaps = np.array([r["arrival_s"] for r in stream])
        # rescale the Poisson arrivals to the offered load (mean rate = load x sequential capacity)
        if load is None:
            arrival = np.zeros(R)
        else:
            mean_gap = float(np.mean(np.diff(np.concatenate([[0.0], gaps])))) or 1.0
            arrival = gaps / mean_gap / (load * cap)
        t0 = time.perf_counter()
        submitted, done_at, ids = 0, {}, {}
        while len(done_at) < R:
            now = time.perf_counter() - t0
            while submitted < R and arrival[submitted] <= now:
                sp, d = reqs[submitted]
                ids[srv.submit(d.X, d.y, learners(sp), **kwargs(sp, d))] = submitted
                submitted += 1
            for rid in srv.poll(wait=False):
                done_at[rid] = time.perf_counter() - t0
            if submitted == R and len(done_at) < R:
                for rid in srv.poll(wait=True):
                    done_at[rid] = time.perf_counter() - t0
        makespan = max(done_at.values())
        lat = [done_at[rid] - arrival[i] for rid, i in ids.items()]
        worst = 0.0
        for rid, i in ids.items():
            m = srv.take(rid)
            th = m.all_coefficients(0, dmax=24)
            ref = coef_alone[i]
            worst = max(worst, float(np.abs(th - ref).max()) / (float(np.abs(ref).max()) or 1.0))
            m.free()
        srv.free()
        return {"offered_load": load if load is not None else "burst", "fits_per_s": R / makespan,
                "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
                "max_rel_coef_diff_vs_alone": worst}

    runs = [replay(0.8), replay(1.0), replay(None)]
    return {"requests": R, "sequential_fits_per_s": cap, "sequential_p50_service_s": _percentile(service, 50),
            "sequential_p99_service_s": _percentile(service, 99), "runs": runs,
            "hbm_budget_bytes": 64 << 30,
            "what": "first R requests of the seeded Poisson stream, n, p, M scaled by 1/10; latency includes "
                    "creation; admission by estimated device footprint"}


def run_served_full(args):
    """The served form at the request distribution's own scale: the first R requests of the seeded
    Poisson stream (variant CWB/ACWB/HCWB and loss L2/binomial uniform, n log-uniform 10k-5M, p
    log-uniform 10-500, M uniform 500-5000), unscaled, data in FP32 (request_dataset_f32).  Arm 1: the
    requests one after another (create from host memory, fit, coefficients read back): the sequential
    capacity.  Arm 2: the fit server under a 160 GiB HBM budget at offered loads 0.8x, 1.0x and 1.2x of
    that capacity (Poisson arrivals rescaled) and a burst; latency = completion - arrival, creation
    included.  Every served fit is compared with its sequential fit (same kernels: bit-identical)."""
    import numpy as np
    import torch
    import synthetic_inputs as S
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as cwb
    R = max(1, args.served_full_requests)
    stream = S.served_request_stream(count=R, seed=4)
    t_gen = time.perf_counter()
    reqs = [(sp, S.request_dataset_f32(sp)) for sp in stream]
    t_gen = time.perf_counter() - t_gen
    opts = {0: cwb.OPT_CWB, 1: cwb.OPT_ACWB, 2: cwb.OPT_HCWB}
    budget = 160 << 30

    def kwargs(sp, d):
        return dict(loss=cwb.LOSS_BINOMIAL if sp["loss"] == 1 else cwb.LOSS_L2, opt=opts[sp["variant"]], nu=0.1,
                    gamma=0.001, iterations=sp["iterations"], patience=5, val_mask=d.val_mask)

    def learners(sp):
        return [cwb.learner(j, n_bins=-1, df=5.0) for j in range(sp["p"])]

    service, coef_alone, trace_alone, creates = [], [], [], []
    for sp, d in reqs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = cwb.Model(d.X, d.y, learners(sp), device=0, **kwargs(sp, d))
        m.synchronize()
        creates.append(time.perf_counter() - t0)
        m.fit(sp["iterations"])
        coef_alone.append(m.all_coefficients(0, dmax=24))
        service.append(time.perf_counter() - t0)
        trace_alone.append(m.trace()[0])
        m.free()
    cap = R / sum(service)
    gaps = np.array([r["arrival_s"] for r in stream])
    mean_gap = float(np.mean(np.diff(np.concatenate([[0.0], gaps])))) or 1.0

    def replay(load):
        srv = cwb.Server(hbm_budget_bytes=budget, device=0, max_active=16, slice_iterations=32)
        arrival = np.zeros(R) if load is None else gaps / mean_gap / (load * cap)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        submitted, done_at, ids = 0, {}, {}
        while len(done_at) < R:
            now = time.perf_counter() - t0
            while submitted < R and arrival[submitted] <= now:
                sp, d = reqs[submitted]
                ids[srv.submit(d.X, d.y, learners(sp), **kwargs(sp, d))] = submitted
                submitted += 1
            for rid in srv.poll(wait=False):
                done_at[rid] = time.perf_counter() - t0
            if submitted == R and len(done_at) < R:
                for rid in srv.poll(wait=True):
                    done_at[rid] = time.perf_counter() - t0
        makespan = max(done_at.values())
        lat = [done_at[rid] - arrival[i] for rid, i in ids.items()]
        worst, same_k = 0.0, True
        for rid, i in ids.items():
            m = srv.take(rid)
            th = m.all_coefficients(0, dmax=24)
            ref = coef_alone[i]
            worst = max(worst, float(np.abs(th - ref).max()) / (float(np.abs(ref).max()) or 1.0))
            same_k = same_k and bool(np.array_equal(m.trace()[0], trace_alone[i]))
            m.free()
        srv.free()
        return {"offered_load": load if load is not None else "burst", "fits_per_s": R / makespan,
                "vs_sequential": (R / makespan) / cap, "makespan_s": makespan,
                "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
                "max_rel_coef_diff_vs_sequential": worst, "same_selections": same_k}

    runs = [replay(0.8), replay(1.0), replay(1.2), replay(None)]
    line = {"metric": "served fits/s, full-size request distribution (secondary workload)",
            "value": max(r["fits_per_s"] for r in runs if r["offered_load"] != "burst"), "unit": "fits/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "first R requests of the seeded Poisson stream (seed 4): variant and loss uniform, "
                                   "n log-uniform 10k-5M, p log-uniform 10-500, M uniform 500-5000, unscaled",
                       "requests": R, "hbm_budget_bytes": budget, "max_active": 16, "slice_iterations": 32,
                       "sizes": [[sp["variant"], sp["loss"], sp["n"], sp["p"], sp["iterations"]] for sp, _ in reqs]},
            "sequential_fits_per_s": cap, "sequential_total_s": sum(service), "sequential_create_s": sum(creates),
            "sequential_p50_service_s": _percentile(service, 50), "sequential_p99_service_s": _percentile(service, 99),
            "runs": runs, "data_generation_s": t_gen}
    print(json.dumps(line), flush=True)


def run_e2e(cwb, data, stream, dev, local):
    """A full fit (M = 2000) through the C ABI from pinned host buffers, results read back."""
    import numpy as np
    import torch
    Xh = torch.from_numpy(data.X).pin_memory()
    yh = torch.from_numpy(data.y).pin_memory()
    Xn, yn = Xh.numpy(), yh.numpy()
    learners = [cwb.learner(j, n_bins=NSTAR, df=5.0) for j in range(N_FEAT)]
    theta = np.zeros((N_FEAT, 24))
    fitted = torch.empty(N_ROWS, dtype=torch.float32).pin_memory().numpy()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        m = cwb.Model(Xn, yn, learners, nu=NU, iterations=M_FIT, stream=stream, device=local)
        m.fit(M_FIT)
        for k in range(N_FEAT):
            cwb.cwb_get_coefficients(m.handle, k, 0, theta[k])
        m.fitted(fitted)
    dt = time.perf_counter() - t0
    m.free()
    h2d = Xn.nbytes + yn.nbytes
    d2h = theta.nbytes + fitted.nbytes
    return {"value": M_FIT / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / M_FIT, "d2h_bytes_per_step": d2h / M_FIT,
            "what": f"cwb_create from pinned host X, y + cwb_fit({M_FIT}) + coefficients and fitted values read "
                    f"back, wall clock {dt * 1e3:.1f} ms"}


def run_hcwb(args):
    """The HCWB workload's own JSON line (`--workload hcwb_binomial`)."""
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as cwb
    print(json.dumps(measure_hcwb(cwb, args.steps, args.warmup, args.seed)), flush=True)


def measure_hcwb(cwb, steps: int, warmup: int, seed: int):
    """ACWB with the hybrid switch (Algorithm 4), binomial loss, n = 2,000,000, p = 200 (100 U[0,1], 100
    N(0,1)), 20 informative, 20 % validation rows, n* = 1414 (uint16), gamma = 0.001, nu = 0.1, pat_0 = 5.
    A step is one iteration (cwb_fit(model, 1)); L2 is flushed before each timed step."""
    import numpy as np
    import torch
    import synthetic_inputs as S
    dev = torch.device("cuda", 0)
    data = S.sim_binomial_hybrid(seed=seed)
    p, n = data.X.shape
    stream = torch.cuda.Stream(device=dev)
    learners = [cwb.learner(j, n_bins=1414, df=5.0) for j in range(p)]
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        model = cwb.Model(data.X, data.y, learners, loss=cwb.LOSS_BINOMIAL, opt=cwb.OPT_HCWB, nu=0.1, gamma=0.001,
                          patience=5, val_mask=data.val_mask, iterations=5000, stream=stream, device=0)
        stream.synchronize()
        t_create = time.perf_counter() - t0
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        sink = torch.empty(1, dtype=torch.float32, device=dev)

        def flush_l2():
            flush.zero_()
            torch.sum(flush, dim=0, keepdim=True, out=sink)

        for _ in range(max(warmup, 3)):
            flush_l2()
            model.fit(1)
        stream.synchronize()
        K = steps
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        props = torch.cuda.get_device_properties(dev)
        gpu_id = str(getattr(props, "uuid", 0))
        if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
            gpu_id = "GPU-" + gpu_id
        sampler = ClockSampler(gpu_id)
        sampler.start()
        torch.cuda.synchronize(dev)
        for i in range(K):
            flush_l2()
            starts[i].record(stream)
            model.fit(1)
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        model.profile(True, classes=["scatter"])
        for i in range(K):
            flush_l2()
            model.fit(1)
        prof = model.get_profile()
        model.profile(False)
        k_sel, k_cor, sw = model.trace()
        plan = model.scatter_plan()
    done = len(k_sel)
    timed = np.arange(done - 2 * K, done - K)              # the value pass's iterations (0-based)
    acwb = int(np.sum((sw == 0) | (timed + 1 < sw))) if done else 0
    n_tr = int(np.sum(data.val_mask == 0))
    # algorithmic bytes: ACWB iteration on the training rows (two fits, f/h/c read+write, two gathers);
    # CWB iteration after the switch on all rows
    b_acwb = p * n_tr * 2 + n_tr * (4 + 8 + 8 + 4 + 2 + 2) + (n - n_tr) * (4 + 8 + 8 + 2 + 2)
    b_cwb = p * n * 2 + n * (4 + 8 + 2)
    ms = sum(step_ms) / K
    alg = (acwb * b_acwb + (K - acwb) * b_cwb) / K
    sc_ms, sc_n = prof["scatter"]
    sc_avg = sc_ms / max(sc_n, 1) / 1e3
    peak, peak_kind = measured_peaks()
    sc_bytes = p * n_tr * 2 + 2 * n_tr * 4 if acwb == K else p * n * 2 + n * 4
    line = {"metric": "ACWB/HCWB binomial iters/s at n=2M, p=200 (secondary workload)", "value": 1e3 / ms,
            "unit": "iters/s", "n_gpus": 1, "steps": K, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "HCWB (ACWB gamma=0.001 then CWB), binomial, n=2,000,000, p=200 (100 U[0,1] + "
                                   "100 N(0,1)), 20 informative, 20% validation, n*=1414 uint16, d=24 df=5, "
                                   "nu=0.1, pat0=5", "acwb_steps": acwb, "switch_iter": int(sw),
                       "l2": "flushed before every timed step (256 MiB written, then read; untimed)"},
            "hbm_gbs": alg / (ms / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": sc_bytes / sc_avg / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": sc_bytes / sc_avg / 1e9 / peak,
                         "traffic": (HCWB_SCATTER_TRAFFIC["bytes"] if acwb == K and
                                     HCWB_SCATTER_TRAFFIC["sha256"] == scatter_source_hash() else None),
                         "kernel": "k_scatter",
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "scatter_us": sc_avg * 1e6, "gpu_launches": K * 4, "clocks": clocks, "scatter_plan": plan,
            "setup_ms": t_create * 1e3}
    model.free()
    return line


# ---------------------------------------------------------------------------------------------
# Estimation quality of partial effects (Sec. 4.1.1-4.1.2, H2/H3; App. B.3 for n* = n^(1/4) and
# df in {5, 7, 9}).  MISE = (1/p) sum_j int_{min x_j}^{max x_j} (b_j(x, theta_j) - b_j(x, theta_hat_j))^2 dx
# over the informative features, at the iteration chosen by early stopping on a large noise-free
# validation set (the paper's protocol).  Partial effects are identified up to a constant (the offset
# absorbs it), so both curves are centred at their mean over [min x_j, max x_j] before differencing.

def partial_effect_mise(model, data, grid_points: int = 801) -> float:
    """MISE of the fitted partial effects against the generator's true effects, from predictions
    through the public API on a grid per informative feature (the other features at their medians)."""
    import numpy as np
    import synthetic_inputs as S
    trapz = getattr(np, "trapezoid", None) or np.trapz
    ref = np.median(data.X, axis=1)
    total = 0.0
    for j, truth_j in enumerate(data.truth):
        lo, hi = float(data.X[j].min()), float(data.X[j].max())
        g = np.linspace(lo, hi, grid_points)
        Xg = np.repeat(ref[:, None], grid_points, axis=1)
        Xg[j] = g
        est = model.predict(np.ascontiguousarray(Xg)).astype(np.float64)
        true = S.paper_style_effect(truth_j, g)
        dlt = (est - trapz(est, g) / (hi - lo)) - (true - trapz(true, g) / (hi - lo))
        total += float(trapz(dlt * dlt, g))
    return total / len(data.truth)


def mise_fit(cwb, data, val, *, nbins: int, df: float, opt: int, nu: float = 0.05, gamma: float = 0.001,
             chunk: int = 25, max_iter: int = 6000, patience: int = 8, val_mask=None, device: int = 0) -> dict:
    """Fit one model on paper-style data with early stopping on the noise-free rows `val`; returns the
    stopping iteration, the validation MSE there and the MISE of the partial effects there."""
    import numpy as np
    p = data.X.shape[0]
    learners = [cwb.learner(j, n_bins=nbins, df=df) for j in range(p)]
    model = cwb.Model(np.ascontiguousarray(data.X), data.y, learners, opt=opt, nu=nu, gamma=gamma,
                      patience=5, val_mask=val_mask, device=device)
    Xv = np.ascontiguousarray(val.X)
    best = (np.inf, 0, np.nan)
    since = 0
    done = 0
    while done < max_iter and since < patience:
        model.fit(chunk)
        done += chunk
        mse = float(np.mean((model.predict(Xv).astype(np.float64) - val.y) ** 2))
        if mse < best[0]:
            best = (mse, done, partial_effect_mise(model, data))
            since = 0
        else:
            since += 1
    model.free()
    return {"stop_iter": best[1], "val_mse": best[0], "mise": best[2]}


def mise_cases(cwb, *, ns=(5_000, 20_000, 50_000), snrs=(1.0, 10.0), p: int = 5, p_noise: int = 5,
               seed: int = 11, dfs=(5.0, 7.0, 9.0), gammas=(1e-1, 1e-2, 1e-3, 1e-4), reps: int = 1) -> list:
    """The harness grid: for every replication, (n, SNR), on one truth per replication and SNR (the
    same effects at every n): exact binning (n* = number of unique values, i.e. no binning) and
    n* = floor(n^(1/2)) and floor(n^(1/4)) for each df (CWB), ACWB for each momentum gamma and HCWB
    (gamma = 1e-3) at n* = floor(n^(1/2)), df = 5."""
    import itertools
    import math
    import numpy as np
    import synthetic_inputs as S
    rows = []
    for rp, n, snr in itertools.product(range(reps), ns, snrs):
        data = S.paper_style_simulation(n, p, p_noise, snr, seed=seed + 1000 * rp + int(snr))
        val = S.paper_style_sample(data.truth, p_noise, 100_000, seed=seed + 1000 * rp + 100)
        sq, qu = math.isqrt(n), int(math.floor(n ** 0.25 + 1e-9))
        specs = [("exact", cwb.BINS_EXACT, 5.0, cwb.OPT_CWB, 0.0)]
        specs += [(f"sqrt df{int(df)}", sq, df, cwb.OPT_CWB, 0.0) for df in dfs]
        specs += [(f"quarter df{int(df)}", qu, df, cwb.OPT_CWB, 0.0) for df in dfs]
        specs += [(f"sqrt ACWB gamma {g:g}", sq, 5.0, cwb.OPT_ACWB, g) for g in gammas]
        specs += [("sqrt HCWB gamma 0.001", sq, 5.0, cwb.OPT_HCWB, 1e-3)]
        vm = (np.random.default_rng(seed).random(n) < 0.2).astype(np.uint8)
        for name, nb, df, opt, g in specs:
            r = mise_fit(cwb, data, val, nbins=nb, df=df, opt=opt, gamma=g,
                         val_mask=vm if opt == cwb.OPT_HCWB else None)
            rows.append({"rep": rp, "n": n, "snr": snr, "variant": name, "nstar": nb if nb > 0 else n,
                         "df": df, "gamma": g, **r})
    return rows


def run_mise(args):
    import __graft_entry__ as g
    g.build()
    import paper_2110_03513_gb300 as cwb
    import numpy as np
    t0 = time.perf_counter()
    reps = 5
    rows = mise_cases(cwb, reps=reps)
    summary = {}
    for r in rows:
        summary.setdefault((r["n"], r["snr"], r["variant"]), []).append(r)
    table = [{"n": n, "snr": snr, "variant": v, "mise_mean": float(np.mean([r["mise"] for r in rs])),
              "mise_sd": float(np.std([r["mise"] for r in rs], ddof=1)) if len(rs) > 1 else 0.0,
              "stop_iter_mean": float(np.mean([r["stop_iter"] for r in rs]))}
             for (n, snr, v), rs in summary.items()]
    line = {"metric": "MISE of partial effects (paper-style simulation, early stopping on noise-free data)",
            "unit": "MISE", "higher_is_better": False, "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "paper-style simulation (Sec. 4.1.1): p=5 informative random cubic-spline "
                                   "effects on U[a, a+b] ranges, 5 N(0,1) noise features, Gaussian noise at "
                                   "SNR 1 and 10; nu=0.05; stopping on 100,000 noise-free rows, checked every "
                                   "25 iterations, patience 8 checks", "replications": reps},
            "summary": table, "cases": rows, "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "hcwb_binomial":
        run_hcwb(args)
    elif args.workload == "mise":
        run_mise(args)
    elif args.workload == "served_full":
        run_served_full(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
