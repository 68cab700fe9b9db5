"""The bench's reference arm (the FP64 oracle on host cores) honours the JSON-line contract, and
under a multi-rank launch only rank 0 prints.  No GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "iters/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["n"] == 1_000_000 and d["config"]["p"] == 50 and d["config"]["nstar"] == 1000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_cpu_baseline_reports_one_thread_and_openmp_figures():
    """The bench's CPU baseline times the oracle on one thread and with its learner loop on every core,
    and names the host CPU (here on a small sample so that the test stays quick)."""
    sys.path.insert(0, ROOT)
    import bench
    import synthetic_inputs as S
    data = S.additive_regression(20_000, 50, 10, seed=1, dtype=S.np.float32)
    cb = bench.cpu_baseline_full(data, iters=2)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert cb["nproc"] >= 1 and isinstance(cb["cpu"], str) and cb["cpu"]
    mt = cb["openmp"]
    assert mt["value"] > 0 and 1 <= mt["cores"] <= cb["nproc"] and mt["unit"] == cb["unit"]
