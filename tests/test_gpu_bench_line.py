"""The benchmark's GPU arm on small workloads: one JSON line per run with the
keys a reader of the line relies on (the roofline, the end-to-end figure,
the clocks, the launch count), for a single solve, the batch and the served
stream."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         cwd=ROOT, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = [json.loads(ln) for ln in res.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, res.stdout[-3000:]
    return lines[0]


def test_single_solve_line():
    d = _line("--matrix", "lap7", "--grid", "24", "--steps", "3", "--warmup", "3", "--no-variants",
              "--no-cpu-baseline", "--latency-solves", "5")
    assert d["unit"] == "solves/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["dtype"] == "f64"
    assert abs(d["ms_per_step"] - 1000.0 / d["value"]) <= 1e-6 * d["ms_per_step"]
    r = d["roofline"]
    assert r["bound"] in ("hbm", "alu") and r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-9 * max(1.0, r["frac"])
    assert d["solve"]["iters"] > 0 and d["accuracy"]["relres_true"] <= 1e-10 * 1.0000001
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 2 * 8 * 24 ** 3 and e["d2h_bytes_per_step"] == 8 * 24 ** 3
    assert d["gpu_launches"] >= 1 and "sm_mhz" in d["clocks"] and d["cpu_baseline"] is None
    assert d["spmv"]["frac"] > 0 and set(d["blas1"]) >= {"dot_5000000", "axpy_5000000", "ewmul_5000000"}


def test_batch_line():
    d = _line("--workload", "batch", "--batch-count", "8", "--budget-gb", "2", "--steps", "1", "--warmup", "1")
    assert d["unit"] == "solves/s" and d["value"] > 0 and d["config"]["systems"] == 8
    assert d["accuracy"]["max_relres_true"] <= 1e-10 * 1.0000001
    assert d["roofline"]["kernel"] == "cg_batch_kernel<false, false>" and d["roofline"]["frac"] > 0
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0


def test_serve_line():
    d = _line("--workload", "serve", "--serve-rate", "200", "--serve-seconds", "0.1", "--budget-gb", "2",
              "--precision", "mixed")
    assert d["unit"] == "solves/s" and d["value"] > 0
    assert d["latency_ms"]["p50"] > 0 and d["latency_ms"]["p99"] >= d["latency_ms"]["p50"]
    assert d["fp64_fifo"]["solves_per_s"] > 0
