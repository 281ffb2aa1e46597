"""Benchmark: classical CG solves of a synthetic Q1 finite-element system.

Workload (one step = one complete solve): the trilinear hexahedral (Q1,
27-point) stiffness matrix of -div(rho grad u) on a 64^3 interior grid
(n = 262,144, nnz = 6,859,000), element densities rho = exp(Z), Z ~ N(0,1)
from the seed, FP64 CSR, b = A x* with x* ~ U(-1,1), x0 = 0, plain
unpreconditioned CG to relative residual 1e-10.  These seeded matrices stand
in for the paper's finite-element gravity matrices (Sec. 5.1), which are not
available.

Printed (rank 0, one JSON line): solves/s with inputs resident in HBM
(``value``), end-to-end solves/s through the C ABI with host buffers
(``e2e``), the roofline of the solve kernel, the CSR product alone in GB/s,
NVML board energy per solve, p50/p99 latency, SM clocks during the timed
region, and the oracle timed on the host cores (``cpu_baseline``).

``--impl reference`` times the CPU oracle (the plain FP64 statement of the
same method) on the same workload instead.

Multi-GPU: one process per GPU (torchrun); every rank solves its own
independently seeded system (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import glob
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("CG solves/s and SpMV HBM GB/s (% of roofline), joules/solve, p50/p99 latency at rel-res 1e-10")
GRID_N = 64
SIGMA = 1.0
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20  # > the 126.5 MiB L2
# FP64 FMA peak of one GB300 (152 SMs x ~2 DFMA/clk x 2 flop at 2.07 GHz);
# measured 600.5 G DFMA/s with an independent-chain probe.
FP64_PEAK_GFLOPS = 1201.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-solves", type=int, default=200)
    ap.add_argument("--grid", type=int, default=GRID_N,
                    help="grid edge of the Q1 system (64 is the benchmark workload; others for profiling)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- counters

def algorithmic_bytes_per_iter(n: int, nnz: int) -> int:
    """One FP64 CG step: the CSR product (12 B per entry + 4 B per row
    pointer) plus 88 B per row of vector traffic (p gather 8, q write 8;
    x, r read+write 32, p, q read 16; r read 8, p read+write 16)."""
    return 12 * nnz + 4 * (n + 1) + 88 * n


def flops_per_iter(n: int, nnz: int) -> int:
    return 2 * nnz + 10 * n


def spmv_bytes(n: int, nnz: int) -> int:
    """y = A x: values and columns (12 B per entry), row pointers, x read once, y written."""
    return 12 * nnz + 4 * (n + 1) + 16 * n


def source_sha() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2112_10823_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = source_sha()
    for line in open(path):
        if not line.startswith("traffic "):
            continue
        kv = dict(tok.split("=", 1) for tok in line.split()[1:] if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("source_sha") == sha:
            return float(kv["dram_bytes_per_launch"])
    return None


def gpu_uuid(torch_dev: int):
    """'GPU-xxxxxxxx-...' of CUDA device `torch_dev` (None if unknown)."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(torch_dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def smi_id(torch_dev: int) -> str:
    u = gpu_uuid(torch_dev)
    if u:
        return u
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if torch_dev < len(ids):
            return ids[torch_dev]
    return str(torch_dev)


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, torch_dev: int):
        self.idx = smi_id(torch_dev)
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


class Energy:
    """NVML board energy counter (millijoules), read only."""

    def __init__(self, torch_dev: int):
        self.ok = False
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            handle = ctypes.c_void_p()
            uuid = gpu_uuid(torch_dev)
            rc = 1
            if uuid:
                rc = self.nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(handle))
            if rc != 0 and not os.environ.get("CUDA_VISIBLE_DEVICES"):
                rc = self.nv.nvmlDeviceGetHandleByIndex_v2(torch_dev, ctypes.byref(handle))
            if rc != 0:
                return
            self.h = handle
            self.ok = True
        except Exception:
            self.ok = False

    def read_j(self):
        if not self.ok:
            return None
        v = ctypes.c_ulonglong(0)
        if self.nv.nvmlDeviceGetTotalEnergyConsumption(self.h, ctypes.byref(v)) != 0:
            return None
        return v.value / 1000.0


# ----------------------------------------------------------------- workload

def make_problem(seed: int, grid: int = GRID_N):
    import fe_inputs as fi
    A = fi.q1(grid, SIGMA, seed)
    xs = fi.xstar(seed, A.n)
    return A, xs


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(seed: int, rank: int) -> int:
    """Seed of the system a rank solves: every replica gets its own system."""
    return seed + rank


def max_over_ranks(t: float, pg, device) -> float:
    """The slowest rank's time (the whole job ends when it ends)."""
    if pg is None:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    pg.all_reduce(tt, op=pg.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(steps: int, world: int, t_max: float) -> float:
    """Solves per second of the whole job: all ranks' solves over the slowest rank's time."""
    return steps * world / t_max


def run_reference(args):
    """The oracle (plain FP64 sequential C) on the same workload, host cores."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    import oracle
    A, xs = make_problem(args.seed, args.grid)
    b = oracle.spmv(A, xs)
    times, iters = [], 0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.cg(A, b, tol=TOL, maxit=10 * A.n)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
        iters = r.iters
    tot = sum(times)
    value = len(times) / tot
    sample = f"{len(times)} full oracle solves of the workload (each step one solve, {iters} iterations)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"Q1 27-point FE, {args.grid}^3 grid, lognormal rho (sigma=1), FP64 CSR, CG to 1e-10",
                   "n": A.n, "nnz": A.nnz, "iters": iters, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(A, xs, budget_s: float = 10.0):
    import oracle
    b = oracle.spmv(A, xs)
    n_done, t_tot, iters = 0, 0.0, 0
    while n_done == 0 or t_tot < budget_s:
        t0 = time.perf_counter()
        r = oracle.cg(A, b, tol=TOL, maxit=10 * A.n)
        t_tot += time.perf_counter() - t0
        n_done += 1
        iters = r.iters
    return {"value": n_done / t_tot, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_done} complete FP64 oracle solves of the same workload ({iters} iterations each), "
                      f"single thread, {t_tot:.1f} s"}


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import paper_2112_10823_gb300 as cg

    seed = replica_seed(args.seed, rank)
    A, xs = make_problem(seed, args.grid)
    n, nnz = A.n, A.nnz
    stream = torch.cuda.current_stream(dev)
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    va = torch.from_numpy(A.val).to(dev)
    h = cg.cg_create(rp, ci, va, stream=stream)
    del rp, ci, va
    xs_d = torch.from_numpy(xs).to(dev)
    b = torch.empty_like(xs_d)
    cg.cg_spmv(h, xs_d, b)                       # b = A x*
    x = torch.zeros_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def one_solve():
        x.zero_()
        return cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)

    for _ in range(args.warmup):
        res = one_solve()
    assert res.status == cg.CG_OK, res
    iters = res.iters

    # ---- timed region: K solves, L2 flushed before each, events around each solve
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k)
            x.zero_()
            ev[k][0].record(stream)
            res = cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if pg:
        pg.barrier()
    solve_ms = [s.elapsed_time(e) for s, e in ev]
    dev_time = sum(solve_ms) / 1000.0
    assert res.status == cg.CG_OK and res.relres <= TOL, res
    t_max = max_over_ranks(dev_time, pg, dev)
    value = whole_job_rate(args.steps, world, t_max)

    # ---- end to end through the C ABI with pinned host buffers
    b_host = torch.empty(n, dtype=torch.float64, pin_memory=True)
    b_host.copy_(b.cpu())
    x_host = torch.zeros(n, dtype=torch.float64, pin_memory=True)
    for _ in range(2):
        x_host.zero_()
        cg.cg_solve(h, b_host, x_host, tol=TOL, maxit=10 * n)
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x_host.zero_()
        r2 = cg.cg_solve(h, b_host, x_host, tol=TOL, maxit=10 * n)
    t_e2e = time.perf_counter() - t0
    assert r2.status == cg.CG_OK
    t_e2e = max_over_ranks(t_e2e, pg, dev)
    e2e = {"value": whole_job_rate(args.steps, world, t_e2e), "unit": "solves/s", "h2d_bytes_per_step": 16 * n,
           "d2h_bytes_per_step": 8 * n}

    # ---- latency percentiles and board energy over back-to-back solves
    energy = Energy(local)
    lat = []
    e0 = energy.read_j()
    tl0 = time.perf_counter()
    for _ in range(args.latency_solves):
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x.zero_()
        s_ev.record(stream)
        cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)
        e_ev.record(stream)
        e_ev.synchronize()
        lat.append(s_ev.elapsed_time(e_ev))
    tl = time.perf_counter() - tl0
    e1 = energy.read_j()
    joules = (e1 - e0) / args.latency_solves if (e0 is not None and e1 is not None) else None
    watts = (e1 - e0) / tl if (e0 is not None and e1 is not None) else None

    # ---- CSR product alone (L2 flushed before each call)
    yv = torch.empty_like(b)
    for _ in range(3):
        cg.cg_spmv(h, xs_d, yv)
    sp = []
    for k in range(20):
        flush.fill_(k)
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        cg.cg_spmv(h, xs_d, yv)
        e_ev.record(stream)
        sp.append((s_ev, e_ev))
    torch.cuda.synchronize()
    spmv_ms = float(np.mean([s.elapsed_time(e) for s, e in sp]))
    hbm_peak, peak_kind = peaks()
    spmv_gbs = spmv_bytes(n, nnz) / (spmv_ms * 1e-3) / 1e9

    # ---- roofline of the solve kernel (one launch per solve)
    launch_s = dev_time / args.steps
    bytes_launch = iters * algorithmic_bytes_per_iter(n, nnz)
    flops_launch = iters * flops_per_iter(n, nnz)
    achieved_gbs = bytes_launch / launch_s / 1e9
    traffic = recorded_traffic("cg_solve_kernel<false>", f"q1_{args.grid}")

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    base = None if args.no_cpu_baseline else cpu_baseline(A, xs)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"Q1 27-point FE, {args.grid}^3 grid, lognormal rho (sigma=1), FP64 CSR, CG to 1e-10",
                   "n": n, "nnz": nnz, "iters": iters, "tol": TOL, "x0": "zero",
                   "l2": "flushed before every timed solve (256 MiB write)", "parallelism": f"replicas x{world}"},
        # The 64^3 system stays in L2 during a solve (DRAM traffic is ~2 % of the
        # algorithmic bytes), so its kernel is bound by the FP64 pipe, not HBM.
        "roofline": {"bound": "alu", "achieved": flops_launch / launch_s / 1e9, "peak": FP64_PEAK_GFLOPS,
                     "unit": "GFLOP/s", "frac": flops_launch / launch_s / 1e9 / FP64_PEAK_GFLOPS,
                     "traffic": traffic, "peak_source": "measured (FP64 FMA probe)",
                     "kernel": "cg_solve_kernel<false>", "algorithmic_gbs": achieved_gbs,
                     "algorithmic_gbs_frac_of_hbm": achieved_gbs / hbm_peak, "hbm_peak_source": peak_kind},
        "spmv": {"gbs": spmv_gbs, "frac": spmv_gbs / hbm_peak, "ms": spmv_ms, "bytes": spmv_bytes(n, nnz),
                 "l2": "flushed before every call"},
        "energy": {"joules_per_solve": joules, "avg_watts": watts, "source": "NVML board energy",
                   "solves": args.latency_solves},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "solves": len(lat)},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
        "gpu": {"name": torch.cuda.get_device_name(dev), "uuid": gpu_uuid(local)},
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    h.close()
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
