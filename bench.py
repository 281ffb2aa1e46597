"""Benchmark: classical CG solves of synthetic Q1 finite-element systems.

Headline workload (one step = one complete solve): the trilinear hexahedral
(Q1, 27-point) stiffness matrix of -div(rho grad u) on a 160^3 interior grid
(n = 4,096,000, nnz = 109,215,352), element densities rho = exp(Z), Z ~ N(0,1)
from the seed, FP64 CSR, b = A x* with x* ~ U(-1,1), x0 = 0, plain
unpreconditioned CG to relative residual 1e-10 -- the largest configuration
that fits one GPU.  These seeded matrices stand in for the paper's
finite-element gravity matrices (Sec. 5.1), which are not available.

Printed (rank 0, one JSON line): solves/s with inputs resident in HBM
(``value``), end-to-end solves/s through the C ABI with host buffers
(``e2e``), the roofline of the solve kernel (HBM bound at 160^3, with the
FP64-pipe fraction against the FP64 peak measured on the same GPU), the CSR
product alone in GB/s, the BLAS-1 kernels, NVML board energy per solve,
p50/p99 latency, SM clocks during the timed region, the oracle timed on all
host cores (``cpu_baseline``), and ``variants``: the same system in mixed
precision (with and without the Jacobi preconditioner), the 64^3 system (FP64,
resident in L2: held against the FP64 pipe), the 16^3 7-point Laplacian, the
batch of 256 uneven systems (FP64 and mixed) and a short served Poisson
stream, each beside plain FP64 CG on the same GPU.

``--impl reference`` times the oracle (the plain FP64 statement of the method,
on all host cores) on the same workload: whole solves, one per step.

Multi-GPU: one process per GPU; every rank solves its own independently
seeded system (weak scaling, no collective on the data path).  With
``--gpus N > 1`` and no torchrun environment the script starts N local ranks
under torchrun itself.
"""
from __future__ import annotations

import argparse
import ctypes
import glob
import hashlib
import json
import math
import os
import socket
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("CG solves/s and SpMV HBM GB/s (% of roofline), joules/solve, p50/p99 latency at rel-res 1e-10")
GRID_N = 160
SIGMA = 1.0
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20  # > the 126.5 MiB L2
ENERGY_MIN_S = 1.0  # board energy and latency percentiles over at least this long
LATENCY_MIN_S = 5.0  # latency percentiles of long solves over at least this long


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="only the headline workload (no variants record)")
    ap.add_argument("--latency-solves", type=int, default=0,
                    help="solves of the latency/energy pass (0: 200, or fewer for solves longer than 25 ms)")
    ap.add_argument("--grid", type=int, default=GRID_N,
                    help="grid edge of the system (160: the headline Q1 system; 64: the L2-resident one)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="fp64: the paper's FP64 CG; mixed: FP32 product with FP64 residual replacement")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve"],
                    help="single: one system per step (default); batch: 256 uneven systems per step; "
                         "serve: Poisson request stream")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="requests per second")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="length of the arrival window")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="device memory budget of the server")
    ap.add_argument("--chunk", type=int, default=50, help="serve: steps per system per round")
    ap.add_argument("--no-autotune", action="store_true", help="batch/serve: built-in group-size model")
    ap.add_argument("--group-target-ms", type=int, default=50, help="batch/serve: solo time a group aims at")
    ap.add_argument("--matrix", default="q1", choices=["q1", "lap7"],
                    help="q1: the Q1 FE system (default); lap7: the 7-point Laplacian (with --grid 16: n = 4096)")
    ap.add_argument("--ctas", type=int, default=0, help="CTAs of the persistent kernel (0: automatic)")
    ap.add_argument("--precond", default="none", choices=["none", "jacobi"],
                    help="none: the paper's plain CG; jacobi: preconditioned by diag(A)")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    return ap.parse_args(argv)


def peaks():
    """Measured HBM copy bandwidth of this machine's GPUs (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
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


def mixed_bytes_per_iter(n: int, nnz: int) -> int:
    """One mixed-precision CG step: FP32 values and column indices (8 B per
    entry), row pointers, and 96 B per row (p32 gather 4, p read 8 and q
    write 8 for the FP64 p.q; x, r read+write 32 and p, q read 16; r read 8,
    p read+write 16, p32 write 4)."""
    return 8 * nnz + 4 * (n + 1) + 96 * n


def replacement_bytes(n: int, nnz: int) -> int:
    """One FP64 residual replacement r = b - A x: the FP64 product (12 B per
    entry, row pointers, x gather 8) plus b read 8 and r write 8 per row."""
    return 12 * nnz + 4 * (n + 1) + 24 * n


def replacements(iters: int, every: int) -> int:
    """Replacements of a mixed solve of `iters` steps: one every `every` steps
    and one before convergence is accepted."""
    return iters // every + 1


def solve_bytes(n: int, nnz: int, iters: int, mixed: bool, every: int = 50, jacobi: bool = False) -> int:
    """Algorithmic bytes of a solve; Jacobi adds the inverse diagonal, read
    in the residual update and in the direction update (16 B per row)."""
    extra = 16 * n * iters if jacobi else 0
    if not mixed:
        return iters * algorithmic_bytes_per_iter(n, nnz) + extra
    return iters * mixed_bytes_per_iter(n, nnz) + replacements(iters, every) * replacement_bytes(n, nnz) + extra


def solve_flops(n: int, nnz: int, iters: int, mixed: bool, every: int = 50, jacobi: bool = False) -> int:
    f = iters * flops_per_iter(n, nnz) + (3 * n * iters if jacobi else 0)
    if mixed:
        f += replacements(iters, every) * (2 * nnz + 2 * n)
    return f


def l2_resident(n: int, nnz: int, mixed: bool) -> bool:
    """Whether the matrix and the vectors of a solve fit in the 126.5 MiB L2."""
    mat = (8 if mixed else 12) * nnz + 4 * (n + 1)
    return mat + 48 * n < 100 * 2**20


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
        if kv.get("kernel") == kernel.replace(" ", "") and kv.get("workload") == workload and kv.get("source_sha") == sha:
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
        sm, mx, reasons, watts = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
                watts.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": float(max(watts)) if watts else None}


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

def make_problem(seed: int, grid: int = GRID_N, matrix: str = "q1"):
    import fe_inputs as fi
    A = fi.q1(grid, SIGMA, seed) if matrix == "q1" else fi.laplace7(grid)
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


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun_command(nproc: int, script: str, argv: list[str], port: int) -> list[str]:
    """The command that runs `script` as `nproc` local ranks (one per GPU)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
            "--master-addr", "127.0.0.1", f"--master-port={port}", script] + list(argv)


def launch_ranks(nproc: int, script: str, argv: list[str]) -> int:
    """Start `nproc` ranks of `script` under torchrun and return its exit code."""
    return subprocess.call(torchrun_command(nproc, script, argv, free_port()))


def workload_name(grid: int, precision: str, precond: str = "none", matrix: str = "q1") -> str:
    prec = "FP64 CSR" if precision == "fp64" else "FP32-value product with FP64 residual replacement every 50 steps"
    method = "CG" if precond == "none" else "Jacobi-preconditioned CG"
    if matrix == "lap7":
        return f"3-D 7-point Laplacian, {grid}^3 grid, Dirichlet, {prec}, x* ~ U(-1,1), {method} from x0 = 0 to 1e-10"
    return f"Q1 27-point FE, {grid}^3 grid, lognormal rho (sigma=1), {prec}, {method} to 1e-10"


def common_config(args, n: int, nnz: int, world: int) -> dict:
    """The workload keys both arms print (identical for the same command line)."""
    big = not l2_resident(n, nnz, args.precision == "mixed")
    return {"workload": workload_name(args.grid, args.precision, args.precond, args.matrix), "n": n, "nnz": nnz,
            "tol": TOL, "x0": "zero", "parallelism": f"replicas x{world}",
            "l2": ("inputs larger than L2, and a 256 MiB write before every timed GPU solve" if big
                   else "flushed before every timed GPU solve (256 MiB write)")}


# ------------------------------------------------------- oracle (host) legs

def host_cpu() -> dict:
    """Model name and logical core count of the host (lscpu; /proc/cpuinfo as a fallback)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model, "nproc": os.cpu_count()}


def oracle_solver(precision: str, precond: str = "none"):
    """The oracle that times a CPU solve: the OpenMP variant on all host cores
    for plain FP64 CG (the configurations' method), the sequential oracle for
    the other variants.  Returns (solve(A, b, maxit, force), cores)."""
    import oracle
    if precond == "none" and precision == "fp64" and oracle.omp_available():
        return (lambda A, b, maxit, force=-1: oracle.omp_cg(A, b, tol=TOL, maxit=maxit, force_iters=force),
                oracle.omp_threads())
    if precond == "jacobi":
        return lambda A, b, maxit, force=-1: oracle.pcg_jacobi(A, b, tol=TOL, maxit=maxit, force_iters=force), 1
    if precision == "mixed":
        return lambda A, b, maxit, force=-1: oracle.cg_mixed(A, b, tol=TOL, maxit=maxit, force_iters=force), 1
    return lambda A, b, maxit, force=-1: oracle.cg(A, b, tol=TOL, maxit=maxit, force_iters=force), 1


def oracle_rate(A, b, precision: str, budget_s: float, iters_full: int, precond: str = "none"):
    """The oracle's solves/s on the host: whole solves when one takes less than
    the budget, else runs of m steps (each with its setup product) whose time
    per step is scaled to an `iters_full`-step solve.  Returns (solves/s,
    cores, description of the sample)."""
    solve, cores = oracle_solver(precision, precond)
    m = 20
    t0 = time.perf_counter()
    solve(A, b, m, m)
    per_step = (time.perf_counter() - t0) / (m + 1)
    who = f"OpenMP oracle on {cores} host cores" if cores > 1 else "oracle, one host core"
    if per_step * (iters_full + 1) <= budget_s:
        n_done, t_tot, its = 0, 0.0, 0
        while n_done == 0 or t_tot < budget_s * 0.5:
            t0 = time.perf_counter()
            r = solve(A, b, 10 * A.n)
            t_tot += time.perf_counter() - t0
            n_done += 1
            its = r.iters
        return n_done / t_tot, cores, f"{n_done} complete solves ({its} iterations each), {who}, {t_tot:.1f} s"
    runs, t_tot = 0, 0.0
    while runs == 0 or t_tot < budget_s:
        t0 = time.perf_counter()
        solve(A, b, m, m)
        t_tot += time.perf_counter() - t0
        runs += 1
    per_step = t_tot / (runs * (m + 1))
    return 1.0 / (per_step * (iters_full + 1)), cores, (
        f"{runs} runs of {m} steps each plus the setup product ({who}, {t_tot:.1f} s), "
        f"time per step scaled to a {iters_full}-step solve")


def run_reference(args):
    """The oracle (plain C, the paper's method as stated; the OpenMP variant on
    every host core) on the same workload: each step one whole solve."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    import oracle
    A, xs = make_problem(args.seed, args.grid, args.matrix)
    b = oracle.omp_spmv(A, xs) if oracle.omp_available() else oracle.spmv(A, xs)
    solve, cores = oracle_solver(args.precision, args.precond)
    times, r = [], None
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = solve(A, b, 10 * A.n)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = len(times) / tot
    who = f"OpenMP oracle on {cores} host cores" if cores > 1 else "oracle, one host core"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": common_config(args, A.n, A.nnz, 1),
        "solve": {"iters": r.iters, "relres_true": r.relres_true},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} whole solves of the workload, one per step "
                                   f"({r.iters} iterations), {who}", "host": host_cpu()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ GPU measurement parts

def timed_solves(cg, h, b, x, n, k, stream, flush=None):
    """k solves from x0 = 0, CUDA events around each (L2 flushed before each
    if `flush`); returns (per-solve ms, last result)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    res = None
    for i in range(k):
        if flush is not None:
            flush.fill_(i)
        x.zero_()
        ev[i][0].record(stream)
        res = cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in ev], res


def energy_pass(cg, h, b, x, n, stream, energy, min_solves: int, min_s: float = ENERGY_MIN_S):
    """Back-to-back solves (at least min_solves and min_s seconds): per-solve
    CUDA-event latencies and NVML board energy per solve."""
    import torch
    torch.cuda.synchronize()
    lat = []
    e0 = energy.read_j()
    t0 = time.perf_counter()
    while len(lat) < min_solves or time.perf_counter() - t0 < min_s:
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x.zero_()
        s_ev.record(stream)
        r = cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)
        e_ev.record(stream)
        e_ev.synchronize()
        assert r.status == cg.CG_OK, r
        lat.append(s_ev.elapsed_time(e_ev))
    tl = time.perf_counter() - t0
    e1 = energy.read_j()
    joules = (e1 - e0) / len(lat) if (e0 is not None and e1 is not None) else None
    watts = (e1 - e0) / tl if (e0 is not None and e1 is not None) else None
    return lat, joules, watts, tl


def idle_power(energy):
    i0, t0 = energy.read_j(), time.perf_counter()
    time.sleep(0.5)
    i1, t = energy.read_j(), time.perf_counter() - t0
    return (i1 - i0) / t if (i0 is not None and i1 is not None) else None


def spmv_alone(cg, h, x, y, stream, flush, reps: int = 20):
    """Mean CUDA-event time (ms) of the product alone, L2 flushed before each call."""
    import torch
    for _ in range(3):
        cg.cg_spmv(h, x, y)
    sp = []
    for k in range(reps):
        flush.fill_(k)
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        cg.cg_spmv(h, x, y)
        e_ev.record(stream)
        sp.append((s_ev, e_ev))
    torch.cuda.synchronize()
    return float(np.mean([s.elapsed_time(e) for s, e in sp]))


def blas1_record(cg, dev, stream, flush, hbm_peak):
    """dot, axpy and element-wise product alone (Sec. 5.2) at the paper's
    largest vector length and at one four times the L2 (L2 flushed before
    each call); bytes: dot 16 per element, axpy and element-wise product 24."""
    import torch
    out = {}
    for nv in (5_000_000, 64_000_000):
        xv = torch.rand(nv, dtype=torch.float64, device=dev)
        yv = torch.rand(nv, dtype=torch.float64, device=dev)
        zv = torch.empty_like(xv)
        outv = torch.zeros(1, dtype=torch.float64, device=dev)
        ops = {"dot": (lambda: cg.cg_dot(xv, yv, outv, stream=stream), 16),
               "axpy": (lambda: cg.cg_axpy(0.5, xv, yv, stream=stream), 24),
               "ewmul": (lambda: cg.cg_ewmul(xv, yv, zv, stream=stream), 24)}
        for name, (fn, bpe) in ops.items():
            for _ in range(3):
                fn()
            tms = []
            for k in range(10):
                flush.fill_(k)
                s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s_ev.record(stream)
                fn()
                e_ev.record(stream)
                e_ev.synchronize()
                tms.append(s_ev.elapsed_time(e_ev))
            ms = float(np.median(tms))
            gbs = bpe * nv / (ms * 1e-3) / 1e9
            out[f"{name}_{nv}"] = {"us": 1000 * ms, "gbs": gbs, "frac": gbs / hbm_peak}
        del xv, yv, zv
    return out


def solve_kernel_name(cg, h, mixed: bool, jac: bool) -> str:
    kind = h.partition_info()[1]
    if kind == cg.CG_SOLVE_KERNEL_CLUSTER:
        return "cg_cluster_kernel"
    small = kind == cg.CG_SOLVE_KERNEL_SMALL_SHARE
    return (f"cg_solve_kernel<{'true' if mixed else 'false'}, {'true' if jac else 'false'}, "
            f"{'true' if small else 'false'}>")


def roofline(n, nnz, iters, launch_s, mixed, jac, kname, workload, hbm_peak, hbm_src, fp64_peak, fp64_src):
    """Roofline of one solve launch: HBM-bound unless the system stays in L2,
    where the FP64 pipe bounds it; both fractions are reported."""
    bytes_launch = solve_bytes(n, nnz, iters, mixed, jacobi=jac)
    flops_launch = solve_flops(n, nnz, iters, mixed, jacobi=jac)
    gbs = bytes_launch / launch_s / 1e9
    gflops = flops_launch / launch_s / 1e9
    traffic = recorded_traffic(kname, workload)
    common = {"traffic": traffic, "kernel": kname, "algorithmic_bytes_per_launch": bytes_launch,
              "flops_per_launch": flops_launch, "launch_ms": 1000.0 * launch_s}
    if l2_resident(n, nnz, mixed):
        return dict({"bound": "alu", "achieved": gflops, "peak": fp64_peak, "unit": "GFLOP/s",
                     "frac": gflops / fp64_peak, "peak_source": fp64_src, "algorithmic_gbs": gbs,
                     "algorithmic_gbs_frac_of_hbm": gbs / hbm_peak, "hbm_peak_source": hbm_src}, **common)
    return dict({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                 "peak_source": hbm_src, "gflops": gflops, "gflops_frac_of_fp64": gflops / fp64_peak,
                 "fp64_peak_source": fp64_src}, **common)


def upload(A, dev):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.row_ptr, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(A.col_idx, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).to(dev))


def single_system_record(cg, A, xs, dev, stream, flush, energy, hbm, fp64, steps, precision="fp64",
                         precond="none", ctas=0, matrix="q1", grid=GRID_N, min_solves=None, x64=None):
    """Solves/s, energy, latency, accuracy and roofline of one system solved
    one step at a time (a variant of the headline line, or the 64^3 / 16^3
    sub-records)."""
    import torch
    mixed, jac = precision == "mixed", precond == "jacobi"
    rp, ci, va = upload(A, dev)
    h = cg.cg_create(rp, ci, va, stream=stream, precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64,
                     preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, ctas=ctas)
    del rp, ci, va
    xs_d = torch.from_numpy(xs).to(dev)
    b = torch.empty_like(xs_d)
    cg.cg_spmv(h, xs_d, b)
    x = torch.zeros_like(b)
    n, nnz = A.n, A.nnz
    ms, res = timed_solves(cg, h, b, x, n, 2, stream)
    assert res.status == cg.CG_OK, (res, cg.last_error(h))
    ms, res = timed_solves(cg, h, b, x, n, steps, stream, flush)
    launch_s = float(np.mean(ms)) / 1000.0
    if min_solves is None:
        min_solves = 200 if launch_s < 0.025 else 3
    lat, joules, watts, tl = energy_pass(cg, h, b, x, n, stream, energy, min_solves)
    kname = solve_kernel_name(cg, h, mixed, jac)
    rec = {"workload": workload_name(grid, precision, precond, matrix), "n": n, "nnz": nnz, "iters": res.iters,
           "value": 1.0 / launch_s, "unit": "solves/s", "ms_per_solve": 1000.0 * launch_s,
           "dtype": "f32+f64" if mixed else "f64", "kernel": kname, "ctas": h.nblocks,
           "energy": {"joules_per_solve": joules, "avg_watts": watts, "solves": len(lat), "seconds": tl},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "solves": len(lat)},
           "accuracy": {"relres_true": res.relres,
                        "err_vs_xstar": float(torch.linalg.vector_norm(x - xs_d) / torch.linalg.vector_norm(xs_d))},
           "roofline": roofline(n, nnz, res.iters, launch_s, mixed, jac, kname, f"{matrix}_{grid}", *hbm, *fp64)}
    if x64 is not None:
        rec["accuracy"]["rel_diff_vs_fp64_solve"] = float(torch.linalg.vector_norm(x - x64)
                                                          / torch.linalg.vector_norm(x64))
    h.close()
    return rec, x


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

    stream = torch.cuda.current_stream(dev)
    hbm_peak, hbm_src = peaks()
    # the FP64 FMA ceiling of this GPU, measured by the library's probe now
    fp64_peak = max(cg.cg_probe_fp64_peak(local) for _ in range(2))
    fp64 = (fp64_peak, "measured on this GPU by cg_probe_fp64_peak before the timed region")

    seed = replica_seed(args.seed, rank)
    A, xs = make_problem(seed, args.grid, args.matrix)
    n, nnz = A.n, A.nnz
    rp, ci, va = upload(A, dev)
    mixed = args.precision == "mixed"
    jac = args.precond == "jacobi"
    h = cg.cg_create(rp, ci, va, stream=stream, precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64,
                     preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, ctas=args.ctas)
    del rp, ci, va
    xs_d = torch.from_numpy(xs).to(dev)
    b = torch.empty_like(xs_d)
    cg.cg_spmv(h, xs_d, b)                       # b = A x*
    x = torch.zeros_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    for _ in range(args.warmup):
        x.zero_()
        res = cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)
    assert res.status == cg.CG_OK, res
    iters = res.iters

    # ---- timed region: K solves, L2 flushed before each, events around each solve
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        solve_ms, res = timed_solves(cg, h, b, x, n, args.steps, stream, flush)
        t_wall = time.perf_counter() - t_wall0
    if pg:
        pg.barrier()
    dev_time = sum(solve_ms) / 1000.0
    assert res.status == cg.CG_OK and res.relres <= TOL, res
    t_max = max_over_ranks(dev_time, pg, dev)
    value = whole_job_rate(args.steps, world, t_max)
    x_fin = x.clone()

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

    # ---- latency percentiles and board energy over back-to-back solves (at
    # least 200 short solves, or LATENCY_MIN_S of long ones, and ENERGY_MIN_S),
    # and the idle board power just before
    energy = Energy(local)
    idle_watts = idle_power(energy)
    launch_s = dev_time / args.steps
    min_solves = args.latency_solves or (200 if launch_s < 0.025 else max(5, math.ceil(LATENCY_MIN_S / launch_s)))
    lat, joules, watts, tl = energy_pass(cg, h, b, x, n, stream, energy, min_solves)

    blas1 = blas1_record(cg, dev, stream, flush, hbm_peak)
    yv = torch.empty_like(b)
    spmv_ms = spmv_alone(cg, h, xs_d, yv, stream, flush)
    spmv_gbs = spmv_bytes(n, nnz) / (spmv_ms * 1e-3) / 1e9

    accuracy = {"relres_true": res.relres, "err_vs_xstar": float(torch.linalg.vector_norm(x_fin - xs_d)
                                                                  / torch.linalg.vector_norm(xs_d))}
    kname = solve_kernel_name(cg, h, mixed, jac)
    roof = roofline(n, nnz, iters, launch_s, mixed, jac, kname, f"{args.matrix}_{args.grid}",
                    hbm_peak, hbm_src, *fp64)
    ctas = h.nblocks
    h.close()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return

    # ---- variants: the same GPU, each beside plain FP64 CG
    variants = None
    if world == 1 and not args.no_variants and args.matrix == "q1" and args.precision == "fp64" \
            and args.precond == "none":
        del yv, flush
        torch.cuda.empty_cache()
        variants = run_variants(args, cg, A, xs, x_fin, dev, stream, energy, (hbm_peak, hbm_src), fp64,
                                {"value": value, "joules_per_solve": joules})

    base = None
    if not args.no_cpu_baseline and world == 1:
        bh = b.cpu().numpy()
        v, cores, sample = oracle_rate(A, bh, args.precision, args.cpu_budget, iters, args.precond)
        base = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample,
                "host": host_cpu()}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": common_config(args, n, nnz, world),
        "solve": {"iters": iters, "kernel": kname, "ctas": ctas},
        "roofline": roof,
        "accuracy": accuracy,
        "spmv": {"gbs": spmv_gbs, "frac": spmv_gbs / hbm_peak, "ms": spmv_ms, "bytes": spmv_bytes(n, nnz),
                 "l2": "flushed before every call", "precision": "fp64", "kernel": "spmv_kernel",
                 "traffic": recorded_traffic("spmv_kernel", f"{args.matrix}_{args.grid}")},
        "blas1": blas1,
        "energy": {"joules_per_solve": joules, "avg_watts": watts, "idle_watts": idle_watts,
                   "joules_per_solve_above_idle": (joules - idle_watts * tl / len(lat)
                                                   if joules is not None and idle_watts is not None else None),
                   "source": "NVML board energy", "solves": len(lat), "seconds": tl},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "solves": len(lat)},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
        "gpu": {"name": torch.cuda.get_device_name(dev), "uuid": gpu_uuid(local)},
        "cpu_baseline": base,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def run_variants(args, cg, A, xs, x64, dev, stream, energy, hbm, fp64, fp64_line):
    """The scope's other rows on the same GPU, each with plain FP64 CG beside
    it: the headline system in mixed precision (plain and Jacobi), the 64^3
    system (FP64, L2-resident: FP64-pipe roofline) and the 16^3 7-point
    Laplacian, the batch of 256 uneven systems (FP64 and mixed, one persistent
    launch each) and a short served Poisson stream."""
    import torch
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    out = {}

    def guarded(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # a failing variant is recorded, the headline line still prints
            out[name] = {"error": f"{type(e).__name__}: {e}"[:400]}
        if isinstance(out[name], dict):
            out[name]["bench_seconds"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()

    def vs_fp64(rec):
        rec["speedup_vs_fp64_cg"] = rec["value"] / fp64_line["value"]
        j, j64 = rec.get("energy", {}).get("joules_per_solve"), fp64_line["joules_per_solve"]
        rec["joules_ratio_vs_fp64_cg"] = j / j64 if j and j64 else None
        return rec

    x64_d = x64.to(dev)
    guarded(f"q1_{args.grid}_mixed", lambda: vs_fp64(single_system_record(
        cg, A, xs, dev, stream, flush, energy, hbm, fp64, 5, "mixed", grid=args.grid, x64=x64_d)[0]))
    guarded(f"q1_{args.grid}_mixed_jacobi", lambda: vs_fp64(single_system_record(
        cg, A, xs, dev, stream, flush, energy, hbm, fp64, 5, "mixed", "jacobi", grid=args.grid, x64=x64_d)[0]))
    del x64_d

    def q1_64():
        A64, xs64 = make_problem(args.seed, 64, "q1")
        rec, _ = single_system_record(cg, A64, xs64, dev, stream, flush, energy, hbm, fp64, 20, grid=64)
        rp, ci, va = upload(A64, dev)
        h = cg.cg_create(rp, ci, va, stream=stream)
        xd = torch.from_numpy(xs64).to(dev)
        y = torch.empty_like(xd)
        ms = spmv_alone(cg, h, xd, y, stream, flush)
        gbs = spmv_bytes(A64.n, A64.nnz) / (ms * 1e-3) / 1e9
        rec["spmv"] = {"gbs": gbs, "frac": gbs / hbm[0], "ms": ms, "bytes": spmv_bytes(A64.n, A64.nnz),
                       "l2": "flushed before every call (the 87.6 MB product barely exceeds L2)"}
        h.close()
        # the three group-wide synchronisations of a small-share step (two
        # sums, one barrier), timed alone on the whole grid
        bar_us, sum_us = cg.cg_probe_group_sync(dev.index or 0, 20000)
        step_us = 1000.0 * rec["ms_per_solve"] / rec["iters"]
        rec["sync_probe"] = {"barrier_us": bar_us, "sum_us": sum_us, "per_step_us": 2 * sum_us + bar_us,
                             "step_us": step_us, "share_of_step": (2 * sum_us + bar_us) / step_us,
                             "source": "cg_probe_group_sync (the solves' group barrier and group sum, one CTA "
                                       "per SM, 20000 of each)"}
        return rec

    guarded("q1_64_fp64", q1_64)

    def lap7_16():
        A16, xs16 = make_problem(args.seed, 16, "lap7")
        return single_system_record(cg, A16, xs16, dev, stream, flush, energy, hbm, fp64, 50, matrix="lap7",
                                    grid=16, min_solves=200)[0]

    guarded("lap7_16_fp64", lap7_16)
    del flush
    torch.cuda.empty_cache()

    systems = []

    def batch(precision):
        if not systems:
            systems.extend(batch_systems(args.seed, args.batch_count, dev))
        return batch_record(cg, systems, dev, stream, energy, hbm[0], precision, "none", steps=3, warmup=1,
                            budget_gb=32.0, autotune=True, group_target_ms=args.group_target_ms,
                            traffic_key=f"batch{args.batch_count}_seed{args.seed}_{precision}")

    guarded("batch256_fp64", lambda: batch("fp64"))
    guarded("batch256_mixed", lambda: batch("mixed"))
    for s in systems:
        s["h"].close()
    systems.clear()
    torch.cuda.empty_cache()
    # the configured stream (2000 requests/s, beyond one GPU's capacity: the
    # sustained rate and the latency under overload) over a quarter second,
    # and a lighter one (100 requests/s) configured for latency below
    # capacity: groups sized for 5 ms solo solves, rounds of 20 steps
    guarded("serve_2000rps_mixed", lambda: serve_record(cg, args.seed, 2000.0, 0.25, dev, stream, energy, hbm[0],
                                                       "mixed", "none", budget_gb=args.budget_gb, chunk=args.chunk,
                                                       autotune=True, group_target_ms=args.group_target_ms))
    guarded("serve_100rps_mixed_5ms", lambda: serve_record(cg, args.seed + 1, 100.0, 1.0, dev, stream, energy,
                                                          hbm[0], "mixed", "none", budget_gb=args.budget_gb,
                                                          chunk=20, autotune=True, group_target_ms=5))
    return out


# ----------------------------------------------------- batched and served

def batch_systems(seed: int, count: int, dev):
    """The uneven batch: edges uniform on {8..48}, own densities and
    manufactured solution per system; matrices and right-hand sides resident
    on the device, with an FP64 handle each (b = A x* on the device)."""
    import torch
    import fe_inputs as fi
    import paper_2112_10823_gb300 as cg
    out = []
    for i, N in enumerate(fi.batch_edges(seed, count)):
        sd = fi.system_seed(seed, i)
        A = fi.q1(int(N), SIGMA, sd)
        rp, ci, va = upload(A, dev)
        h = cg.cg_create(rp, ci, va)
        xs = torch.from_numpy(fi.xstar(sd, A.n)).to(dev)
        b = torch.empty_like(xs)
        cg.cg_spmv(h, xs, b)
        out.append({"N": int(N), "n": A.n, "nnz": A.nnz, "rp": rp, "ci": ci, "va": va, "h": h, "b": b,
                    "x": torch.zeros_like(b), "xs": xs})
    torch.cuda.synchronize()
    return out


def solve_sequential(systems, stream):
    """Plain FP64 CG, one system after another (one cooperative launch each);
    returns (device seconds, iterations per system)."""
    import torch
    import paper_2112_10823_gb300 as cg
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its = []
    e0.record(stream)
    for s in systems:
        s["x"].zero_()
        r = cg.cg_solve(s["h"], s["b"], s["x"], tol=TOL, maxit=10 * s["n"])
        assert r.status == cg.CG_OK, r
        its.append(r.iters)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1000.0, its


def batch_record(cg, systems, dev, stream, energy, hbm_peak, precision, precond, steps, warmup, budget_gb,
                 autotune, group_target_ms, e2e=False, traffic_key=None):
    """The batch per step in one persistent launch (batched API), against the
    same systems solved one after another by cg_solve in FP64.  traffic_key
    names the workload's line in the ncu traffic record (DRAM bytes of one
    whole batch, every round of it), if it has one."""
    import torch
    count = len(systems)
    mixed = precision == "mixed"
    jac = precond == "jacobi"
    solve_sequential(systems, stream)
    x64 = [s["x"].clone() for s in systems]
    j0 = energy.read_j()
    t_seq = 0.0
    t0 = time.perf_counter()
    k_seq = 0
    while k_seq < steps or time.perf_counter() - t0 < ENERGY_MIN_S:
        dt, _ = solve_sequential(systems, stream)
        t_seq += dt
        k_seq += 1
    j1 = energy.read_j()
    seq = {"solves_per_s": count * k_seq / t_seq, "ms_per_batch": 1000.0 * t_seq / k_seq,
           "joules_per_solve": (j1 - j0) / (count * k_seq) if j0 is not None and j1 is not None else None,
           "launches_per_batch": count}
    bt = cg.Batch(precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64, chunk_iters=0, validate=False,
                  budget_bytes=int(budget_gb * 2**30), max_systems=max(1024, count),
                  preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, autotune=autotune,
                  group_target_ms=group_target_ms)
    model = {k: bt.stats()[k] for k in ("autotuned", "cta_bytes_per_s", "group_cta_bytes_per_s", "step_overhead_s",
                                        "group_step_overhead_s", "shape_tuned", "step_kind")}

    def step():
        reqs = [cg.Request(s["rp"], s["ci"], s["va"], s["b"], s["x"], tol=TOL, maxit=10 * s["n"], tag=i)
                for i, s in enumerate(systems)]
        res = bt.wait_all(bt.submit(reqs))
        bad = [r for r in res if r.status != cg.CG_OK or r.relres > TOL]
        assert not bad, bad[:3]
        return res

    for _ in range(warmup):
        res = step()
    st0 = bt.stats()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    with ClockSampler(dev.index or 0) as clk:
        j0 = energy.read_j()
        tw0 = time.perf_counter()
        k = 0
        while k < steps or time.perf_counter() - tw0 < ENERGY_MIN_S:
            flush.fill_(k)
            torch.cuda.synchronize()
            res = step()
            k += 1
        t_wall = time.perf_counter() - tw0
        j1 = energy.read_j()
    steps = k
    st1 = bt.stats()
    rounds = st1["rounds"] - st0["rounds"]
    dev_s = (st1["round_ms_total"] - st0["round_ms_total"]) / 1000.0
    value = count * steps / dev_s
    iters = [r.iters for r in res]
    groups = [r.group for r in res]
    err = max(float(torch.linalg.vector_norm(s["x"] - x) / torch.linalg.vector_norm(x)) for s, x in zip(systems, x64))
    bytes_batch = sum(solve_bytes(s["n"], s["nnz"], it, mixed, jacobi=jac) for s, it in zip(systems, iters))
    flops_batch = sum(solve_flops(s["n"], s["nnz"], it, mixed, jacobi=jac) for s, it in zip(systems, iters))
    achieved = bytes_batch * steps / dev_s / 1e9
    kernel = f"cg_batch_kernel<{'true' if mixed else 'false'}, {'true' if jac else 'false'}>"
    rec = {
        "value": value, "unit": "solves/s", "ms_per_batch": 1000.0 * dev_s / steps, "steps": steps,
        "dtype": "f32+f64" if mixed else "f64",
        "workload": f"batch of {count} Q1 27-point FE systems, grid edges uniform in [8, 48], lognormal rho "
                    f"(sigma=1), own b per system, {'mixed precision' if mixed else 'FP64'}, one persistent launch "
                    f"per batch (CUDA graph), {'Jacobi-preconditioned ' if jac else ''}CG to 1e-10",
        "systems": count, "sum_n": int(sum(s["n"] for s in systems)), "sum_nnz": int(sum(s["nnz"] for s in systems)),
        "iters_min": min(iters), "iters_max": max(iters),
        "groups": {str(g): groups.count(g) for g in sorted(set(groups))},
        "rounds_per_step": rounds / steps, "graph": bool(st1["graph"]), "group_model": model,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak,
                     "traffic": recorded_traffic(kernel, traffic_key) if traffic_key else None,
                     "traffic_per": "batch (the DRAM bytes of all rounds of one batch)",
                     "algorithmic_bytes_per_batch": bytes_batch,
                     "kernel": kernel,
                     "gflops": flops_batch * steps / dev_s / 1e9},
        "accuracy": {"max_relres_true": max(r.relres for r in res), "max_rel_diff_vs_fp64_cg_solve": err},
        "fp64_sequential": seq,
        "speedup_vs_fp64_sequential": value / seq["solves_per_s"],
        "energy": {"joules_per_solve": (j1 - j0) / (count * steps) if j0 is not None and j1 is not None else None,
                   "source": "NVML board energy (whole steps, host admission included)"},
        "joules_ratio_vs_fp64_sequential": None,
        "device_resident_inputs_solves_per_s": count * steps / t_wall,
        "gpu_launches": int(rounds + (count * steps if mixed else 0)),
        "clocks": clk.summary(),
    }
    if rec["energy"]["joules_per_solve"] and seq["joules_per_solve"]:
        rec["joules_ratio_vs_fp64_sequential"] = rec["energy"]["joules_per_solve"] / seq["joules_per_solve"]
    if e2e:
        hosts = []
        for s_ in systems:
            hosts.append({k: s_[k].cpu().pin_memory() for k in ("rp", "ci", "va", "b")})
            hosts[-1]["x"] = torch.zeros(s_["n"], dtype=torch.float64).pin_memory()
        h2d = sum(4 * (s_["n"] + 1) + 12 * s_["nnz"] + 8 * s_["n"] for s_ in systems)
        d2h = sum(8 * s_["n"] for s_ in systems)

        def step_host():
            reqs = [cg.Request(hs["rp"], hs["ci"], hs["va"], hs["b"], hs["x"], tol=TOL, maxit=10 * s_["n"], tag=i)
                    for i, (hs, s_) in enumerate(zip(hosts, systems))]
            res_h = bt.wait_all(bt.submit(reqs))
            assert all(r.status == cg.CG_OK and r.relres <= TOL for r in res_h)
            return res_h

        step_host()
        te0 = time.perf_counter()
        spans = []
        for _ in range(steps):
            res_h = step_host()
            sub0 = min(r.submit_ms for r in res_h)
            adm1 = max(r.admit_ms for r in res_h)
            spans.append((adm1 - sub0, max(r.done_ms for r in res_h) - adm1))
        t_e2e = time.perf_counter() - te0
        rec["e2e"] = {"value": count * steps / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h),
                      "note": "wall clock through cg_batch_submit/wait with every system's CSR arrays and b in pinned "
                              "host memory (admission copies them to the device) and x read back to the host",
                      "admission_ms": float(np.mean([a for a, _ in spans])),
                      "round_and_readback_ms": float(np.mean([r for _, r in spans]))}
    bt.close()
    return rec


def serve_record(cg, seed, rate, seconds, dev, stream, energy, hbm_peak, precision, precond, budget_gb, chunk,
                 autotune, group_target_ms):
    """Continuous batching of a Poisson request stream (served API), against
    a FIFO server of plain FP64 CG solves on the same GPU."""
    import torch
    import fe_inputs as fi
    mixed = precision == "mixed"
    count = max(1, int(round(rate * seconds)))
    t_arr, edges = fi.arrivals(seed, count, rate)
    # request i solves the pool system of its edge with right-hand side k = i % 4
    pool = {}
    for N in sorted(set(int(e) for e in edges)):
        sd = fi.system_seed(seed, 100000 + N)
        A = fi.q1(N, SIGMA, sd)
        rp, ci, va = upload(A, dev)
        h = cg.cg_create(rp, ci, va)
        bs = []
        for k in range(4):
            xs = torch.from_numpy(fi.xstar(fi.system_seed(sd, k), A.n)).to(dev)
            b = torch.empty_like(xs)
            cg.cg_spmv(h, xs, b)
            bs.append(b)
        pool[N] = {"n": A.n, "nnz": A.nnz, "rp": rp, "ci": ci, "va": va, "h": h, "b": bs}
    torch.cuda.synchronize()

    # FIFO server of plain FP64 CG: measured service time of every (edge, rhs)
    # pair, then the single-server queue over the same arrival times
    service = {}
    j_fifo0 = energy.read_j()
    for N, P in pool.items():
        x = torch.zeros(P["n"], dtype=torch.float64, device=dev)
        for k in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            r = cg.cg_solve(P["h"], P["b"][k], x, tol=TOL, maxit=10 * P["n"])
            e1.record(stream)
            e1.synchronize()
            assert r.status == cg.CG_OK
            service[(N, k)] = e0.elapsed_time(e1) / 1000.0
    j_fifo1 = energy.read_j()
    fin, lat64, busy = 0.0, [], 0.0
    for i in range(count):
        sv = service[(int(edges[i]), i % 4)]
        fin = max(fin, t_arr[i]) + sv
        busy += sv
        lat64.append(fin - t_arr[i])
    fifo = {"solves_per_s": count / fin, "p50_ms": 1000 * float(np.percentile(lat64, 50)),
            "p99_ms": 1000 * float(np.percentile(lat64, 99)), "capacity_solves_per_s": count / busy,
            "joules_per_solve_of_the_measured_pairs": ((j_fifo1 - j_fifo0) / len(service)
                                                       if j_fifo0 is not None and j_fifo1 is not None else None),
            "note": "single FIFO server of cg_solve (FP64, whole GPU per solve): measured service time per "
                    "(edge, rhs) pair applied to the same arrival times"}

    jac = precond == "jacobi"
    bt = cg.Batch(precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64, chunk_iters=chunk,
                  validate=False, budget_bytes=int(budget_gb * 2**30), max_systems=1024,
                  preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, autotune=autotune,
                  group_target_ms=group_target_ms)
    outs = [torch.zeros(pool[int(N)]["n"], dtype=torch.float64, device=dev) for N in edges]
    reqs = [cg.Request(pool[int(N)]["rp"], pool[int(N)]["ci"], pool[int(N)]["va"], pool[int(N)]["b"][i % 4],
                       outs[i], tol=TOL, maxit=10 * pool[int(N)]["n"], tag=i) for i, N in enumerate(edges)]
    warm = {}
    for i, N in enumerate(edges):
        warm.setdefault(int(N), i)
    bt.wait_all(bt.submit([reqs[i] for i in warm.values()]))
    st0 = bt.stats()
    depth = []
    stop = threading.Event()

    def sample():
        while not stop.is_set():
            s = bt.stats()
            depth.append((s["pending"], s["resident"]))
            time.sleep(0.01)

    th = threading.Thread(target=sample, daemon=True)
    tickets = []
    with ClockSampler(dev.index or 0) as clk:
        j0 = energy.read_j()
        th.start()
        t0 = time.perf_counter()
        for i in range(count):
            d = t0 + t_arr[i] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(bt.submit([reqs[i]])[0])
        res = bt.wait_all(tickets)
        t_end = time.perf_counter() - t0
        stop.set()
        th.join()
        j1 = energy.read_j()
    st1 = bt.stats()
    bad = [r for r in res if r.status != cg.CG_OK or r.relres > TOL]
    assert not bad, bad[:3]
    lat = [r.latency_ms for r in res]
    first = min(r.submit_ms for r in res)
    last = max(r.done_ms for r in res)
    value = count / ((last - first) / 1000.0)
    dev_s = (st1["round_ms_total"] - st0["round_ms_total"]) / 1000.0
    bytes_all = sum(solve_bytes(pool[int(edges[r.tag])]["n"], pool[int(edges[r.tag])]["nnz"], r.iters, mixed,
                                jacobi=jac) for r in res)
    achieved = bytes_all / dev_s / 1e9
    rec = {
        "value": value, "unit": "solves/s", "dtype": "f32+f64" if mixed else "f64",
        "workload": f"served stream: Poisson arrivals at {rate:g} req/s for {seconds:g} s, Q1 27-point FE systems "
                    f"with grid edge lognormal in [16, 96], {'mixed precision' if mixed else 'FP64'}, "
                    f"{'Jacobi-preconditioned ' if jac else ''}CG to 1e-10, {budget_gb:g} GB device budget, "
                    f"{chunk} steps per system per round",
        "requests": count, "distinct_edges": len(pool), "rhs_per_edge": 4,
        "mean_nnz": float(np.mean([pool[int(N)]["nnz"] for N in edges])),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(np.max(lat))},
        "offered_solves_per_s": rate,
        "queue": {"max_pending": max(d[0] for d in depth) if depth else None,
                  "max_resident": max(d[1] for d in depth) if depth else None,
                  "bytes_peak": st1["bytes_peak"], "rounds": st1["rounds"] - st0["rounds"]},
        "fp64_fifo": fifo,
        "speedup_vs_fp64_fifo": value / fifo["solves_per_s"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None,
                     "kernel": f"cg_batch_kernel<{'true' if mixed else 'false'}, {'true' if jac else 'false'}>",
                     "device_busy_frac": dev_s / t_end},
        "energy": {"joules_per_solve": (j1 - j0) / count if j0 is not None and j1 is not None else None,
                   "source": "NVML board energy over the whole stream (idle gaps between arrivals included)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "request submission to solution written, through cg_batch_submit/wait"},
        "gpu_launches": int(st1["rounds"] - st0["rounds"] + (count if mixed else 0)),
        "clocks": clk.summary(),
    }
    bt.close()
    for P in pool.values():
        P["h"].close()
    return rec


def run_batch(args):
    """Many uneven systems per step in one persistent launch (batched API)."""
    import torch
    import paper_2112_10823_gb300 as cg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    systems = batch_systems(args.seed, args.batch_count, dev)
    hbm_peak, _ = peaks()
    rec = batch_record(cg, systems, dev, stream, Energy(0), hbm_peak, args.precision, args.precond, args.steps,
                       args.warmup, args.budget_gb, not args.no_autotune, args.group_target_ms, e2e=True,
                       traffic_key=(f"batch{args.batch_count}_seed{args.seed}_{args.precision}"
                                    if args.precond == "none" else None))
    line = {"metric": METRIC, "value": rec["value"], "unit": "solves/s", "n_gpus": 1, "steps": rec["steps"],
            "warmup": args.warmup, "ms_per_step": rec["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
            "config": {"workload": rec["workload"], "systems": rec["systems"], "sum_n": rec["sum_n"],
                       "sum_nnz": rec["sum_nnz"],
                       "l2": "flushed before every step (256 MiB write); the batch's matrices exceed L2"},
            "cpu_baseline": None}
    line.update({k: v for k, v in rec.items() if k not in ("value", "unit", "dtype", "workload", "steps")})
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Continuous batching of a Poisson request stream (served API)."""
    import torch
    import paper_2112_10823_gb300 as cg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    hbm_peak, _ = peaks()
    rec = serve_record(cg, args.seed, args.serve_rate, args.serve_seconds, dev, stream, Energy(0), hbm_peak,
                       args.precision, args.precond, args.budget_gb, args.chunk, not args.no_autotune,
                       args.group_target_ms)
    line = {"metric": METRIC, "value": rec["value"], "unit": "solves/s", "n_gpus": 1, "steps": rec["requests"],
            "warmup": rec["distinct_edges"], "ms_per_step": 1000.0 / rec["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic",
            "config": {"workload": rec["workload"], "requests": rec["requests"]}, "cpu_baseline": None}
    line.update({k: v for k, v in rec.items() if k not in ("value", "unit", "dtype", "workload")})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks under torchrun and pass its status on
        sys.exit(launch_ranks(args.gpus, os.path.abspath(__file__), sys.argv[1:]))
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
