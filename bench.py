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
# Steps of an FP64 solve per grid edge on these systems (396 at 64^3), used
# only to size the oracle's sample on systems too large to solve on the host.
ITERS_PER_EDGE = 6.2
SIGMA = 1.0
TOL = 1e-10
L2_FLUSH_BYTES = 256 << 20  # > the 126.5 MiB L2
ENERGY_MIN_S = 1.0  # board energy and latency percentiles over at least this long
# FP64 FMA peak of one GB300 (152 SMs x ~2 DFMA/clk x 2 flop at 2.07 GHz);
# measured 600.5 G DFMA/s with an independent-chain probe.
FP64_PEAK_GFLOPS = 1201.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-solves", type=int, default=200)
    ap.add_argument("--grid", type=int, default=GRID_N,
                    help="grid edge of the Q1 system (64 is the benchmark workload; 160 the large system)")
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
    ap.add_argument("--cpu-budget", type=float, default=10.0,
                    help="seconds of oracle work for cpu_baseline (and per reference-arm step on large systems)")
    return ap.parse_args(argv)


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


def workload_name(grid: int, precision: str, precond: str = "none", matrix: str = "q1") -> str:
    prec = "FP64 CSR" if precision == "fp64" else "FP32-value product with FP64 residual replacement every 50 steps"
    method = "CG" if precond == "none" else "Jacobi-preconditioned CG"
    if matrix == "lap7":
        return f"3-D 7-point Laplacian, {grid}^3 grid, Dirichlet, {prec}, x* ~ U(-1,1), {method} from x0 = 0 to 1e-10"
    return f"Q1 27-point FE, {grid}^3 grid, lognormal rho (sigma=1), {prec}, {method} to 1e-10"


def oracle_solver(precision: str, precond: str = "none"):
    import oracle
    if precond == "jacobi":
        return lambda A, b, maxit: oracle.pcg_jacobi(A, b, tol=TOL, maxit=maxit)
    if precision == "mixed":
        return lambda A, b, maxit: oracle.cg_mixed(A, b, tol=TOL, maxit=maxit)
    return lambda A, b, maxit: oracle.cg(A, b, tol=TOL, maxit=maxit)


def oracle_rate(A, b, precision: str, budget_s: float, iters_full: int, precond: str = "none"):
    """The oracle's solves/s on one host core: whole solves when one takes
    less than half the budget, else runs of 20 steps (each with its setup
    product) whose time per step is scaled to an `iters_full`-step solve.
    Returns (solves/s, description of the sample)."""
    solve = oracle_solver(precision, precond)
    m = 20
    t0 = time.perf_counter()
    solve(A, b, m)
    per_step = (time.perf_counter() - t0) / (m + 1)
    if per_step * (iters_full + 1) <= budget_s / 2:
        n_done, t_tot = 0, 0.0
        while n_done == 0 or t_tot < budget_s:
            t0 = time.perf_counter()
            r = solve(A, b, 10 * A.n)
            t_tot += time.perf_counter() - t0
            n_done += 1
        return n_done / t_tot, (f"{n_done} complete oracle solves ({r.iters} iterations each), "
                                f"single thread, {t_tot:.1f} s")
    runs, t_tot = 0, 0.0
    while runs == 0 or t_tot < budget_s:
        t0 = time.perf_counter()
        solve(A, b, m)
        t_tot += time.perf_counter() - t0
        runs += 1
    per_step = t_tot / (runs * (m + 1))
    return 1.0 / (per_step * (iters_full + 1)), (
        f"{runs} oracle runs of {m} steps each plus the setup product (single thread, {t_tot:.1f} s), "
        f"time per step scaled to a {iters_full}-step solve")


def run_reference(args):
    """The oracle (plain sequential C, the paper's method as stated) on the same
    workload, on the host cores."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    import oracle
    A, xs = make_problem(args.seed, args.grid, args.matrix)
    b = oracle.spmv(A, xs)
    times, iters, sample = [], 0, ""
    # a full solve per step where it takes seconds; a bounded sample otherwise
    iters_hint = None if args.grid <= GRID_N else int(round(ITERS_PER_EDGE * args.grid))
    for s in range(args.warmup + args.steps):
        if iters_hint is None:
            t0 = time.perf_counter()
            r = oracle_solver(args.precision, args.precond)(A, b, 10 * A.n)
            dt = time.perf_counter() - t0
            iters = r.iters
            sample = f"{args.steps} full oracle solves of the workload (each step one solve, {iters} iterations)"
        else:
            iters = iters_hint
            v, sample = oracle_rate(A, b, args.precision, args.cpu_budget / 4, iters_hint, args.precond)
            dt = 1.0 / v
            sample = "each step: " + sample
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": workload_name(args.grid, args.precision, args.precond, args.matrix),
                   "n": A.n, "nnz": A.nnz, "iters": iters, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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
    A, xs = make_problem(seed, args.grid, args.matrix)
    n, nnz = A.n, A.nnz
    stream = torch.cuda.current_stream(dev)
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    va = torch.from_numpy(A.val).to(dev)
    mixed = args.precision == "mixed"
    jac = args.precond == "jacobi"
    h = cg.cg_create(rp, ci, va, stream=stream, precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64,
                     preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, ctas=args.ctas)
    h64 = cg.cg_create(rp, ci, va, stream=stream) if mixed else None   # FP64 solve for the accuracy record
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

    # ---- latency percentiles and board energy over back-to-back solves, and
    # the idle board power (nothing running) over half a second just before
    energy = Energy(local)
    torch.cuda.synchronize()
    idle_watts = None
    i0, ti0 = energy.read_j(), time.perf_counter()
    time.sleep(0.5)
    i1, ti = energy.read_j(), time.perf_counter() - ti0
    if i0 is not None and i1 is not None:
        idle_watts = (i1 - i0) / ti
    lat = []
    e0 = energy.read_j()
    tl0 = time.perf_counter()
    # at least latency_solves solves and at least ENERGY_MIN_S seconds of them
    # (the board energy counter needs a second or so to resolve a small solve)
    while len(lat) < args.latency_solves or time.perf_counter() - tl0 < ENERGY_MIN_S:
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x.zero_()
        s_ev.record(stream)
        cg.cg_solve(h, b, x, tol=TOL, maxit=10 * n)
        e_ev.record(stream)
        e_ev.synchronize()
        lat.append(s_ev.elapsed_time(e_ev))
    tl = time.perf_counter() - tl0
    e1 = energy.read_j()
    joules = (e1 - e0) / len(lat) if (e0 is not None and e1 is not None) else None
    watts = (e1 - e0) / tl if (e0 is not None and e1 is not None) else None

    # ---- BLAS-1 kernels alone (the vector operations of Sec. 5.2): the paper's
    # largest vector length and one four times the L2 (L2 flushed before each
    # call); bytes: dot 16 per element, axpy and element-wise product 24
    blas1 = {}
    for nv in (5_000_000, 64_000_000):
        xv = torch.rand(nv, dtype=torch.float64, device=dev)
        yv = torch.rand(nv, dtype=torch.float64, device=dev)
        zv = torch.empty_like(xv)
        outv = torch.zeros(1, dtype=torch.float64, device=dev)
        ops = {"dot": (lambda: cg.cg_dot(h, xv, yv, outv), 16), "axpy": (lambda: cg.cg_axpy(h, 0.5, xv, yv), 24),
               "ewmul": (lambda: cg.cg_ewmul(h, xv, yv, zv), 24)}
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
            blas1[f"{name}_{nv}"] = {"us": 1000 * ms, "gbs": bpe * nv / (ms * 1e-3) / 1e9}
        del xv, yv, zv

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

    # ---- accuracy of the timed solve: against x* and (mixed) the FP64 solve
    x_fin = x.clone()
    accuracy = {"relres_true": res.relres, "err_vs_xstar": float(torch.linalg.vector_norm(x_fin - xs_d)
                                                                  / torch.linalg.vector_norm(xs_d))}
    if mixed:
        x64 = torch.zeros_like(b)
        r64 = cg.cg_solve(h64, b, x64, tol=TOL, maxit=10 * n)
        accuracy.update({"fp64_iters": r64.iters, "fp64_relres_true": r64.relres,
                         "rel_diff_vs_fp64_solve": float(torch.linalg.vector_norm(x_fin - x64)
                                                         / torch.linalg.vector_norm(x64))})
        h64.close()

    # ---- roofline of the solve kernel (one launch per solve)
    launch_s = dev_time / args.steps
    bytes_launch = solve_bytes(n, nnz, iters, mixed, jacobi=jac)
    flops_launch = solve_flops(n, nnz, iters, mixed, jacobi=jac)
    achieved_gbs = bytes_launch / launch_s / 1e9
    achieved_gflops = flops_launch / launch_s / 1e9
    kernel_kind = h.partition_info()[1]  # the solve kernel the library runs on this system
    if kernel_kind == cg.CG_SOLVE_KERNEL_CLUSTER:
        kname = "cg_cluster_kernel"
    else:
        small = kernel_kind == cg.CG_SOLVE_KERNEL_SMALL_SHARE
        kname = (f"cg_solve_kernel<{'true' if mixed else 'false'}, {'true' if jac else 'false'}, "
                 f"{'true' if small else 'false'}>")
    traffic = recorded_traffic(kname, f"{args.matrix}_{args.grid}")
    if l2_resident(n, nnz, mixed) or not mixed and achieved_gflops / FP64_PEAK_GFLOPS > achieved_gbs / hbm_peak:
        # the system stays in L2 during a solve (or the FP64 pipe is nearer its
        # peak than HBM is): the FP64 pipe bounds the kernel
        roof = {"bound": "alu", "achieved": achieved_gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved_gflops / FP64_PEAK_GFLOPS, "traffic": traffic,
                "peak_source": "measured (FP64 FMA probe)", "kernel": kname, "algorithmic_gbs": achieved_gbs,
                "algorithmic_gbs_frac_of_hbm": achieved_gbs / hbm_peak, "hbm_peak_source": peak_kind}
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic, "peak_source": peak_kind,
                "kernel": kname, "gflops": achieved_gflops, "gflops_frac_of_fp64": achieved_gflops / FP64_PEAK_GFLOPS}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    base = None
    if not args.no_cpu_baseline:
        import oracle
        b_host = b.cpu().numpy()
        v, sample = oracle_rate(A, b_host, args.precision, args.cpu_budget, iters, args.precond)
        base = {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.grid, args.precision, args.precond, args.matrix),
                   "n": n, "nnz": nnz, "iters": iters, "tol": TOL, "x0": "zero",
                   "l2": "flushed before every timed solve (256 MiB write)", "parallelism": f"replicas x{world}",
                   "ctas": h.nblocks},
        "roofline": roof,
        "accuracy": accuracy,
        "spmv": {"gbs": spmv_gbs, "frac": spmv_gbs / hbm_peak, "ms": spmv_ms, "bytes": spmv_bytes(n, nnz),
                 "l2": "flushed before every call", "precision": "fp64"},
        "blas1": {k: dict(v, frac=v["gbs"] / hbm_peak) for k, v in blas1.items()},
        "energy": {"joules_per_solve": joules, "avg_watts": watts, "idle_watts": idle_watts,
                   "joules_per_solve_above_idle": (joules - idle_watts * tl / len(lat)
                                                   if joules is not None and idle_watts is not None else None),
                   "source": "NVML board energy",
                   "solves": len(lat), "seconds": tl},
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


# ----------------------------------------------------- batched and served

def _upload(A, dev):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.row_ptr, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(A.col_idx, dtype=np.int32)).to(dev),
            torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).to(dev))


def _batch_systems(seed: int, count: int, dev):
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
        rp, ci, va = _upload(A, dev)
        h = cg.cg_create(rp, ci, va)
        xs = torch.from_numpy(fi.xstar(sd, A.n)).to(dev)
        b = torch.empty_like(xs)
        cg.cg_spmv(h, xs, b)
        out.append({"N": int(N), "n": A.n, "nnz": A.nnz, "rp": rp, "ci": ci, "va": va, "h": h, "b": b,
                    "x": torch.zeros_like(b), "xs": xs})
    torch.cuda.synchronize()
    return out


def _solve_sequential(systems, stream):
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


def run_batch(args):
    """Many uneven systems per step in one persistent launch (batched API)."""
    import torch
    import paper_2112_10823_gb300 as cg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    systems = _batch_systems(args.seed, args.batch_count, dev)
    count = len(systems)
    mixed = args.precision == "mixed"
    hbm_peak, peak_kind = peaks()
    energy = Energy(0)

    # plain FP64 CG on the same GPU, system after system
    _solve_sequential(systems, stream)
    x64 = [s["x"].clone() for s in systems]
    j0 = energy.read_j()
    t_seq, its64 = 0.0, None
    for _ in range(args.steps):
        dt, its64 = _solve_sequential(systems, stream)
        t_seq += dt
    j1 = energy.read_j()
    seq = {"solves_per_s": count * args.steps / t_seq, "ms_per_batch": 1000.0 * t_seq / args.steps,
           "joules_per_solve": (j1 - j0) / (count * args.steps) if j0 is not None and j1 is not None else None,
           "launches_per_batch": count}

    jac = args.precond == "jacobi"
    bt = cg.Batch(precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64, chunk_iters=0, validate=False,
                  budget_bytes=int(args.budget_gb * 2**30), max_systems=max(1024, count),
                  preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, autotune=not args.no_autotune,
                  group_target_ms=args.group_target_ms)
    model = {k: bt.stats()[k] for k in ("autotuned", "cta_bytes_per_s", "group_cta_bytes_per_s", "step_overhead_s",
                                        "group_step_overhead_s")}

    def step():
        reqs = [cg.Request(s["rp"], s["ci"], s["va"], s["b"], s["x"], tol=TOL, maxit=10 * s["n"], tag=i)
                for i, s in enumerate(systems)]
        res = bt.wait_all(bt.submit(reqs))
        bad = [r for r in res if r.status != cg.CG_OK or r.relres > TOL]
        assert not bad, bad[:3]
        return res

    for _ in range(args.warmup):
        res = step()
    st0 = bt.stats()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    with ClockSampler(0) as clk:
        j0 = energy.read_j()
        tw0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k)
            torch.cuda.synchronize()
            res = step()
        t_wall = time.perf_counter() - tw0
        j1 = energy.read_j()
    st1 = bt.stats()
    rounds = st1["rounds"] - st0["rounds"]

    # end to end through the public API from pinned host memory: every step
    # copies each system's CSR arrays and b to the device (admission) and its
    # solution back to the host
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
    for _ in range(args.steps):
        res_h = step_host()
        # where an end-to-end step goes: admission (host checks, partition,
        # copies) from the first submit to the last system resident, then the
        # round and the copies of x back
        sub0 = min(r.submit_ms for r in res_h)
        adm1 = max(r.admit_ms for r in res_h)
        spans.append((adm1 - sub0, max(r.done_ms for r in res_h) - adm1))
    t_e2e = time.perf_counter() - te0
    dev_s = (st1["round_ms_total"] - st0["round_ms_total"]) / 1000.0
    value = count * args.steps / dev_s
    iters = [r.iters for r in res]
    groups = [r.group for r in res]
    err = max(float(torch.linalg.vector_norm(s["x"] - x) / torch.linalg.vector_norm(x)) for s, x in zip(systems, x64))
    bytes_batch = sum(solve_bytes(s["n"], s["nnz"], it, mixed, jacobi=jac) for s, it in zip(systems, iters))
    flops_batch = sum(solve_flops(s["n"], s["nnz"], it, mixed, jacobi=jac) for s, it in zip(systems, iters))
    per_round = dev_s / rounds
    achieved = bytes_batch * args.steps / dev_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"batch of {count} Q1 27-point FE systems, grid edges uniform in [8, 48], "
                               f"lognormal rho (sigma=1), own b per system, "
                               f"{'mixed precision' if mixed else 'FP64'}, one persistent launch per batch "
                               f"(CUDA graph), {'Jacobi-preconditioned ' if jac else ''}CG to 1e-10",
                   "systems": count, "sum_n": int(sum(s["n"] for s in systems)),
                   "sum_nnz": int(sum(s["nnz"] for s in systems)), "iters_min": min(iters), "iters_max": max(iters),
                   "groups": {str(g): groups.count(g) for g in sorted(set(groups))},
                   "rounds_per_step": rounds / args.steps, "graph": bool(st1["graph"]), "group_model": model,
                   "l2": "flushed before every step (256 MiB write); the batch's matrices exceed L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_kind,
                     "kernel": f"cg_batch_kernel<{'true' if mixed else 'false'}, {'true' if jac else 'false'}>",
                     "gflops": flops_batch * args.steps / dev_s / 1e9, "round_ms": 1000.0 * per_round},
        "accuracy": {"max_relres_true": max(r.relres for r in res),
                     "max_rel_diff_vs_fp64_cg_solve": err},
        "fp64_sequential": seq,
        "speedup_vs_fp64_sequential": value / seq["solves_per_s"],
        "energy": {"joules_per_solve": (j1 - j0) / (count * args.steps) if j0 is not None and j1 is not None else None,
                   "source": "NVML board energy (whole steps, host admission included)"},
        "e2e": {"value": count * args.steps / t_e2e, "unit": "solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "note": "wall clock through cg_batch_submit/wait with every system's CSR arrays and b in pinned "
                        "host memory (admission copies them to the device) and x read back to the host",
                "admission_ms": float(np.mean([a for a, _ in spans])),
                "round_and_readback_ms": float(np.mean([r for _, r in spans])),
                "device_resident_inputs_solves_per_s": count * args.steps / t_wall},
        "gpu_launches": int(rounds + (count * args.steps if mixed else 0)),
        "clocks": clk.summary(),
        "gpu": {"name": torch.cuda.get_device_name(dev), "uuid": gpu_uuid(0)},
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    bt.close()


def run_serve(args):
    """Continuous batching of a Poisson request stream (served API), against
    a FIFO server of plain FP64 CG solves on the same GPU."""
    import torch
    import fe_inputs as fi
    import paper_2112_10823_gb300 as cg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    mixed = args.precision == "mixed"
    count = max(1, int(round(args.serve_rate * args.serve_seconds)))
    t_arr, edges = fi.arrivals(args.seed, count, args.serve_rate)
    # request i solves the pool system of its edge with right-hand side k = i % 4
    pool = {}
    for N in sorted(set(int(e) for e in edges)):
        sd = fi.system_seed(args.seed, 100000 + N)
        A = fi.q1(N, SIGMA, sd)
        rp, ci, va = _upload(A, dev)
        h = cg.cg_create(rp, ci, va)
        bs = []
        for k in range(4):
            xs = torch.from_numpy(fi.xstar(fi.system_seed(sd, k), A.n)).to(dev)
            b = torch.empty_like(xs)
            cg.cg_spmv(h, xs, b)
            bs.append(b)
        pool[N] = {"n": A.n, "nnz": A.nnz, "rp": rp, "ci": ci, "va": va, "h": h, "b": bs}
    torch.cuda.synchronize()
    energy = Energy(0)

    # FIFO server of plain FP64 CG: measured service time of every (edge, rhs)
    # pair, then the single-server queue over the same arrival times
    service = {}
    x = None
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
    fin, lat64, busy = 0.0, [], 0.0
    for i in range(count):
        sv = service[(int(edges[i]), i % 4)]
        fin = max(fin, t_arr[i]) + sv
        busy += sv
        lat64.append(fin - t_arr[i])
    fifo = {"solves_per_s": count / fin, "p50_ms": 1000 * float(np.percentile(lat64, 50)),
            "p99_ms": 1000 * float(np.percentile(lat64, 99)), "capacity_solves_per_s": count / busy,
            "note": "single FIFO server of cg_solve (FP64, whole GPU per solve): measured service time per "
                    "(edge, rhs) pair applied to the same arrival times"}

    jac = args.precond == "jacobi"
    bt = cg.Batch(precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64, chunk_iters=args.chunk,
                  validate=False, budget_bytes=int(args.budget_gb * 2**30), max_systems=1024,
                  preconditioner=cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE, autotune=not args.no_autotune,
                  group_target_ms=args.group_target_ms)
    outs = [torch.zeros(pool[int(N)]["n"], dtype=torch.float64, device=dev) for N in edges]
    reqs = [cg.Request(pool[int(N)]["rp"], pool[int(N)]["ci"], pool[int(N)]["va"], pool[int(N)]["b"][i % 4],
                       outs[i], tol=TOL, maxit=10 * pool[int(N)]["n"], tag=i) for i, N in enumerate(edges)]
    # warm-up: one request of each edge
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
    with ClockSampler(0) as clk:
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
    hbm_peak, peak_kind = peaks()
    achieved = bytes_all / dev_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": count, "warmup": len(warm),
        "ms_per_step": (last - first) / count, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"served stream: Poisson arrivals at {args.serve_rate:g} req/s for "
                               f"{args.serve_seconds:g} s, Q1 27-point FE systems with grid edge lognormal in "
                               f"[16, 96], {'mixed precision' if mixed else 'FP64'}, "
                               f"{'Jacobi-preconditioned ' if jac else ''}CG to 1e-10, "
                               f"{args.budget_gb:g} GB device budget, {args.chunk} steps per system per round",
                   "requests": count, "distinct_edges": len(pool), "rhs_per_edge": 4,
                   "mean_nnz": float(np.mean([pool[int(N)]["nnz"] for N in edges]))},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(np.max(lat))},
        "offered_solves_per_s": args.serve_rate,
        "queue": {"max_pending": max(d[0] for d in depth) if depth else None,
                  "max_resident": max(d[1] for d in depth) if depth else None,
                  "bytes_peak": st1["bytes_peak"], "rounds": st1["rounds"] - st0["rounds"]},
        "fp64_fifo": fifo,
        "speedup_vs_fp64_fifo": value / fifo["solves_per_s"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_kind,
                     "kernel": f"cg_batch_kernel<{'true' if mixed else 'false'}, {'true' if jac else 'false'}>",
                     "device_busy_frac": dev_s / t_end},
        "energy": {"joules_per_solve": (j1 - j0) / count if j0 is not None and j1 is not None else None,
                   "fp64_fifo_joules_per_solve": None, "source": "NVML board energy over the whole stream"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "request submission to solution written, through cg_batch_submit/wait"},
        "gpu_launches": int(st1["rounds"] - st0["rounds"] + (count if mixed else 0)),
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    bt.close()


def main():
    args = parse()
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
