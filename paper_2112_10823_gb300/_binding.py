"""ctypes binding of ``libcg.so`` (the C ABI in ``include/cg.h``).

Argument marshalling only: every operation runs in the library's CUDA
kernels.  Tensors are torch tensors (CUDA for device arguments; CPU tensors
or numpy arrays where the C ABI accepts host memory).  If the library has not
been built this module raises at import: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcg.so")

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_ENOTCONV, CG_EBREAKDOWN, CG_ETIMEOUT, CG_EBUSY = range(8)
STATUS_NAMES = {0: "CG_OK", 1: "CG_EINVAL", 2: "CG_ENOMEM", 3: "CG_ECUDA", 4: "CG_ENOTCONV",
                5: "CG_EBREAKDOWN", 6: "CG_ETIMEOUT", 7: "CG_EBUSY"}
CG_PREC_FP64, CG_PREC_MIXED = 0, 1
CG_PRECOND_NONE, CG_PRECOND_JACOBI = 0, 1
CG_SOLVE_KERNEL_LARGE_SHARE, CG_SOLVE_KERNEL_SMALL_SHARE, CG_SOLVE_KERNEL_CLUSTER = 0, 1, 2


class CGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class cg_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("index_base", ctypes.c_int32), ("on_device", ctypes.c_int32)]


class cg_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("device", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("replace_every", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("wait_limit_ms", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
                ("ctas", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class cg_batch_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32), ("budget_bytes", ctypes.c_int64),
                ("max_systems", ctypes.c_int32), ("chunk_iters", ctypes.c_int32),
                ("replace_every", ctypes.c_int32), ("wait_limit_ms", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("group_override", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("preconditioner", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("group_target_ms", ctypes.c_int32), ("step_shape", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class cg_request(ctypes.Structure):
    _fields_ = [("csr", cg_csr), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("tol", ctypes.c_double), ("maxit", ctypes.c_int64),
                ("tag", ctypes.c_uint64)]


class cg_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("done", ctypes.c_int32),
                ("status", ctypes.c_int32), ("iters", ctypes.c_int64), ("relres", ctypes.c_double),
                ("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("group", ctypes.c_int32), ("rounds", ctypes.c_int32)]


class cg_batch_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("pending", ctypes.c_int64), ("resident", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("bytes_peak", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("graph", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("round_ms_total", ctypes.c_double),
                ("last_round_ms", ctypes.c_double), ("cta_bytes_per_s", ctypes.c_double),
                ("group_cta_bytes_per_s", ctypes.c_double), ("step_overhead_s", ctypes.c_double),
                ("group_step_overhead_s", ctypes.c_double), ("autotuned", ctypes.c_int32),
                ("shape_tuned", ctypes.c_int32), ("step_kind", ctypes.c_int32 * 6), ("pad", ctypes.c_int32),
                ("rounds_stream_rows", ctypes.c_int64)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcg.so is not built ({LIB_PATH}); run paper_2112_10823_gb300.build.build() "
                          "(nvcc for sm_103a) first: there is no non-CUDA fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    lib.cg_opts_default.restype = None
    lib.cg_opts_default.argtypes = [P(cg_opts)]
    lib.cg_create.restype = ctypes.c_int
    lib.cg_create.argtypes = [P(vp), P(cg_csr), i64, i64, P(cg_opts)]
    lib.cg_destroy.restype = ctypes.c_int
    lib.cg_destroy.argtypes = [vp]
    lib.cg_last_error.restype = ctypes.c_char_p
    lib.cg_last_error.argtypes = [vp]
    lib.cg_info.restype = ctypes.c_int
    lib.cg_info.argtypes = [vp, P(i64), P(i64), P(i32)]
    lib.cg_partition_info.restype = ctypes.c_int
    lib.cg_partition_info.argtypes = [vp, P(i32), P(i32)]
    lib.cg_spmv.restype = ctypes.c_int
    lib.cg_spmv.argtypes = [vp, vp, vp]
    lib.cg_dot.restype = ctypes.c_int
    lib.cg_dot.argtypes = [i64, vp, vp, vp, vp]
    lib.cg_dot_host.restype = ctypes.c_int
    lib.cg_dot_host.argtypes = [i64, vp, vp, P(ctypes.c_double), vp]
    lib.cg_axpy.restype = ctypes.c_int
    lib.cg_axpy.argtypes = [i64, dbl, vp, vp, vp]
    lib.cg_ewmul.restype = ctypes.c_int
    lib.cg_ewmul.argtypes = [i64, vp, vp, vp, vp]
    lib.cg_blas_release.restype = ctypes.c_int
    lib.cg_blas_release.argtypes = []
    lib.cg_probe_fp64_peak.restype = ctypes.c_int
    lib.cg_probe_fp64_peak.argtypes = [i32, P(dbl)]
    lib.cg_probe_group_sync.restype = ctypes.c_int
    lib.cg_probe_group_sync.argtypes = [i32, i32, P(dbl), P(dbl)]
    lib.cg_solve.restype = ctypes.c_int
    lib.cg_solve.argtypes = [vp, vp, vp, dbl, i64, P(i64), P(dbl)]
    lib.cg_dot_noalloc.restype = ctypes.c_int
    lib.cg_dot_noalloc.argtypes = [i64, vp, vp, vp, vp]
    lib.cg_selftest_wait_timeout.restype = ctypes.c_int
    lib.cg_selftest_wait_timeout.argtypes = [i32, P(i32)]
    lib.cg_batch_opts_default.restype = None
    lib.cg_batch_opts_default.argtypes = [P(cg_batch_opts)]
    lib.cg_batch_create.restype = ctypes.c_int
    lib.cg_batch_create.argtypes = [P(vp), P(cg_batch_opts)]
    lib.cg_batch_destroy.restype = ctypes.c_int
    lib.cg_batch_destroy.argtypes = [vp]
    lib.cg_batch_submit.restype = ctypes.c_int
    lib.cg_batch_submit.argtypes = [vp, P(cg_request), i32, P(ctypes.c_uint64)]
    lib.cg_batch_poll.restype = ctypes.c_int
    lib.cg_batch_poll.argtypes = [vp, ctypes.c_uint64, P(cg_result)]
    lib.cg_batch_wait.restype = ctypes.c_int
    lib.cg_batch_wait.argtypes = [vp, ctypes.c_uint64, i32, P(cg_result)]
    lib.cg_batch_get_stats.restype = ctypes.c_int
    lib.cg_batch_get_stats.argtypes = [vp, P(cg_batch_stats)]
    lib.cg_batch_group_for.restype = ctypes.c_int
    lib.cg_batch_group_for.argtypes = [vp, vp, i64, P(i32)]
    lib.cg_batch_last_error.restype = ctypes.c_char_p
    lib.cg_batch_last_error.argtypes = [vp]
    return lib


lib = _load()


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (None -> 0)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    if hasattr(a, "ctypes"):
        return int(a.ctypes.data)
    if isinstance(a, int):
        return a
    raise TypeError(f"expected a tensor, an array or an address, got {type(a)}")


def _is_cuda(a) -> bool:
    return bool(getattr(a, "is_cuda", False))


def _check(status: int, handle=None) -> int:
    if status != CG_OK:
        raise CGError(status, lib.cg_last_error(handle).decode(errors="replace"))
    return status


def _check_f64(name, t, n=None, cuda=True):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if cuda and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")


@dataclass
class SolveResult:
    status: int
    iters: int
    relres: float

    @property
    def ok(self) -> bool:
        return self.status == CG_OK


class Handle:
    """A matrix resident on the GPU (wraps ``cg_handle``)."""

    def __init__(self, ptr: int, n: int, nnz: int, stream: int):
        self._h = ctypes.c_void_p(ptr)
        self.n, self.nnz, self.stream = n, nnz, stream

    @property
    def value(self):
        return self._h.value

    @property
    def nblocks(self) -> int:
        nb = ctypes.c_int32(0)
        _check(lib.cg_info(self._h, None, None, ctypes.byref(nb)), self._h)
        return nb.value

    def partition_info(self):
        """(most rows in one CTA's range, the CG_SOLVE_KERNEL_* that cg_solve runs)."""
        mr, kern = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(lib.cg_partition_info(self._h, ctypes.byref(mr), ctypes.byref(kern)), self._h)
        return mr.value, kern.value

    def close(self):
        if self._h is not None and self._h.value:
            lib.cg_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def cg_create(row_ptr, col_idx, val, n: int | None = None, nnz: int | None = None, index_base: int = 0,
              stream=None, device: int | None = None, precision: int = CG_PREC_FP64,
              replace_every: int = 50, validate: bool = True, wait_limit_ms: int = 2000,
              preconditioner: int = CG_PRECOND_NONE, ctas: int = 0) -> Handle:
    """cg_create: copy a CSR matrix (IA/JA/AA; host or CUDA arrays) to the GPU.

    ``stream``: a ``torch.cuda.Stream``, a raw ``cudaStream_t`` int, or None for
    torch's current stream on ``device``.
    """
    import numpy as np
    import torch
    n = int(row_ptr.shape[0]) - 1 if n is None else int(n)
    nnz = int(col_idx.shape[0]) if nnz is None else int(nnz)
    on_dev = _is_cuda(row_ptr)
    if on_dev != _is_cuda(col_idx) or on_dev != _is_cuda(val):
        raise ValueError("row_ptr, col_idx and val must all be host or all be CUDA")
    for name, a, dt in (("row_ptr", row_ptr, "int32"), ("col_idx", col_idx, "int32"), ("val", val, "float64")):
        if isinstance(a, torch.Tensor):
            if str(a.dtype) != f"torch.{dt}" or not a.is_contiguous():
                raise TypeError(f"{name} must be a contiguous {dt} tensor")
        elif isinstance(a, np.ndarray):
            if a.dtype != np.dtype(dt) or not a.flags["C_CONTIGUOUS"]:
                raise TypeError(f"{name} must be a C-contiguous {dt} array")
        else:
            raise TypeError(f"{name} must be a torch tensor or a numpy array")
    if device is None:
        device = row_ptr.device.index if on_dev else (torch.cuda.current_device() if torch.cuda.is_available() else -1)
    if stream is None and torch.cuda.is_available() and device is not None and device >= 0:
        stream = torch.cuda.current_stream(device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (int(stream) if stream else 0)
    csr = cg_csr(_ptr(row_ptr), _ptr(col_idx), _ptr(val), int(index_base), 1 if on_dev else 0)
    o = cg_opts()
    lib.cg_opts_default(ctypes.byref(o))
    o.stream = s
    o.device = -1 if device is None else int(device)
    o.precision = int(precision)
    o.replace_every = int(replace_every)
    o.validate = 1 if validate else 0
    o.wait_limit_ms = int(wait_limit_ms)
    o.preconditioner = int(preconditioner)
    o.ctas = int(ctas)
    out = ctypes.c_void_p(0)
    _check(lib.cg_create(ctypes.byref(out), ctypes.byref(csr), n, nnz, ctypes.byref(o)))
    return Handle(out.value, n, nnz, s)


def cg_destroy(h: Handle) -> None:
    h.close()


def cg_spmv(h: Handle, x, y) -> None:
    """y = A x (CUDA float64 tensors of n elements)."""
    _check_f64("x", x, h.n)
    _check_f64("y", y, h.n)
    _check(lib.cg_spmv(h._h, _ptr(x), _ptr(y)), h._h)


def _stream_of(t, stream) -> int:
    """Raw cudaStream_t: the given torch stream or int, else torch's current
    stream on the tensor's device."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(t.device)
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def cg_dot(x, y, out, n: int | None = None, stream=None) -> None:
    """out[0] = x . y (CUDA float64 tensors of one device; out has at least one
    element).  Runs on ``stream`` (default: torch's current stream)."""
    import torch
    n = x.numel() if n is None else int(n)
    _check_f64("x", x, n)
    _check_f64("y", y, n)
    _check_f64("out", out, 1)
    with torch.cuda.device(x.device):
        _check(lib.cg_dot(n, _ptr(x), _ptr(y), _ptr(out), _stream_of(x, stream)))


def cg_dot_host(x, y, n: int | None = None, stream=None) -> float:
    """x . y (CUDA float64 tensors) returned to the host; synchronous."""
    import torch
    n = x.numel() if n is None else int(n)
    _check_f64("x", x, n)
    _check_f64("y", y, n)
    r = ctypes.c_double(float("nan"))
    with torch.cuda.device(x.device):
        _check(lib.cg_dot_host(n, _ptr(x), _ptr(y), ctypes.byref(r), _stream_of(x, stream)))
    return r.value


def cg_dot_noalloc(x, y, out, n: int | None = None, stream=None) -> None:
    """out[0] = x . y without any allocation (fixed library scratch;
    n <= 33,554,432; concurrent calls race).  The call runs with the tensors'
    device current, which the library's lookup of its scratch relies on."""
    import torch
    n = x.numel() if n is None else int(n)
    _check_f64("x", x, n)
    _check_f64("y", y, n)
    _check_f64("out", out, 1)
    if x.device != out.device or y.device != out.device:
        raise ValueError("x, y and out must be on one device")
    with torch.cuda.device(out.device):
        _check(lib.cg_dot_noalloc(n, _ptr(x), _ptr(y), _ptr(out), _stream_of(out, stream)))


def cg_axpy(a: float, x, y, n: int | None = None, stream=None) -> None:
    """y <- a x + y."""
    import torch
    n = x.numel() if n is None else int(n)
    _check_f64("x", x, n)
    _check_f64("y", y, n)
    with torch.cuda.device(x.device):
        _check(lib.cg_axpy(n, float(a), _ptr(x), _ptr(y), _stream_of(x, stream)))


def cg_ewmul(x, y, z, n: int | None = None, stream=None) -> None:
    """z = x * y element-wise."""
    import torch
    n = x.numel() if n is None else int(n)
    for nm, t in (("x", x), ("y", y), ("z", z)):
        _check_f64(nm, t, n)
    with torch.cuda.device(x.device):
        _check(lib.cg_ewmul(n, _ptr(x), _ptr(y), _ptr(z), _stream_of(x, stream)))


def cg_blas_release() -> None:
    """Free the dot product's per-stream scratch (no dot call may be in flight)."""
    _check(lib.cg_blas_release())


def cg_probe_fp64_peak(device: int = -1) -> float:
    """Measured FP64 FMA throughput of the device, GFLOP/s."""
    g = ctypes.c_double(0.0)
    _check(lib.cg_probe_fp64_peak(int(device), ctypes.byref(g)))
    return g.value


def cg_probe_group_sync(device: int = -1, iters: int = 20000) -> tuple[float, float]:
    """Measured cost of the solves' group barrier and group sum on the whole
    grid: (microseconds per barrier, microseconds per sum)."""
    bar, summ = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.cg_probe_group_sync(int(device), int(iters), ctypes.byref(bar), ctypes.byref(summ)))
    return bar.value, summ.value


def cg_solve(h: Handle, b, x, tol: float = 1e-10, maxit: int | None = None, raise_on_error: bool = False
             ) -> SolveResult:
    """Solve A x = b; b and x are CUDA tensors, CPU tensors or numpy arrays
    (float64, n elements; x holds the initial guess and receives the solution)."""
    maxit = 10 * h.n if maxit is None else int(maxit)
    for nm, t in (("b", b), ("x", x)):
        if hasattr(t, "dtype") and str(t.dtype) not in ("torch.float64", "float64"):
            raise TypeError(f"{nm} must be float64")
        if (t.numel() if hasattr(t, "numel") else t.size) < h.n:
            raise ValueError(f"{nm} is shorter than n")
    it = ctypes.c_int64(0)
    rr = ctypes.c_double(0.0)
    st = lib.cg_solve(h._h, _ptr(b), _ptr(x), float(tol), maxit, ctypes.byref(it), ctypes.byref(rr))
    if st not in (CG_OK, CG_ENOTCONV, CG_EBREAKDOWN) or (raise_on_error and st != CG_OK):
        _check(st, h._h)
    return SolveResult(st, it.value, rr.value)


def cg_selftest_wait_timeout(limit_ms: int = 200) -> int:
    """Run the bounded-wait self-test; returns the status the kernel reported."""
    ks = ctypes.c_int32(-1)
    _check(lib.cg_selftest_wait_timeout(int(limit_ms), ctypes.byref(ks)))
    return ks.value


def last_error(h: Handle | None = None) -> str:
    return lib.cg_last_error(h._h if h is not None else None).decode(errors="replace")


# ----------------------------------------------------------- batched solves

@dataclass
class Request:
    """One system A x = b (x0 = 0) for a Batch.  Arrays are host (numpy / CPU
    torch) or CUDA tensors; the Batch keeps references to them until the
    request's result is done (the library reads b and the matrix at admission
    and writes x at the end)."""
    row_ptr: object
    col_idx: object
    val: object
    b: object
    x: object
    tol: float = 1e-10
    maxit: int | None = None
    index_base: int = 0
    tag: int = 0

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0]) - 1

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])


@dataclass
class BatchResult:
    ticket: int
    tag: int
    done: bool
    status: int
    iters: int
    relres: float
    submit_ms: float
    admit_ms: float
    done_ms: float
    group: int
    rounds: int

    @property
    def latency_ms(self) -> float:
        return self.done_ms - self.submit_ms


def _result(r: cg_result) -> BatchResult:
    return BatchResult(int(r.ticket), int(r.tag), bool(r.done), int(r.status), int(r.iters), float(r.relres),
                       float(r.submit_ms), float(r.admit_ms), float(r.done_ms), int(r.group), int(r.rounds))


class Batch:
    """Many independent systems on one GPU (wraps ``cg_batch``): requests are
    queued by submit(), admitted by the library's worker as the memory budget
    allows, and advanced together by one persistent kernel launch per round."""

    def __init__(self, precision: int = CG_PREC_FP64, budget_bytes: int = 0, max_systems: int = 1024,
                 chunk_iters: int = 0, replace_every: int = 50, wait_limit_ms: int = 2000,
                 max_pending: int = 65536, use_graph: bool = True, group_override: int = 0,
                 validate: bool = True, device: int = -1, preconditioner: int = CG_PRECOND_NONE,
                 autotune: bool = False, group_target_ms: int = 50, step_shape: int = 0):
        o = cg_batch_opts()
        lib.cg_batch_opts_default(ctypes.byref(o))
        o.device, o.precision, o.budget_bytes = int(device), int(precision), int(budget_bytes)
        o.max_systems, o.chunk_iters, o.replace_every = int(max_systems), int(chunk_iters), int(replace_every)
        o.wait_limit_ms, o.max_pending, o.use_graph = int(wait_limit_ms), int(max_pending), 1 if use_graph else 0
        o.group_override, o.validate = int(group_override), 1 if validate else 0
        o.preconditioner = int(preconditioner)
        o.autotune = 1 if autotune else 0
        o.group_target_ms = int(group_target_ms)
        o.step_shape = int(step_shape)
        out = ctypes.c_void_p(0)
        st = lib.cg_batch_create(ctypes.byref(out), ctypes.byref(o))
        if st != CG_OK:
            raise CGError(st, lib.cg_batch_last_error(None).decode(errors="replace"))
        self._b = out
        self._keep: dict[int, Request] = {}

    def _check(self, st: int) -> None:
        if st != CG_OK:
            raise CGError(st, lib.cg_batch_last_error(self._b).decode(errors="replace"))

    def submit(self, reqs: list[Request]) -> list[int]:
        """Queue the requests; returns their tickets.  CUDA arrays must hold
        their values when the library copies them, so torch's current stream
        is synchronised first if any request names a CUDA array."""
        if any(_is_cuda(a) for r in reqs for a in (r.row_ptr, r.col_idx, r.val, r.b, r.x)):
            import torch
            torch.cuda.current_stream().synchronize()
        arr = (cg_request * len(reqs))()
        for i, r in enumerate(reqs):
            on_dev = _is_cuda(r.row_ptr)
            if on_dev != _is_cuda(r.col_idx) or on_dev != _is_cuda(r.val):
                raise ValueError("row_ptr, col_idx and val must all be host or all be CUDA")
            arr[i].csr = cg_csr(_ptr(r.row_ptr), _ptr(r.col_idx), _ptr(r.val), int(r.index_base), 1 if on_dev else 0)
            arr[i].n, arr[i].nnz = r.n, r.nnz
            arr[i].b, arr[i].x = _ptr(r.b), _ptr(r.x)
            arr[i].tol = float(r.tol)
            arr[i].maxit = 10 * r.n if r.maxit is None else int(r.maxit)
            arr[i].tag = int(r.tag)
        tickets = (ctypes.c_uint64 * max(1, len(reqs)))()
        self._check(lib.cg_batch_submit(self._b, arr, len(reqs), tickets))
        out = [int(tickets[i]) for i in range(len(reqs))]
        for t, r in zip(out, reqs):
            self._keep[t] = r
        return out

    def poll(self, ticket: int) -> BatchResult:
        return self.wait(ticket, 0)

    def wait(self, ticket: int, timeout_ms: int = -1) -> BatchResult:
        r = cg_result()
        self._check(lib.cg_batch_wait(self._b, int(ticket), int(timeout_ms), ctypes.byref(r)))
        res = _result(r)
        if res.done:
            self._keep.pop(ticket, None)
        return res

    def wait_all(self, tickets: list[int], timeout_ms: int = -1) -> list[BatchResult]:
        return [self.wait(t, timeout_ms) for t in tickets]

    def stats(self) -> dict:
        s = cg_batch_stats()
        self._check(lib.cg_batch_get_stats(self._b, ctypes.byref(s)))
        out = {f: getattr(s, f) for f, _ in cg_batch_stats._fields_}
        out["step_kind"] = list(s.step_kind)
        out.pop("pad")
        return out

    def group_for(self, row_ptr) -> int:
        import numpy as np
        rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int32))
        g = ctypes.c_int32(0)
        self._check(lib.cg_batch_group_for(self._b, _ptr(rp), int(rp.shape[0]) - 1, ctypes.byref(g)))
        return g.value

    def close(self) -> None:
        if getattr(self, "_b", None) is not None and self._b.value:
            lib.cg_batch_destroy(self._b)
            self._b = ctypes.c_void_p(0)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False
