"""ORACLE — test infrastructure only.

Plain sequential FP64 CPU statement of the CG hot path (``cg_oracle.c``),
built with the host C compiler and called through ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the product (``paper_2112_10823_gb300``) never does and
shares no code with it.

Functions follow the paper's definitions:
  spmv   CSR product y_i = sum_{k=IA(i)}^{IA(i+1)-1} AA(k) x(JA(k))  (Sec. 2.3)
  dot / axpy / ewmul  the vector operations benchmarked in Sec. 5.2
  cg     classical unpreconditioned CG (Sec. 5.3), Hestenes-Stiefel form
  cg_mixed   FP32-matrix product with FP64 scalars and residual replacement
  matrix_stats  the columns of the paper's Table 1 (Sec. 5.1)
  omp_cg / omp_cg_mixed / omp_spmv / omp_dot   the same CG (FP64 and mixed) and product spread over the host's
             cores with OpenMP (``cg_oracle_omp.c``): the timing variant behind
             the CPU baseline, pinned against the sequential functions
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libcg_oracle.so")
_OMP_SRC = os.path.join(_HERE, "cg_oracle_omp.c")
_OMP_LIB_PATH = os.path.join(_HERE, "_build", "libcg_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None
_omp_build_path = None  # set by using_omp

OK, NOTCONV, BREAKDOWN, NOMEM = 0, 4, 5, 2


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -ffp-contract=off: no fused multiply-adds)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    build_omp(force)
    return _LIB_PATH


def build_omp(force: bool = False) -> str | None:
    """Compile the OpenMP timing variant (gcc -fopenmp).  Returns None, with a
    warning, if the host compiler has no OpenMP: the sequential oracle still
    works and the CPU baseline then reports one core."""
    if not force and os.path.exists(_OMP_LIB_PATH) and os.path.getmtime(_OMP_LIB_PATH) >= os.path.getmtime(_OMP_SRC):
        return _OMP_LIB_PATH
    tmp = _OMP_LIB_PATH + f".{os.getpid()}.tmp"
    res = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                          "-std=c11", "-o", tmp, _OMP_SRC, "-lm"], capture_output=True, text=True)
    if res.returncode != 0:
        import warnings
        warnings.warn("OpenMP oracle not built (gcc -fopenmp failed): " + res.stderr[-500:])
        return None
    os.replace(tmp, _OMP_LIB_PATH)
    return _OMP_LIB_PATH


def _bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    i64, dbl, vp, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
    lib.oracle_spmv.restype = None
    lib.oracle_spmv.argtypes = [i64, vp, vp, vp, ci, vp, vp]
    lib.oracle_spmv_rows.restype = None
    lib.oracle_spmv_rows.argtypes = [i64, vp, vp, vp, vp, ci, vp, vp]
    lib.oracle_dot.restype = dbl
    lib.oracle_dot.argtypes = [i64, vp, vp]
    lib.oracle_axpy.restype = None
    lib.oracle_axpy.argtypes = [i64, dbl, vp, vp]
    lib.oracle_ewmul.restype = None
    lib.oracle_ewmul.argtypes = [i64, vp, vp, vp]
    lib.oracle_cg.restype = ci
    lib.oracle_cg.argtypes = [i64, vp, vp, vp, ci, vp, vp, dbl, i64, i64,
                              vp, vp, vp, vp, vp, vp, i64]
    lib.oracle_spmv_f32.restype = None
    lib.oracle_spmv_f32.argtypes = [i64, vp, vp, vp, ci, vp, vp]
    lib.oracle_cg_mixed.restype = ci
    lib.oracle_cg_mixed.argtypes = [i64, vp, vp, vp, vp, ci, vp, vp, dbl, i64, i64, i64, vp, vp, vp]
    lib.oracle_jacobi_dinv.restype = ci
    lib.oracle_jacobi_dinv.argtypes = [i64, vp, vp, vp, ci, vp]
    lib.oracle_pcg_jacobi.restype = ci
    lib.oracle_pcg_jacobi.argtypes = [i64, vp, vp, vp, ci, vp, vp, dbl, i64, i64, vp, vp, vp]
    lib.oracle_matrix_stats.restype = None
    lib.oracle_matrix_stats.argtypes = [i64, vp, vp, ci, vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _load_omp():
    """The OpenMP variant's library, or None if it cannot be built here."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            path = _omp_build_path or build_omp()
            if path is None:
                return None
            lib = ctypes.CDLL(path)
            i64, dbl, vp, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            lib.oracle_omp_threads.restype = ci
            lib.oracle_omp_threads.argtypes = []
            lib.oracle_omp_set_threads.restype = None
            lib.oracle_omp_set_threads.argtypes = [ci]
            lib.oracle_omp_spmv.restype = None
            lib.oracle_omp_spmv.argtypes = [i64, vp, vp, vp, ci, vp, vp]
            lib.oracle_omp_dot.restype = dbl
            lib.oracle_omp_dot.argtypes = [i64, vp, vp]
            lib.oracle_omp_cg.restype = ci
            lib.oracle_omp_cg.argtypes = [i64, vp, vp, vp, ci, vp, vp, dbl, i64, i64, vp, vp, vp]
            lib.oracle_omp_cg_mixed.restype = ci
            lib.oracle_omp_cg_mixed.argtypes = [i64, vp, vp, vp, vp, ci, vp, vp, dbl, i64, i64, i64, vp, vp, vp]
            _omp_lib = lib
    return _omp_lib


def omp_available() -> bool:
    return _load_omp() is not None


def omp_threads() -> int:
    """Threads the OpenMP variant uses (all host cores unless OMP_NUM_THREADS says otherwise)."""
    lib = _load_omp()
    return int(lib.oracle_omp_threads()) if lib is not None else 1


def omp_set_threads(t: int) -> None:
    """Threads of the OpenMP variant's following calls."""
    _need_omp().oracle_omp_set_threads(int(t))


class using_omp:
    """Context manager: route the OpenMP variant's calls through another
    compiled copy (the tests that plant mistakes in a copy of its source)."""

    def __init__(self, lib_path: str):
        self._path = lib_path

    def __enter__(self):
        global _omp_lib, _omp_build_path
        _load_omp()
        self._old = _omp_lib
        _omp_lib = None
        _omp_build_path = self._path
        _load_omp()
        return self

    def __exit__(self, *exc):
        global _omp_lib, _omp_build_path
        _omp_lib, _omp_build_path = self._old, None
        return False


class using:
    """Context manager: route every oracle call through another compiled copy
    (used by the tests that plant mistakes in a copy of the oracle source)."""

    def __init__(self, lib_path: str):
        self._new = _bind(ctypes.CDLL(lib_path))

    def __enter__(self):
        global _lib
        _load()
        self._old, _lib = _lib, self._new
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._old
        return False


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def spmv(A, x) -> np.ndarray:
    """y = A x for a CSR ``A`` (attributes row_ptr, col_idx, val, n, index_base)."""
    rp, ci, va, x = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(x)
    y = np.empty(A.n, dtype=np.float64)
    _load().oracle_spmv(A.n, _p(rp), _p(ci), _p(va), int(getattr(A, "index_base", 0)), _p(x), _p(y))
    return y


def spmv_rows(A, x, rows) -> np.ndarray:
    """(A x)[rows] computed row by row."""
    rp, ci, va, x = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(rows.shape[0], dtype=np.float64)
    _load().oracle_spmv_rows(rows.shape[0], _p(rows), _p(rp), _p(ci), _p(va),
                             int(getattr(A, "index_base", 0)), _p(x), _p(y))
    return y


def dot(x, y) -> float:
    x, y = _f64(x), _f64(y)
    return float(_load().oracle_dot(x.shape[0], _p(x), _p(y)))


def axpy(a: float, x, y) -> np.ndarray:
    """Returns a*x + y (y is not modified)."""
    x, out = _f64(x), np.array(y, dtype=np.float64, copy=True)
    _load().oracle_axpy(x.shape[0], float(a), _p(x), _p(out))
    return out


def ewmul(x, y) -> np.ndarray:
    x, y = _f64(x), _f64(y)
    z = np.empty_like(x)
    _load().oracle_ewmul(x.shape[0], _p(x), _p(y), _p(z))
    return z


@dataclass
class CGResult:
    x: np.ndarray
    status: int
    iters: int
    relres_rec: float
    relres_true: float
    alpha: np.ndarray | None = None
    beta: np.ndarray | None = None
    res: np.ndarray | None = None


def cg(A, b, tol: float = 1e-10, maxit: int | None = None, x0=None, force_iters: int = -1,
       history: bool = False) -> CGResult:
    """Classical CG; ``force_iters >= 0`` runs exactly that many steps."""
    n = A.n
    rp, ci, va, b = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    maxit = n if maxit is None else maxit
    it = ctypes.c_int64(0)
    rr, rt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    hl = (max(maxit, force_iters) + 2) if history else 0
    ah = np.zeros(max(hl, 1)); bh = np.zeros(max(hl, 1)); rh = np.zeros(max(hl, 1))
    st = _load().oracle_cg(n, _p(rp), _p(ci), _p(va), int(getattr(A, "index_base", 0)), _p(b), _p(x),
                           float(tol), int(maxit), int(force_iters), ctypes.byref(it), ctypes.byref(rr),
                           ctypes.byref(rt), _p(ah) if history else None, _p(bh) if history else None,
                           _p(rh) if history else None, hl)
    k = it.value
    res = CGResult(x, st, k, rr.value, rt.value)
    if history:
        res.alpha, res.beta, res.res = ah[:k].copy(), bh[:k].copy(), rh[:k + 1].copy()
    return res


def spmv_f32(A, val32, x32) -> np.ndarray:
    rp, ci = _i32(A.row_ptr), _i32(A.col_idx)
    v = np.ascontiguousarray(val32, dtype=np.float32)
    x = np.ascontiguousarray(x32, dtype=np.float32)
    y = np.empty(A.n, dtype=np.float32)
    _load().oracle_spmv_f32(A.n, _p(rp), _p(ci), _p(v), int(getattr(A, "index_base", 0)), _p(x), _p(y))
    return y


def cg_mixed(A, b, tol: float = 1e-10, maxit: int | None = None, replace_every: int = 50,
             force_iters: int = -1) -> CGResult:
    """Mixed-precision CG (FP32 values and product, FP64 sums, scalars, x and
    a true-residual replacement every ``replace_every`` steps); ``force_iters
    >= 0`` runs exactly that many steps."""
    n = A.n
    rp, ci, va, b = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(b)
    v32 = va.astype(np.float32)
    x = np.zeros(n)
    maxit = 10 * n if maxit is None else maxit
    it = ctypes.c_int64(0)
    rr, rt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = _load().oracle_cg_mixed(n, _p(rp), _p(ci), _p(va), _p(v32), int(getattr(A, "index_base", 0)),
                                 _p(b), _p(x), float(tol), int(maxit), int(replace_every), int(force_iters),
                                 ctypes.byref(it), ctypes.byref(rr), ctypes.byref(rt))
    return CGResult(x, st, it.value, rr.value, rt.value)


def jacobi_dinv(A):
    """1 / diag(A), or None if a diagonal entry is not positive."""
    rp, ci, va = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val)
    out = np.zeros(A.n)
    st = _load().oracle_jacobi_dinv(A.n, _p(rp), _p(ci), _p(va), int(getattr(A, "index_base", 0)), _p(out))
    return out if st == OK else None


def pcg_jacobi(A, b, tol: float = 1e-10, maxit: int | None = None, x0=None, force_iters: int = -1) -> CGResult:
    """Jacobi-preconditioned CG (M = diag(A)); ``force_iters >= 0`` runs exactly that many steps."""
    n = A.n
    rp, ci, va, b = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    maxit = n if maxit is None else maxit
    it = ctypes.c_int64(0)
    rr, rt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = _load().oracle_pcg_jacobi(n, _p(rp), _p(ci), _p(va), int(getattr(A, "index_base", 0)), _p(b), _p(x),
                                   float(tol), int(maxit), int(force_iters), ctypes.byref(it), ctypes.byref(rr),
                                   ctypes.byref(rt))
    return CGResult(x, st, it.value, rr.value, rt.value)


def matrix_stats(A) -> dict:
    rp, ci = _i32(A.row_ptr), _i32(A.col_idx)
    out = np.zeros(7)
    _load().oracle_matrix_stats(A.n, _p(rp), _p(ci), int(getattr(A, "index_base", 0)), _p(out))
    keys = ["h", "nz", "density", "bandwidth", "max_row", "nz_per_h", "nz_per_h_stddev"]
    return dict(zip(keys, out.tolist()))


# ------------------------------------------------ OpenMP timing variant

def _need_omp():
    lib = _load_omp()
    if lib is None:
        raise RuntimeError("the OpenMP oracle is not available (gcc -fopenmp failed)")
    return lib


def omp_spmv(A, x) -> np.ndarray:
    """y = A x, rows spread over the host's cores (each row as ``spmv``: the same bits)."""
    rp, ci, va, x = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(x)
    y = np.empty(A.n, dtype=np.float64)
    _need_omp().oracle_omp_spmv(A.n, _p(rp), _p(ci), _p(va), int(getattr(A, "index_base", 0)), _p(x), _p(y))
    return y


def omp_dot(x, y) -> float:
    x, y = _f64(x), _f64(y)
    return float(_need_omp().oracle_omp_dot(x.shape[0], _p(x), _p(y)))


def omp_cg(A, b, tol: float = 1e-10, maxit: int | None = None, x0=None, force_iters: int = -1) -> CGResult:
    """Classical CG on all host cores (the steps of ``cg``); ``force_iters >= 0``
    runs exactly that many steps."""
    n = A.n
    rp, ci, va, b = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    maxit = n if maxit is None else maxit
    it = ctypes.c_int64(0)
    rr, rt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = _need_omp().oracle_omp_cg(n, _p(rp), _p(ci), _p(va), int(getattr(A, "index_base", 0)), _p(b), _p(x),
                                   float(tol), int(maxit), int(force_iters), ctypes.byref(it), ctypes.byref(rr),
                                   ctypes.byref(rt))
    return CGResult(x, st, it.value, rr.value, rt.value)


def omp_cg_mixed(A, b, tol: float = 1e-10, maxit: int | None = None, replace_every: int = 50,
                 force_iters: int = -1) -> CGResult:
    """Mixed-precision CG on all host cores (the steps of ``cg_mixed``);
    ``force_iters >= 0`` runs exactly that many steps."""
    n = A.n
    rp, ci, va, b = _i32(A.row_ptr), _i32(A.col_idx), _f64(A.val), _f64(b)
    v32 = va.astype(np.float32)
    x = np.zeros(n)
    maxit = 10 * n if maxit is None else maxit
    it = ctypes.c_int64(0)
    rr, rt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = _need_omp().oracle_omp_cg_mixed(n, _p(rp), _p(ci), _p(va), _p(v32), int(getattr(A, "index_base", 0)),
                                         _p(b), _p(x), float(tol), int(maxit), int(replace_every), int(force_iters),
                                         ctypes.byref(it), ctypes.byref(rr), ctypes.byref(rt))
    return CGResult(x, st, it.value, rr.value, rt.value)
