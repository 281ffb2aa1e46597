"""Seeded synthetic inputs: finite-element CSR matrices and random vectors.

This module builds test problems for the CG solver and for its CPU oracle.
It contains no solver arithmetic: it only writes the CSR arrays of SPD
finite-element operators and seeded random vectors, which both sides read.

The paper solves Q1 finite-element discretisations of a Poisson-type gravity
equation with Dirichlet boundary conditions (Sec. 5.1, Table 1).  Its
matrices are not available, so seeded stand-ins with the same element type,
stencil and boundary structure are built here:

* ``laplace7(N)``: 7-point Laplacian on an N^3 grid, Dirichlet nodes
  eliminated (diag 6, off-diagonal -1).
* ``q1(N, sigma, seed)``: trilinear hexahedral stiffness of -div(rho grad u)
  with one lognormal density per element, rho_e = exp(sigma * Z_e).
* ``uniform`` / ``normal``: counter-based SplitMix64 streams.
* ``random_csr`` / ``random_spd``: small irregular matrices for edge cases.

The C part (``fe_gen.c``) is compiled on first use with the host C compiler.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_gen.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libfe_gen.so")
_lock = threading.Lock()
_lib = None

# Stream identifiers of the counter-based generator (any fixed distinct values).
STREAM_XSTAR = 1
STREAM_RHO = 2
STREAM_RANDOM_CSR = 3
STREAM_BATCH = 4
STREAM_ARRIVALS = 5


def build(force: bool = False) -> str:
    """Compile ``fe_gen.c`` into a shared library (host compiler, -O2)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, u64, dbl, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.fe_draw_u64.restype = u64
            lib.fe_draw_u64.argtypes = [u64, u64, u64]
            lib.fe_uniform.restype = None
            lib.fe_uniform.argtypes = [u64, u64, i64, dbl, dbl, vp]
            lib.fe_normal.restype = None
            lib.fe_normal.argtypes = [u64, u64, i64, vp]
            lib.fe_laplace7_nnz.restype = i64
            lib.fe_laplace7_nnz.argtypes = [i64]
            lib.fe_laplace7.restype = i64
            lib.fe_laplace7.argtypes = [i64, vp, vp, vp]
            lib.fe_q1_nnz.restype = i64
            lib.fe_q1_nnz.argtypes = [i64]
            lib.fe_q1_rho.restype = None
            lib.fe_q1_rho.argtypes = [i64, dbl, u64, u64, vp]
            lib.fe_q1.restype = i64
            lib.fe_q1.argtypes = [i64, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class CSR:
    """A CSR matrix (0-based unless ``index_base`` is 1): the paper's IA/JA/AA."""

    row_ptr: np.ndarray  # int32[n+1]  (IA)
    col_idx: np.ndarray  # int32[nnz]  (JA)
    val: np.ndarray      # float64[nnz] (AA)
    n: int
    index_base: int = 0

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        b = self.index_base
        for i in range(self.n):
            for k in range(self.row_ptr[i] - b, self.row_ptr[i + 1] - b):
                d[i, self.col_idx[k] - b] += self.val[k]
        return d


def draw_u64(seed: int, stream: int, i: int) -> int:
    return int(_load().fe_draw_u64(seed, stream, i))


def uniform(seed: int, stream: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().fe_uniform(seed, stream, n, lo, hi, _ptr(out))
    return out


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().fe_normal(seed, stream, n, _ptr(out))
    return out


def laplace7(N: int) -> CSR:
    lib = _load()
    n = N ** 3
    nnz = int(lib.fe_laplace7_nnz(N))
    rp = np.empty(n + 1, dtype=np.int32)
    ci = np.empty(max(nnz, 0), dtype=np.int32)
    va = np.empty(max(nnz, 0), dtype=np.float64)
    got = lib.fe_laplace7(N, _ptr(rp), _ptr(ci), _ptr(va))
    if got != nnz:
        raise ValueError(f"laplace7({N}) does not fit int32 CSR indices")
    return CSR(rp, ci, va, n)


def q1_rho(N: int, sigma: float, seed: int, stream: int = STREAM_RHO) -> np.ndarray:
    rho = np.empty((N + 1) ** 3, dtype=np.float64)
    _load().fe_q1_rho(N, sigma, seed, stream, _ptr(rho))
    return rho


def q1(N: int, sigma: float = 1.0, seed: int = 0, rho: np.ndarray | None = None,
       stream: int = STREAM_RHO) -> CSR:
    """Q1 stiffness on an N^3 interior grid; rho_e = exp(sigma Z_e) unless given."""
    lib = _load()
    if rho is None:
        rho = q1_rho(N, sigma, seed, stream)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.shape != ((N + 1) ** 3,):
        raise ValueError("rho must hold (N+1)^3 element densities")
    n = N ** 3
    nnz = int(lib.fe_q1_nnz(N))
    rp = np.empty(n + 1, dtype=np.int32)
    ci = np.empty(max(nnz, 0), dtype=np.int32)
    va = np.empty(max(nnz, 0), dtype=np.float64)
    got = lib.fe_q1(N, _ptr(rho), _ptr(rp), _ptr(ci), _ptr(va))
    if got != nnz:
        raise ValueError(f"q1({N}) does not fit int32 CSR indices")
    return CSR(rp, ci, va, n)


def xstar(seed: int, n: int) -> np.ndarray:
    """Manufactured solution x* ~ U(-1, 1) from the seed."""
    return uniform(seed, STREAM_XSTAR, n, -1.0, 1.0)


def system_seed(seed: int, i: int) -> int:
    """Seed of system i of a batch or request stream drawn from `seed`
    (each system has its own densities and manufactured solution)."""
    return draw_u64(seed, STREAM_BATCH, 2 * i + 1) & 0x7FFFFFFFFFFFFFFF


def batch_edges(seed: int, count: int, lo: int = 8, hi: int = 48) -> np.ndarray:
    """Grid edges of a batch: N_i uniform on {lo, ..., hi}."""
    u = np.array([draw_u64(seed, STREAM_BATCH, 2 * i) for i in range(count)], dtype=np.uint64)
    return (lo + (u % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def arrivals(seed: int, count: int, rate: float, lo: int = 16, hi: int = 96,
             mu: float | None = None, sigma: float = 0.448) -> tuple[np.ndarray, np.ndarray]:
    """A request stream: Poisson arrivals at `rate` per second (times in s of
    seeded exponential gaps) and grid edges lognormal, ln N ~ N(mu, sigma^2)
    with mu = ln sqrt(lo hi) by default, rounded and clipped to [lo, hi]."""
    if mu is None:
        mu = 0.5 * (np.log(lo) + np.log(hi))
    u = uniform(seed, STREAM_ARRIVALS, count, 0.0, 1.0)
    gaps = -np.log1p(-u) / rate
    z = normal(seed, STREAM_ARRIVALS + 100, count)
    edges = np.clip(np.rint(np.exp(mu + sigma * z)), lo, hi).astype(np.int64)
    return np.cumsum(gaps), edges


def random_csr(n: int, seed: int, min_len: int = 0, max_len: int = 40,
               empty_frac: float = 0.1, long_rows: tuple[int, ...] = (),
               integer: bool = False, ncols: int | None = None) -> CSR:
    """Irregular CSR with sorted unique columns; some empty rows, some long rows.

    ``long_rows`` lists lengths of extra rows (placed at seeded positions) used
    to exercise rows longer than a warp or a staged tile.
    """
    ncols = n if ncols is None else ncols
    rng = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, STREAM_RANDOM_CSR]))
    lens = rng.integers(min_len, max_len + 1, size=n)
    if n > 0 and empty_frac > 0:
        lens[rng.random(n) < empty_frac] = 0
    for L in long_rows:
        if n > 0:
            lens[int(rng.integers(0, n))] = L
    lens = np.minimum(lens, ncols)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    nnz = int(rp[-1])
    ci = np.empty(nnz, dtype=np.int32)
    for i in range(n):
        L = int(lens[i])
        if L:
            ci[rp[i]:rp[i + 1]] = np.sort(rng.choice(ncols, size=L, replace=False))
    if integer:
        va = rng.integers(-8, 9, size=nnz).astype(np.float64)
    else:
        va = rng.uniform(-1.0, 1.0, size=nnz)
    return CSR(rp.astype(np.int32), ci, va, n)


def random_spd(n: int, seed: int, density: float = 0.3, shift: float = 1.0) -> CSR:
    """Small sparse SPD matrix: symmetric pattern, diagonally dominant values."""
    rng = np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, STREAM_RANDOM_CSR + 100]))
    d = np.zeros((n, n))
    mask = np.triu(rng.random((n, n)) < density, 1)
    vals = rng.uniform(-1.0, 1.0, size=(n, n))
    d[mask] = vals[mask]
    d = d + d.T
    d[np.diag_indices(n)] = np.abs(d).sum(axis=1) + shift * rng.uniform(0.5, 1.5, size=n)
    return dense_to_csr(d)


def dense_to_csr(d: np.ndarray) -> CSR:
    n = d.shape[0]
    rp = [0]
    ci: list[int] = []
    va: list[float] = []
    for i in range(n):
        nz = np.nonzero(d[i])[0]
        ci.extend(int(c) for c in nz)
        va.extend(float(d[i, c]) for c in nz)
        rp.append(len(ci))
    return CSR(np.array(rp, dtype=np.int32), np.array(ci, dtype=np.int32),
               np.array(va, dtype=np.float64), n)


def to_one_based(a: CSR) -> CSR:
    return CSR((a.row_ptr + 1).astype(np.int32), (a.col_idx + 1).astype(np.int32), a.val.copy(), a.n, 1)
