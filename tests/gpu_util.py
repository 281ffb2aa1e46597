"""Helpers of the GPU parity tests: upload CSR matrices, compare with the oracle."""
from __future__ import annotations

import math

import numpy as np

import fe_inputs as fi
import oracle


def cg_mod():
    import paper_2112_10823_gb300 as cg
    return cg


def dev_csr(A, device="cuda"):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.row_ptr, dtype=np.int32)).to(device),
            torch.from_numpy(np.ascontiguousarray(A.col_idx, dtype=np.int32)).to(device),
            torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).to(device))


def handle(A, **kw):
    cg = cg_mod()
    rp, ci, va = dev_csr(A)
    return cg.cg_create(rp, ci, va, n=A.n, nnz=A.nnz, index_base=getattr(A, "index_base", 0), **kw)


def abs_scale(A, x):
    """sum_k |a_ik| |x_jk| per row: the magnitude a rounding error is measured against."""
    return oracle.spmv(fi.CSR(A.row_ptr, A.col_idx, np.abs(A.val), A.n, getattr(A, "index_base", 0)), np.abs(x))


def spmv_tol(A, x, rel=1e-12):
    return rel * np.maximum(abs_scale(A, x), 1e-300)


def kappa_estimate(A, b):
    """Extreme Ritz values from the oracle's CG coefficients (Lanczos)."""
    r = oracle.cg(A, b, tol=1e-12, maxit=min(A.n, 3000), history=True)
    k = r.iters
    al, be = r.alpha, r.beta
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / al[i] + (be[i - 1] / al[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = math.sqrt(be[i]) / al[i]
    ev = np.linalg.eigvalsh(T)
    return ev[-1] / ev[0]


def iters_close(k_gpu: int, k_orc: int) -> bool:
    """Stopping iterations may differ by rounding of the sums near the threshold."""
    return abs(k_gpu - k_orc) <= max(2, math.ceil(0.01 * k_orc))


def hub_matrix(N: int, seed: int):
    """The 7-point operator on an N^3 grid with coupling rows of three kinds
    added symmetrically: row 0 coupled to every other row (a row longer than
    several ring pieces), row n/2 to every third row, 50 rows to 30 random
    rows each and 50 rows to 70 (rows of about 40 and 80 entries: two-lane
    and warp steps);
    each added coupling is -0.01 and adds 0.01 to both diagonals, plus 0.05
    on every diagonal (strictly diagonally dominant, hence SPD)."""
    L = fi.laplace7(N)
    n = L.n
    rows = [dict(zip(L.col_idx[L.row_ptr[i]:L.row_ptr[i + 1]].tolist(),
                     L.val[L.row_ptr[i]:L.row_ptr[i + 1]].tolist())) for i in range(n)]
    rng = np.random.default_rng(seed)

    def couple(i, j):
        if i == j or j in rows[i]:
            return
        rows[i][j] = -0.01
        rows[j][i] = -0.01
        rows[i][i] += 0.01
        rows[j][j] += 0.01

    for j in range(1, n):
        couple(0, j)
    for j in range(0, n, 3):
        couple(n // 2, j)
    for i in range(100, 200):
        for j in rng.choice(n, size=30 if i < 150 else 70, replace=False):
            couple(i, int(j))
    rp, ci, va = [0], [], []
    for i in range(n):
        rows[i][i] += 0.05
        cols = sorted(rows[i])
        ci.extend(cols)
        va.extend(rows[i][c] for c in cols)
        rp.append(len(ci))
    return fi.CSR(np.array(rp, dtype=np.int32), np.array(ci, dtype=np.int32), np.array(va), n)
