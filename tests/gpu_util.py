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
