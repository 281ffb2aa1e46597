"""Jacobi-preconditioned CG (M = diag(A)) on the GPU against the oracle's
preconditioned CG, through the C ABI: single-system solves (FP64 and mixed)
and batched solves.  Same bar as plain CG: true residual <= 1e-10, stopping
step within max(2, 1%), solution within 1e-8 of the oracle run for the same
number of steps."""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
from gpu_util import cg_mod, handle, iters_close, kappa_estimate

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _solve(h, b):
    import torch
    cg = cg_mod()
    bd = torch.as_tensor(b, dtype=torch.float64).cuda()
    xd = torch.zeros_like(bd)
    res = cg.cg_solve(h, bd, xd, tol=TOL, maxit=10 * b.shape[0])
    return res, xd.cpu().numpy()


def _check(A, b, res, x):
    cg = cg_mod()
    assert res.status == cg.CG_OK, (res, cg.last_error())
    ref = oracle.pcg_jacobi(A, b, tol=TOL, maxit=10 * A.n)
    assert ref.status == oracle.OK
    assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
    same = oracle.pcg_jacobi(A, b, tol=0.0, maxit=res.iters, force_iters=res.iters)
    assert np.linalg.norm(x - same.x) <= 1e-8 * np.linalg.norm(same.x)
    true_rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert res.relres <= TOL and true_rel <= TOL * 1.0000001


@pytest.mark.parametrize("N,seed", [(7, 1), (24, 3), (40, 5)])
def test_jacobi_q1(N, seed):
    cg = cg_mod()
    A = fi.q1(N, 1.0, seed)
    b = oracle.spmv(A, fi.xstar(seed, A.n))
    with handle(A, preconditioner=cg.CG_PRECOND_JACOBI) as h:
        res, x = _solve(h, b)
    _check(A, b, res, x)
    # the preconditioner pays on the lognormal densities
    assert res.iters < oracle.cg(A, b, tol=TOL, maxit=10 * A.n).iters


def test_jacobi_irregular_spd_and_one_based():
    cg = cg_mod()
    A = fi.random_spd(300, 17, density=0.05, shift=2.0)
    b = oracle.spmv(A, fi.xstar(17, A.n))
    with handle(fi.to_one_based(A), preconditioner=cg.CG_PRECOND_JACOBI) as h:
        res, x = _solve(h, b)
    _check(A, b, res, x)


def test_jacobi_mixed_precision():
    cg = cg_mod()
    A = fi.q1(20, 1.0, 8)
    b = oracle.spmv(A, fi.xstar(8, A.n))
    with handle(A, precision=cg.CG_PREC_MIXED, preconditioner=cg.CG_PRECOND_JACOBI) as h:
        res, x = _solve(h, b)
    assert res.status == cg.CG_OK and res.relres <= TOL
    assert np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b) <= TOL * 1.0000001
    ref = oracle.pcg_jacobi(A, b, tol=TOL, maxit=10 * A.n)
    kap = kappa_estimate(A, b)
    assert np.linalg.norm(x - ref.x) <= 2.02 * kap * TOL * np.linalg.norm(ref.x)


def test_jacobi_refuses_nonpositive_diagonal():
    cg = cg_mod()
    A = fi.dense_to_csr(np.array([[2.0, 0.5, 0.0], [0.5, -1.0, 0.1], [0.0, 0.1, 3.0]]))
    with pytest.raises(cg.CGError) as e:
        handle(A, preconditioner=cg.CG_PRECOND_JACOBI)
    assert e.value.status == cg.CG_EINVAL and "not positive" in str(e.value)


def test_jacobi_batch():
    cg = cg_mod()
    systems = []
    for N, seed in ((5, 41), (9, 42), (14, 43), (22, 44)):
        A = fi.q1(N, 1.0, seed)
        systems.append((A, oracle.spmv(A, fi.xstar(seed, A.n))))
    bad = fi.dense_to_csr(np.array([[1.0, 0.0], [0.0, -2.0]]))
    with cg.Batch(preconditioner=cg.CG_PRECOND_JACOBI, group_override=0) as bt:
        reqs = [cg.Request(A.row_ptr, A.col_idx, A.val, b.copy(), np.zeros(A.n)) for A, b in systems]
        reqs.append(cg.Request(bad.row_ptr, bad.col_idx, bad.val, np.ones(2), np.zeros(2)))
        res = bt.wait_all(bt.submit(reqs), 120000)
    assert all(r.done for r in res)
    for (A, b), req, r in zip(systems, reqs, res):
        _check(A, b, cg.SolveResult(r.status, r.iters, r.relres), req.x)
    assert res[-1].status == cg.CG_EINVAL
