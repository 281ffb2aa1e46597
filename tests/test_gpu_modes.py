"""Solver paths that the finite-element systems do not reach, through the C
ABI: the mixed-precision product on rows of two-lanes-per-row and whole-warp
steps (rows of 33-64 and of more than 64 entries), and explicit CTA counts of
the persistent kernel (one CTA: no group barrier at all, and a share too
large for the small-share kernel; a few CTAs; the automatic choice)."""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
from gpu_util import cg_mod, handle, hub_matrix, iters_close, kappa_estimate

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _solve(h, b):
    import torch
    cg = cg_mod()
    bd = torch.as_tensor(b, dtype=torch.float64).cuda()
    xd = torch.zeros_like(bd)
    res = cg.cg_solve(h, bd, xd, tol=TOL, maxit=20 * b.shape[0])
    return res, xd.cpu().numpy()


@pytest.mark.parametrize("n,density", [(500, 0.09), (300, 0.3)])
def test_mixed_precision_irregular_rows(n, density):
    cg = cg_mod()
    A = fi.random_spd(n, 50 + n, density=density, shift=0.05)
    lens = np.diff(A.row_ptr)
    assert lens.max() > 32  # the FP32 ring product's pair / long-row steps are used
    b = oracle.spmv(A, fi.xstar(5, A.n))
    with handle(A, precision=cg.CG_PREC_MIXED) as h:
        res, x = _solve(h, b)
    assert res.status == cg.CG_OK, (res, cg.last_error())
    assert np.linalg.norm(b - oracle.spmv(A, x)) <= TOL * np.linalg.norm(b) * 1.0000001
    ref = oracle.cg_mixed(A, b, tol=TOL, maxit=20 * A.n)
    assert ref.status == oracle.OK
    kap = kappa_estimate(A, b)
    assert np.linalg.norm(x - ref.x) <= 2.02 * kap * TOL * np.linalg.norm(ref.x)


@pytest.mark.parametrize("ctas", [1, 3, 17, 0])
def test_cta_counts(ctas):
    cg = cg_mod()
    A = fi.q1(14, 1.0, 61)
    b = oracle.spmv(A, fi.xstar(61, A.n))
    with handle(A, ctas=ctas) as h:
        if ctas:
            assert h.nblocks == ctas
        else:
            assert 1 <= h.nblocks
        # one CTA holds all 2744 rows: the kernel with r in global memory;
        # 3 or 17 CTAs: the small-share kernel (r in shared memory); the CTA
        # count left automatic: the cluster kernel (a system this small)
        max_rows, kernel = h.partition_info()
        if ctas == 0:
            assert kernel == cg.CG_SOLVE_KERNEL_CLUSTER and max_rows == 256  # 2744 rows: 16 x 256 >= 2744
        else:
            assert max_rows == (A.n if ctas == 1 else max_rows) and max_rows >= -(-A.n // h.nblocks)
            assert kernel == (cg.CG_SOLVE_KERNEL_LARGE_SHARE if ctas == 1 else cg.CG_SOLVE_KERNEL_SMALL_SHARE)
        res, x = _solve(h, b)
    assert res.status == cg.CG_OK and res.relres <= TOL
    ref = oracle.cg(A, b, tol=TOL, maxit=20 * A.n)
    assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
    same = oracle.cg(A, b, tol=0.0, maxit=res.iters, force_iters=res.iters)
    assert np.linalg.norm(x - same.x) <= 1e-8 * np.linalg.norm(same.x)


def test_cta_count_products_agree_bitwise():
    """The CSR product's bits do not depend on the CTA count (each row is
    summed by one lane in storage order)."""
    import torch
    cg = cg_mod()
    A = fi.q1(13, 1.0, 62)
    x = torch.from_numpy(fi.xstar(62, A.n)).cuda()
    ys = []
    for c in (1, 5, 0):
        with handle(A, ctas=c) as h:
            y = torch.empty_like(x)
            cg.cg_spmv(h, x, y)
            ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])


def _permuted(A, seed):
    """P A P^T for a random permutation P: SPD, with each row's columns spread
    over the whole matrix (every CTA gathers p from every other)."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.n, A.n))
    perm = np.random.default_rng(seed).permutation(A.n)
    Mp = M[perm][:, perm].tocsr()
    Mp.sort_indices()
    return fi.CSR(Mp.indptr.astype(np.int32), Mp.indices.astype(np.int32), Mp.data.astype(np.float64), A.n)


@pytest.mark.parametrize("kind", ["q1_banded", "laplace_permuted"])
def test_large_share_kernel_neighbour_waits(kind):
    """CTA shares above 2560 rows with several CTAs: the kernel whose steps end
    with a wait for the CTAs owning the columns a CTA's rows reach (a banded Q1
    matrix: the adjacent CTAs; a randomly permuted Laplacian: all of them)."""
    cg = cg_mod()
    A = fi.q1(24, 1.0, 64) if kind == "q1_banded" else _permuted(fi.laplace7(20), 65)
    b = oracle.spmv(A, fi.xstar(64, A.n))
    with handle(A, ctas=3) as h:
        max_rows, kernel = h.partition_info()
        assert h.nblocks == 3 and max_rows > 2560 and kernel == cg.CG_SOLVE_KERNEL_LARGE_SHARE
        res, x = _solve(h, b)
        res2, x2 = _solve(h, b)  # the flags of the first solve do not leak into the second
    assert res.status == cg.CG_OK and res.relres <= TOL
    assert res2.iters == res.iters and np.array_equal(x, x2)
    ref = oracle.cg(A, b, tol=TOL, maxit=20 * A.n)
    assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
    same = oracle.cg(A, b, tol=0.0, maxit=res.iters, force_iters=res.iters)
    assert np.linalg.norm(x - same.x) <= 1e-8 * np.linalg.norm(same.x)


@pytest.mark.parametrize("N,precision", [(20, "fp64"), (20, "mixed"), (30, "fp64")])
def test_large_share_kernel_all_step_kinds(N, precision):
    """The large-share kernel over two CTAs on rows of every step kind at
    once (up to 9 entries, about 40, about 80, n/3 and n entries: one lane,
    two lanes, a warp per row, and rows spanning several 2,048-entry ring
    pieces; at N = 30 the longest row, 27,000 entries, is longer than the
    whole 16,384-entry ring): in FP64 the oracle's iterate at the GPU's step
    count, in mixed precision the FP64 solution within the residual's reach;
    the true residual, and the same bits on a second solve."""
    cg = cg_mod()
    A = hub_matrix(N, 71)
    lens = np.diff(A.row_ptr)
    assert lens.max() >= N ** 3 and ((lens > 32) & (lens <= 64)).any() and ((lens > 64) & (lens < 1000)).any()
    b = oracle.spmv(A, fi.xstar(71, A.n))
    mixed = precision == "mixed"
    with handle(A, ctas=2, precision=cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64) as h:
        assert h.partition_info()[1] == cg.CG_SOLVE_KERNEL_LARGE_SHARE
        res, x = _solve(h, b)
        res2, x2 = _solve(h, b)
    assert res.status == cg.CG_OK and res.relres <= TOL, res
    assert res2.iters == res.iters and np.array_equal(x, x2)
    assert np.linalg.norm(b - oracle.spmv(A, x)) <= 1.0000001 * TOL * np.linalg.norm(b)
    if mixed:
        # a long row's FP32 sum is split over a warp's lanes, which rounds
        # differently from the oracle's one FP32 chain per row, so the mixed
        # run is held to the FP64 solution (as for the other irregular rows)
        ref = oracle.cg(A, b, tol=TOL, maxit=20 * A.n)
        kap = kappa_estimate(A, b)
        assert np.linalg.norm(x - ref.x) <= 2.02 * kap * TOL * np.linalg.norm(ref.x)
    else:
        ref = oracle.cg(A, b, tol=TOL, maxit=20 * A.n)
        assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
        same = oracle.cg(A, b, tol=0.0, maxit=res.iters, force_iters=res.iters)
        assert np.linalg.norm(x - same.x) <= 1e-8 * np.linalg.norm(same.x)


@pytest.mark.parametrize("variant", ["mixed", "jacobi", "mixed_jacobi"])
def test_large_share_kernel_neighbour_waits_variants(variant):
    """The mixed-precision and Jacobi variants of the large-share kernel (the
    same neighbour wait) on the permuted Laplacian over three CTAs: the
    variant's own oracle, and the same bits on a second solve."""
    cg = cg_mod()
    A = _permuted(fi.laplace7(20), 66)
    b = oracle.spmv(A, fi.xstar(66, A.n))
    mixed = variant.startswith("mixed")
    jac = variant.endswith("jacobi")
    opts = {"precision": cg.CG_PREC_MIXED if mixed else cg.CG_PREC_FP64,
            "preconditioner": cg.CG_PRECOND_JACOBI if jac else cg.CG_PRECOND_NONE}
    with handle(A, ctas=3, **opts) as h:
        assert h.partition_info()[1] == cg.CG_SOLVE_KERNEL_LARGE_SHARE
        res, x = _solve(h, b)
        res2, x2 = _solve(h, b)
    assert res.status == cg.CG_OK and res.relres <= TOL, res
    assert res2.iters == res.iters and np.array_equal(x, x2)
    assert np.linalg.norm(b - oracle.spmv(A, x)) <= 1.0000001 * TOL * np.linalg.norm(b)
    ref = oracle.pcg_jacobi(A, b, tol=TOL, maxit=20 * A.n) if jac else oracle.cg_mixed(A, b, tol=TOL, maxit=20 * A.n)
    assert ref.status == oracle.OK
    if not mixed:  # FP64 Jacobi: the oracle's own steps
        assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
    kap = kappa_estimate(A, b)
    assert np.linalg.norm(x - ref.x) <= 2.02 * kap * TOL * np.linalg.norm(ref.x)


@pytest.mark.parametrize("kind", ["lap7_16", "q1_16", "rows_fewer_than_ctas", "irregular_long_rows"])
def test_cluster_kernel(kind):
    """Small plain FP64 systems with the CTA count left automatic run on one
    cluster of 16 CTAs holding the system in shared memory: parity with the
    oracle at equal iterations, the same bits on a second solve; systems with
    fewer rows than CTAs (empty CTAs) and rows longer than a batch of loads."""
    cg = cg_mod()
    if kind == "lap7_16":
        A = fi.laplace7(16)
    elif kind == "q1_16":
        A = fi.q1(16, 1.0, 67)
    elif kind == "rows_fewer_than_ctas":
        A = fi.random_spd(5, 68, density=0.6, shift=0.5)
    else:
        A = fi.random_spd(300, 69, density=0.3, shift=0.05)
        assert np.diff(A.row_ptr).max() > 16
    b = oracle.spmv(A, fi.xstar(67, A.n))
    with handle(A) as h:
        assert h.partition_info()[1] == cg.CG_SOLVE_KERNEL_CLUSTER
        res, x = _solve(h, b)
        res2, x2 = _solve(h, b)
    assert res.status == cg.CG_OK and res.relres <= TOL, res
    assert res2.iters == res.iters and np.array_equal(x, x2)
    assert np.linalg.norm(b - oracle.spmv(A, x)) <= 1.0000001 * TOL * np.linalg.norm(b)
    ref = oracle.cg(A, b, tol=TOL, maxit=20 * A.n)
    assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
    same = oracle.cg(A, b, tol=0.0, maxit=res.iters, force_iters=res.iters)
    assert np.linalg.norm(x - same.x) <= 1e-8 * np.linalg.norm(same.x)
