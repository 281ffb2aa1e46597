"""Checks that tie the oracle to mathematics outside itself.

Each function raises AssertionError when the oracle disagrees with the fact
it states.  ``test_oracle_pins.py`` runs them against the oracle;
``test_oracle_mutants.py`` runs them against copies of the oracle with
planted mistakes and requires that some check fails for every mutant.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import fe_inputs as fi
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_paper_example():
    with open(os.path.join(GOLDEN, "paper_csr_example.json")) as f:
        g = json.load(f)
    A1 = fi.CSR(np.array(g["IA"], dtype=np.int32), np.array(g["JA"], dtype=np.int32),
                np.array(g["AA"], dtype=np.float64), 5, index_base=1)
    A0 = fi.CSR(A1.row_ptr - 1, A1.col_idx - 1, A1.val.copy(), 5, 0)
    return g, A1, A0


def pin_spmv_paper_example():
    """Sec. 2.3 worked example: exact integer products, 1-based and 0-based CSR."""
    g, A1, A0 = load_paper_example()
    for p in g["products"]:
        x = np.array(p["x"], dtype=np.float64)
        assert np.array_equal(oracle.spmv(A1, x), np.array(p["Ax"], dtype=np.float64))
        assert np.array_equal(oracle.spmv(A0, x), np.array(p["Ax"], dtype=np.float64))
    # The CSR arrays describe the printed dense matrix.
    assert np.array_equal(A1.to_dense(), np.array(g["dense"], dtype=np.float64))


def pin_spmv_dense_bruteforce(seed: int = 3):
    """Irregular CSR (empty rows, rows longer than 32) against a dense product."""
    for s in range(seed, seed + 3):
        A = fi.random_csr(60, s, 0, 12, empty_frac=0.2, long_rows=(45, 70), ncols=80)
        A.n = 60
        x = fi.uniform(s, 9, 80)
        D = np.zeros((60, 80))
        for i in range(60):
            for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
                D[i, A.col_idx[k]] += A.val[k]
        y = oracle.spmv(A, x)
        ref = D @ x
        scale = np.abs(D) @ np.abs(x)
        assert np.all(np.abs(y - ref) <= 1e-14 * np.maximum(scale, 1e-300))
        # integer-valued matrix and vector: every partial sum is exact
        Ai = fi.random_csr(60, s + 100, 0, 40, empty_frac=0.1, integer=True)
        xi = np.round(fi.uniform(s, 10, 60, -9, 9))
        Di = Ai.to_dense()
        assert np.array_equal(oracle.spmv(Ai, xi), Di @ xi)


def pin_spmv_rows():
    """The row-selected product (Sec. 2.3 definition restricted to listed rows):
    on the paper's 5x5 example its entries are the printed products' entries
    for any row list (shuffled, repeated), 1- and 0-based; on irregular 1-based
    CSR (empty rows, rows longer than 32) with a shuffled row list it equals
    the dense product's rows, exactly for integer data."""
    g, A1, A0 = load_paper_example()
    rows = np.array([4, 0, 2, 2, 3, 1, 4], dtype=np.int64)
    for p in g["products"]:
        x = np.array(p["x"], dtype=np.float64)
        want = np.array(p["Ax"], dtype=np.float64)[rows]
        assert np.array_equal(oracle.spmv_rows(A1, x, rows), want)
        assert np.array_equal(oracle.spmv_rows(A0, x, rows), want)
    assert oracle.spmv_rows(A1, np.ones(5), np.zeros(0, dtype=np.int64)).shape == (0,)
    for s in (5, 6):
        A = fi.random_csr(70, s, 0, 12, empty_frac=0.2, long_rows=(45, 70), ncols=70)
        A.n = 70
        A1i = fi.to_one_based(A)
        D = A.to_dense()
        x = fi.uniform(s, 19, 70)
        sel = np.random.default_rng(s).permutation(70)[:41].astype(np.int64)
        ref = (D @ x)[sel]
        scale = (np.abs(D) @ np.abs(x))[sel]
        for M in (A, A1i):
            y = oracle.spmv_rows(M, x, sel)
            assert np.all(np.abs(y - ref) <= 1e-14 * np.maximum(scale, 1e-300))
        Ai = fi.random_csr(70, s + 50, 0, 40, empty_frac=0.1, integer=True)
        xi = np.round(fi.uniform(s, 20, 70, -9, 9))
        assert np.array_equal(oracle.spmv_rows(fi.to_one_based(Ai), xi, sel), (Ai.to_dense() @ xi)[sel])


def laplace7_eigpair(N: int, j: int, k: int, l: int):
    idx = np.arange(1, N + 1)
    th = np.pi / (N + 1)
    sx, sy, sz = np.sin(j * th * idx), np.sin(k * th * idx), np.sin(l * th * idx)
    v = (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).ravel()
    lam = sum(4.0 * math.sin(m * math.pi / (2 * (N + 1))) ** 2 for m in (j, k, l))
    return v, lam


def pin_laplace7_eigenpairs(N: int = 9):
    """A v = lambda v for the sine modes of the 7-point operator (closed form)."""
    A = fi.laplace7(N)
    for (j, k, l) in [(1, 1, 1), (N, N, N), (1, 2, 3), (4, 1, 7), (2, 9, 5)]:
        v, lam = laplace7_eigpair(N, j, k, l)
        Av = oracle.spmv(A, v)
        assert np.linalg.norm(Av - lam * v) <= 1e-13 * lam * np.linalg.norm(v)


def q1_eigpair(N: int, j: int, k: int, l: int):
    v, _ = laplace7_eigpair(N, j, k, l)
    h = 1.0 / (N + 1)

    def km(m):
        c = math.cos(m * math.pi / (N + 1))
        return 2.0 - 2.0 * c, (4.0 + 2.0 * c) / 6.0

    (kj, mj), (kk, mk), (kl, ml) = km(j), km(k), km(l)
    return v, h * (kj * mk * ml + mj * kk * ml + mj * mk * kl)


def pin_q1_eigenpairs(N: int = 7):
    """Constant-density Q1 operator: sine modes with lambda = h(k m m + m k m + m m k)."""
    A = fi.q1(N, sigma=0.0, seed=0)
    for (j, k, l) in [(1, 1, 1), (N, N, N), (2, 3, 1), (6, 1, 4)]:
        v, lam = q1_eigpair(N, j, k, l)
        Av = oracle.spmv(A, v)
        assert np.linalg.norm(Av - lam * v) <= 1e-12 * lam * np.linalg.norm(v)


def pin_blas1(seed: int = 5):
    """dot against an exactly rounded sum; axpy and ewmul elementwise."""
    n = 1001
    x, y = fi.uniform(seed, 1, n), fi.uniform(seed, 2, n)
    exact = math.fsum(float(a) * float(b) for a, b in zip(x, y))  # products are rounded, sum exact
    d = oracle.dot(x, y)
    assert abs(d - exact) <= n * 2.0 ** -53 * float(np.sum(np.abs(x * y))) * 2
    xi, yi = np.round(x * 1000), np.round(y * 1000)
    assert oracle.dot(xi, yi) == float(np.sum(xi.astype(np.int64) * yi.astype(np.int64)))
    assert oracle.dot(x[:0], y[:0]) == 0.0
    a = 0.37
    assert np.array_equal(oracle.axpy(a, xi, yi), a * xi + yi)
    assert np.array_equal(oracle.axpy(2.0, xi, yi), 2.0 * xi + yi)
    assert np.array_equal(oracle.ewmul(x, y), x * y)


def pin_cg_finite_termination():
    """Tiny SPD systems: CG reaches 1e-10 in at most n (+2 rounding slack) steps
    and matches a dense direct solve."""
    for s, n in [(1, 5), (2, 12), (3, 20)]:
        A = fi.random_spd(n, s, density=0.5)
        D = A.to_dense()
        xs = fi.uniform(s, 7, n)
        b = D @ xs
        r = oracle.cg(A, b, tol=1e-10, maxit=n + 2)
        assert r.status == oracle.OK
        assert r.iters <= n + 2
        xd = np.linalg.solve(D, b)
        assert np.linalg.norm(r.x - xd) <= 1e-8 * np.linalg.norm(xd)
        assert r.relres_true <= 1e-9


def pin_cg_monotone_error(N: int = 6):
    """||x_k - x*||_A and ||x_k - x*||_2 decrease monotonically (Hestenes-Stiefel)."""
    A = fi.q1(N, sigma=1.0, seed=11)
    D = A.to_dense()
    xs = fi.xstar(11, A.n)
    b = D @ xs
    full = oracle.cg(A, b, tol=1e-10, maxit=10 * A.n)
    assert full.status == oracle.OK
    prev_a, prev_2 = math.inf, math.inf
    for k in range(0, full.iters + 1):
        xk = oracle.cg(A, b, force_iters=k).x
        e = xk - xs
        ea, e2 = math.sqrt(e @ D @ e), np.linalg.norm(e)
        assert ea <= prev_a * (1 + 1e-12) + 1e-13
        assert e2 <= prev_2 * (1 + 1e-12) + 1e-13
        prev_a, prev_2 = ea, e2


def pin_cg_laplace_bounds(N: int = 16):
    """7-point operator with closed-form kappa: Chebyshev residual bound, the
    iteration count it implies, Lanczos extreme Ritz values, and the error of
    the manufactured solution."""
    A = fi.laplace7(N)
    lmin = 3 * 4.0 * math.sin(math.pi / (2 * (N + 1))) ** 2
    lmax = 3 * 4.0 * math.sin(N * math.pi / (2 * (N + 1))) ** 2
    kappa = lmax / lmin
    xs = fi.xstar(0, A.n)
    b = oracle.spmv(A, xs)
    r = oracle.cg(A, b, tol=1e-10, maxit=A.n, history=True)
    assert r.status == oracle.OK and r.relres_true <= 1.5e-10
    c = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    for k, rk in enumerate(r.res):
        assert rk / r.res[0] <= 2 * math.sqrt(kappa) * c ** k * (1 + 1e-9)
    kmax = math.ceil(math.log(1e-10 / (2 * math.sqrt(kappa))) / math.log(c))
    assert r.iters <= kmax
    # Lanczos tridiagonal from the CG coefficients (Saad, Sec. 6.7.3)
    k = r.iters
    al, be = r.alpha, r.beta
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / al[i] + (be[i - 1] / al[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = math.sqrt(be[i]) / al[i]
    ev = np.linalg.eigvalsh(T)
    assert abs(ev[0] - lmin) <= 1e-6 * lmin
    assert abs(ev[-1] - lmax) <= 1e-6 * lmax
    err = np.linalg.norm(r.x - xs) / np.linalg.norm(xs)
    assert err <= kappa * r.relres_true * 1.01


def pin_cg_orthogonality():
    """Residuals of early steps are mutually orthogonal, and the search
    directions are A-conjugate: d_k = x_{k+1} - x_k = alpha_k p_k gives
    d_i . A d_j = 0 for i != j (Hestenes-Stiefel)."""
    A = fi.q1(5, sigma=1.0, seed=4)
    xs = fi.xstar(4, A.n)
    b = oracle.spmv(A, xs)
    rs, xk = [], []
    for k in range(7):
        xk.append(oracle.cg(A, b, force_iters=k).x)
        rs.append(b - oracle.spmv(A, xk[-1]))
    for i in range(6):
        for j in range(i):
            c = abs(rs[i] @ rs[j]) / (np.linalg.norm(rs[i]) * np.linalg.norm(rs[j]))
            assert c <= 1e-8, (i, j, c)
    d = [xk[k + 1] - xk[k] for k in range(6)]
    Ad = [oracle.spmv(A, v) for v in d]
    for i in range(6):
        for j in range(i):
            c = abs(d[i] @ Ad[j]) / math.sqrt((d[i] @ Ad[i]) * (d[j] @ Ad[j]))
            assert c <= 1e-8, (i, j, c)


def pin_cg_special_cases():
    """b = 0; maxit reached; an indefinite matrix; a nonzero initial guess."""
    A = fi.laplace7(4)
    r = oracle.cg(A, np.zeros(A.n))
    assert r.status == oracle.OK and r.iters == 0 and np.all(r.x == 0)
    b = oracle.spmv(A, fi.xstar(1, A.n))
    r = oracle.cg(A, b, tol=1e-14, maxit=2)
    assert r.status == oracle.NOTCONV and r.iters == 2
    Ind = fi.dense_to_csr(np.diag([1.0, -1.0]))
    r = oracle.cg(Ind, np.array([1.0, 1.0]))
    assert r.status == oracle.BREAKDOWN
    xs = fi.xstar(2, A.n)
    b = oracle.spmv(A, xs)
    r = oracle.cg(A, b, tol=1e-12, maxit=A.n, x0=xs)   # exact guess: no step needed
    assert r.iters == 0 and r.relres_true <= 1e-15


def pin_mixed_cg():
    """Mixed precision reaches the FP64 true residual 1e-10 and the solution
    agrees with a dense solve; its FP32 product matches the FP64 product to
    FP32 rounding."""
    A = fi.q1(8, sigma=1.0, seed=21)
    D = A.to_dense()
    xs = fi.xstar(21, A.n)
    b = D @ xs
    r = oracle.cg_mixed(A, b, tol=1e-10, replace_every=20)
    assert r.status == oracle.OK, r
    assert r.relres_true <= 1e-10
    xd = np.linalg.solve(D, b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(r.x - xd) <= kappa * 1e-10 * np.linalg.norm(xd) * 2
    v32 = A.val.astype(np.float32)
    x32 = xs.astype(np.float32)
    y32 = oracle.spmv_f32(A, v32, x32).astype(np.float64)
    ref = np.abs(D) @ np.abs(xs)
    assert np.all(np.abs(y32 - D @ xs) <= 40 * 2.0 ** -24 * ref)
    # Systems whose recursive residual reaches the tolerance before the first
    # periodic replacement (the FP32 product has drifted it away from the true
    # one by then): mixed precision must still reach the FP64 true residual,
    # within a few steps of what FP64 CG needs (a refinement step costs a few).
    for N, seed in ((4, 1), (6, 906), (10, 910)):
        A = fi.q1(N, sigma=1.0, seed=seed)
        D = A.to_dense()
        b = D @ fi.xstar(seed, A.n)
        r = oracle.cg_mixed(A, b, tol=1e-10, replace_every=50)
        r64 = oracle.cg(A, b, tol=1e-10, maxit=10 * A.n)
        assert r.status == oracle.OK, (N, r.status, r.iters)
        assert np.linalg.norm(b - D @ r.x) <= 1e-10 * np.linalg.norm(b) * 1.0000001
        assert r.iters <= 1.5 * r64.iters + 10, (N, r.iters, r64.iters)


def pin_mixed_forced_steps():
    """The mixed iteration run for exactly k steps (force_iters), against facts
    outside it:
    (1) one step from x0 = 0 on an integer matrix with an integer right-hand
        side: the FP32 product of integers below 2^24 is exact, so the step is
        the textbook first CG step x1 = (b.b / b.Ab) b, to the bit;
    (2) a residual replacement every `every` steps: after a multiple of
        `every` steps the recursive residual is the true residual b - A x, to
        the bit, and in between it is not (the FP32 product drifts it);
    (3) early iterates stay within FP32 rounding of FP64 CG's iterates for the
        same step count, far closer than to the neighbouring steps';
    (4) forcing the converged run's step count reproduces it to the bit, and
        forcing more steps than convergence needs runs them all."""
    L = fi.laplace7(5)
    D = L.to_dense()
    bi = np.round(fi.uniform(41, 3, L.n, -9, 9))
    r1 = oracle.cg_mixed(L, bi, tol=0.0, replace_every=50, force_iters=1)
    bb, bab = int(np.dot(bi.astype(np.int64), bi.astype(np.int64))), int(bi.astype(np.int64) @ (D.astype(np.int64) @ bi.astype(np.int64)))
    alpha = float(bb) / float(bab)
    assert r1.iters == 1 and np.array_equal(r1.x, alpha * bi)
    # (2)
    A = fi.q1(6, sigma=1.0, seed=43)
    b = oracle.spmv(A, fi.xstar(43, A.n))
    every = 4
    differ = 0
    for k in range(1, 13):
        r = oracle.cg_mixed(A, b, tol=1e-30, replace_every=every, force_iters=k)
        assert r.iters == k
        if k % every == 0:
            assert r.relres_rec == r.relres_true, (k, r.relres_rec, r.relres_true)
        else:
            differ += r.relres_rec != r.relres_true
    assert differ >= 6, differ
    # (3)
    prev = None
    for k in range(1, 9):
        xm = oracle.cg_mixed(A, b, tol=0.0, replace_every=50, force_iters=k).x
        x64 = oracle.cg(A, b, tol=0.0, maxit=k, force_iters=k).x
        d = np.linalg.norm(xm - x64)
        assert d <= 1e-5 * np.linalg.norm(x64), (k, d)
        if prev is not None:
            assert np.linalg.norm(x64 - prev) >= 100 * d, k
        prev = x64
    # (4)
    conv = oracle.cg_mixed(A, b, tol=1e-10, replace_every=every)
    assert conv.status == oracle.OK
    again = oracle.cg_mixed(A, b, tol=1e-10, replace_every=every, force_iters=conv.iters)
    assert again.iters == conv.iters and np.array_equal(again.x, conv.x)
    more = oracle.cg_mixed(A, b, tol=1e-10, replace_every=every, force_iters=conv.iters + 7)
    assert more.iters == conv.iters + 7 and more.relres_true <= 1e-9


def pin_matrix_stats(golden_table1=True):
    """Table 1 column definitions: the 5x5 example by hand and the paper's own
    density and nz/h columns recomputed from its h and nz."""
    g, A1, A0 = load_paper_example()
    st = oracle.matrix_stats(A1)
    for key, v in g["stats"].items():
        assert abs(st[key] - v) <= 1e-12, (key, st[key], v)
    with open(os.path.join(GOLDEN, "paper_table1.json")) as f:
        t1 = json.load(f)
    for row in t1["rows"][1:3]:  # row 0 holds a misprinted nz/h (see the fixture's reading)
        h, nz = int(row[0]), int(row[1])
        lens = np.full(h, nz // h, dtype=np.int64)
        lens[: nz % h] += 1
        rp = np.zeros(h + 1, dtype=np.int64)
        rp[1:] = np.cumsum(lens)
        ci = np.zeros(nz, dtype=np.int32)  # columns do not enter density or nz/h
        A = fi.CSR(rp.astype(np.int32), ci, np.zeros(nz), h)
        s = oracle.matrix_stats(A)
        assert round(100.0 * s["density"], 3) == row[2]
        assert round(s["nz_per_h"], 3) == row[5]
    # Stencil matrices: bandwidth, max_row and nz in closed form.
    N = 5
    s7 = oracle.matrix_stats(fi.laplace7(N))
    assert s7["bandwidth"] == N * N and s7["max_row"] == 7 and s7["nz"] == 7 * N**3 - 6 * N**2
    sq = oracle.matrix_stats(fi.q1(N, 1.0, 0))
    assert sq["bandwidth"] == N * N + N + 1 and sq["max_row"] == 27 and sq["nz"] == (3 * N - 2) ** 3
    # row lengths of the Q1 pattern: 27 inside, fewer next to the boundary
    lens = np.where((np.arange(N) > 0) & (np.arange(N) < N - 1), 3, 2)
    L = (lens[:, None, None] * lens[None, :, None] * lens[None, None, :]).ravel()
    assert abs(sq["nz_per_h_stddev"] - float(np.std(L))) <= 1e-12


def pin_pcg_jacobi():
    """Jacobi-preconditioned CG against facts outside it.
    (1) Symmetric scaling: with D = diag(A), PCG's iterates are D^(-1/2) times
        those of plain CG on D^(-1/2) A D^(-1/2) with right-hand side
        D^(-1/2) b (the textbook equivalence), step by step.
    (2) A diagonal matrix is its own preconditioner: one step gives the exact
        solution.
    (3) A constant diagonal (the 7-point operator, diagonal 6) makes the
        preconditioner a multiple of the identity: the iterates are CG's.
    (4) The inverse diagonal is the reciprocal of the brute-force diagonal;
        a non-positive diagonal is refused (breakdown).
    (5) The stopping test is on the unpreconditioned residual: with a large
        diagonal the stop is the first step with ||b - A x|| <= tol ||b||."""
    A = fi.q1(5, sigma=1.0, seed=31)
    D = A.to_dense()
    d = np.diag(D).copy()
    dinv = oracle.jacobi_dinv(A)
    assert dinv is not None and np.allclose(dinv, 1.0 / d, rtol=1e-15, atol=0)
    s = 1.0 / np.sqrt(d)
    As = fi.dense_to_csr(D * s[:, None] * s[None, :])
    b = D @ fi.xstar(31, A.n)
    for k in (1, 2, 3, 5, 8, 13):
        xp = oracle.pcg_jacobi(A, b, tol=0.0, maxit=k, force_iters=k).x
        xh = oracle.cg(As, s * b, tol=0.0, maxit=k, force_iters=k).x
        assert np.linalg.norm(xp - s * xh) <= 1e-10 * np.linalg.norm(xp), k
    r = oracle.pcg_jacobi(A, b, tol=1e-10, maxit=10 * A.n)
    assert r.status == oracle.OK and r.relres_true <= 1e-10 * 1.0000001
    xd = np.linalg.solve(D, b)
    assert np.linalg.norm(r.x - xd) <= 2 * np.linalg.cond(D) * 1e-10 * np.linalg.norm(xd)
    # (2)
    Dg = fi.dense_to_csr(np.diag(np.arange(1.0, 9.0)))
    bg = np.arange(1.0, 9.0) ** 2
    r = oracle.pcg_jacobi(Dg, bg, tol=1e-14, maxit=10)
    assert r.iters == 1 and np.allclose(r.x, np.arange(1.0, 9.0), rtol=1e-15)
    # (3)
    L = fi.laplace7(6)
    bl = oracle.spmv(L, fi.xstar(32, L.n))
    rp, rc = oracle.pcg_jacobi(L, bl, tol=1e-10, maxit=1000), oracle.cg(L, bl, tol=1e-10, maxit=1000)
    assert abs(rp.iters - rc.iters) <= 1
    assert np.linalg.norm(rp.x - rc.x) <= 1e-9 * np.linalg.norm(rc.x)
    # (5) the stopping test is on the unpreconditioned residual: on a system
    # whose diagonal is large (z = r / 6000) the solve stops at the first
    # step whose ||b - A x|| (recursive, and recomputed) is within tol ||b||
    Lb = fi.laplace7(6)
    Lb.val = Lb.val * 1000.0
    bb = oracle.spmv(Lb, fi.xstar(33, Lb.n))
    r = oracle.pcg_jacobi(Lb, bb, tol=1e-8, maxit=1000)
    assert r.status == oracle.OK and r.relres_rec <= 1e-8 and r.relres_true <= 1.01e-8
    prev = oracle.pcg_jacobi(Lb, bb, tol=0.0, maxit=r.iters - 1, force_iters=r.iters - 1)
    res_prev = np.linalg.norm(bb - oracle.spmv(Lb, prev.x)) / np.linalg.norm(bb)
    assert res_prev > 1e-8 * 0.99
    # (4)
    Bad = fi.dense_to_csr(np.array([[2.0, 0.5], [0.5, -1.0]]))
    assert oracle.jacobi_dinv(Bad) is None
    assert oracle.pcg_jacobi(Bad, np.ones(2)).status == oracle.BREAKDOWN


def pin_omp_variant():
    """The OpenMP timing variant against the sequential oracle (itself pinned
    above) and against mathematics: with one thread the same bits for CG,
    mixed-precision CG and the product; with every host core the product's
    bits, iterates at equal step counts within 1e-9 relative (the dot
    products' block order is the only difference), stopping steps within
    max(2, 1 %) (mixed: max(5, 5 %)); the mixed run's replacement schedule;
    the 7-point Laplacian's Chebyshev step bound; b = 0 and breakdown."""
    if not oracle.omp_available():
        import pytest
        pytest.skip("no OpenMP on this host compiler")
    cases = [(fi.laplace7(16), 0), (fi.q1(12, 1.0, 1), 1), (fi.q1(20, 1.0, 3), 3)]
    full = oracle.omp_threads()
    try:
        for T in (1, max(full, 3)):
            oracle.omp_set_threads(T)
            for A, seed in cases:
                b = oracle.spmv(A, fi.xstar(seed, A.n))
                assert np.array_equal(oracle.omp_spmv(A, b), oracle.spmv(A, b))
                seq = oracle.cg(A, b, tol=1e-10, maxit=10 * A.n)
                par = oracle.omp_cg(A, b, tol=1e-10, maxit=10 * A.n)
                assert par.status == oracle.OK and par.relres_true <= 1e-10 * 1.0000001
                if T == 1:
                    assert par.iters == seq.iters and np.array_equal(par.x, seq.x)
                    assert par.relres_true == seq.relres_true
                    assert oracle.omp_dot(b, b) == oracle.dot(b, b)
                else:
                    assert abs(par.iters - seq.iters) <= max(2, math.ceil(0.01 * seq.iters))
                    same = oracle.cg(A, b, force_iters=par.iters)
                    assert np.linalg.norm(par.x - same.x) <= 1e-9 * np.linalg.norm(same.x)
                    exact = math.fsum((b * b).tolist())
                    assert abs(oracle.omp_dot(b, b) - exact) <= 2 * A.n * 2.0 ** -53 * exact
        # the mixed-precision iteration: bitwise the sequential one with one
        # thread; on every core the same iterates at equal steps within 1e-9 and
        # stopping steps within max(5, 5 %) (the mixed stop's own spread)
        Am = fi.q1(12, 1.0, 5)
        bm = oracle.spmv(Am, fi.xstar(5, Am.n))
        for T in (1, max(full, 3)):
            oracle.omp_set_threads(T)
            seqm = oracle.cg_mixed(Am, bm, tol=1e-10, replace_every=20)
            parm = oracle.omp_cg_mixed(Am, bm, tol=1e-10, replace_every=20)
            assert parm.status == oracle.OK and parm.relres_true <= 1e-10 * 1.0000001
            if T == 1:
                assert parm.iters == seqm.iters and np.array_equal(parm.x, seqm.x)
                assert parm.relres_rec == seqm.relres_rec
            else:
                assert abs(parm.iters - seqm.iters) <= max(5, math.ceil(0.05 * seqm.iters))
                same = oracle.cg_mixed(Am, bm, tol=1e-10, replace_every=20, force_iters=parm.iters)
                assert np.linalg.norm(parm.x - same.x) <= 1e-9 * np.linalg.norm(same.x)
            forced = oracle.omp_cg_mixed(Am, bm, tol=1e-30, replace_every=4, force_iters=8)
            assert forced.iters == 8 and forced.relres_rec == forced.relres_true
            beyond = oracle.omp_cg_mixed(Am, bm, tol=1e-10, replace_every=20, force_iters=parm.iters + 5)
            assert beyond.iters == parm.iters + 5 and beyond.relres_true <= 1e-9
        oracle.omp_set_threads(full)
        N = 16
        A = fi.laplace7(N)
        lmin = 12.0 * math.sin(math.pi / (2 * (N + 1))) ** 2
        lmax = 12.0 * math.sin(N * math.pi / (2 * (N + 1))) ** 2
        c = (math.sqrt(lmax / lmin) - 1) / (math.sqrt(lmax / lmin) + 1)
        kmax = math.ceil(math.log(1e-10 / (2 * math.sqrt(lmax / lmin))) / math.log(c))
        r = oracle.omp_cg(A, oracle.spmv(A, fi.xstar(0, A.n)), tol=1e-10, maxit=A.n)
        assert r.status == oracle.OK and r.iters <= kmax
        z = oracle.omp_cg(A, np.zeros(A.n), x0=np.ones(A.n))
        assert z.status == oracle.OK and z.iters == 0 and np.all(z.x == 0)
        Ind = fi.dense_to_csr(np.diag([1.0, -1.0]))
        assert oracle.omp_cg(Ind, np.array([1.0, 1.0])).status == oracle.BREAKDOWN
    finally:
        oracle.omp_set_threads(full)


ALL_PINS = [
    pin_spmv_paper_example,
    pin_spmv_dense_bruteforce,
    pin_spmv_rows,
    pin_laplace7_eigenpairs,
    pin_q1_eigenpairs,
    pin_blas1,
    pin_cg_finite_termination,
    pin_cg_monotone_error,
    pin_cg_laplace_bounds,
    pin_cg_orthogonality,
    pin_cg_special_cases,
    pin_mixed_cg,
    pin_mixed_forced_steps,
    pin_pcg_jacobi,
    pin_matrix_stats,
    pin_omp_variant,
]
