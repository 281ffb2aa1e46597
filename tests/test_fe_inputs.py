"""The seeded input generator: structure of the operators and the random streams (CPU only)."""

import numpy as np

import fe_inputs as fi


def test_rng_counter_based_and_distributions():
    a = fi.uniform(7, fi.STREAM_XSTAR, 1000)
    b = fi.uniform(7, fi.STREAM_XSTAR, 1000)
    assert np.array_equal(a, b)                       # same seed -> same bits
    assert not np.array_equal(a, fi.uniform(8, fi.STREAM_XSTAR, 1000))
    assert not np.array_equal(a, fi.uniform(7, fi.STREAM_RHO, 1000))
    # counter-based: a prefix of a longer draw equals the shorter draw
    assert np.array_equal(fi.uniform(7, 1, 10), fi.uniform(7, 1, 1000)[:10])
    u = fi.uniform(1, 1, 200000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
    z = fi.normal(1, 2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    # SplitMix64 output function on a known input (Vigna's reference values for seed 0:
    # the first outputs of splitmix64 with state 0 are 0xe220a8397b1dcdaf, ...).
    # Here: key = mix(0) = 0, draw(0, 0, 0) = mix(GOLDEN) = first splitmix64 output.
    assert fi.draw_u64(0, 0, 0) == 0xE220A8397B1DCDAF


def test_laplace7_structure():
    for N in (1, 2, 3, 16):
        A = fi.laplace7(N)
        assert A.n == N ** 3 and A.nnz == 7 * N ** 3 - 6 * N ** 2
        D = A.to_dense() if A.n <= 512 else None
        if D is not None:
            assert np.array_equal(D, D.T)
            assert np.all(np.linalg.eigvalsh(D) > 0)
    A = fi.laplace7(5)
    assert np.all(np.diff(A.row_ptr) <= 7)
    for i in range(A.n):
        cols = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_q1_structure_and_symmetry():
    N = 6
    A = fi.q1(N, sigma=1.0, seed=3)
    assert A.n == N ** 3 and A.nnz == (3 * N - 2) ** 3
    D = A.to_dense()
    assert np.array_equal(D, D.T)                      # bitwise symmetric
    assert np.all(np.linalg.eigvalsh(D) > 0)           # SPD
    lens = np.diff(A.row_ptr)
    assert lens.max() == 27 and lens.min() == 8
    # face-neighbour entries are stored and exactly zero
    for i in [0, 37, A.n - 1, (N // 2) * (1 + N + N * N)]:
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = int(A.col_idx[k])
            d = np.array(np.unravel_index(j, (N, N, N))) - np.array(np.unravel_index(i, (N, N, N)))
            if np.count_nonzero(d) == 1:
                assert A.val[k] == 0.0
            else:
                assert A.val[k] != 0.0


def test_q1_row_sums_vanish_before_elimination():
    """Interior rows whose 27 neighbours are all unknowns sum to zero (the
    element matrices annihilate constants), up to assembly rounding."""
    N = 6
    A = fi.q1(N, sigma=1.0, seed=5)
    for k in range(1, N - 1):
        for j in range(1, N - 1):
            for i in range(1, N - 1):
                row = i + N * (j + N * k)
                vals = A.val[A.row_ptr[row]:A.row_ptr[row + 1]]
                assert len(vals) == 27
                assert abs(vals.sum()) <= 1e-14 * np.abs(vals).sum()


def test_q1_density_is_lognormal_and_seeded():
    N = 20
    rho = fi.q1_rho(N, 1.0, 9)
    z = np.log(rho)
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1.0) < 0.05
    assert np.array_equal(rho, fi.q1_rho(N, 1.0, 9))
    assert np.all(fi.q1_rho(N, 0.0, 9) == 1.0)
    # the matrix only depends on rho: given the same rho it is identical
    A1 = fi.q1(N, 1.0, 9)
    A2 = fi.q1(N, rho=rho)
    assert np.array_equal(A1.val, A2.val)


def test_config_sizes():
    assert fi.laplace7(16).nnz == 27136
    assert 262144 == 64 ** 3 and (3 * 64 - 2) ** 3 == 6859000
    assert (3 * 160 - 2) ** 3 == 109215352


def test_random_csr_edge_cases():
    A = fi.random_csr(100, 1, 0, 10, empty_frac=0.3, long_rows=(300,), ncols=400)
    lens = np.diff(A.row_ptr)
    assert (lens == 0).any() and lens.max() == 300
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz
    B = fi.to_one_based(A)
    assert B.row_ptr[0] == 1 and B.index_base == 1


def test_batch_edges_uniform_and_seeded():
    e = fi.batch_edges(0, 4000)
    assert e.min() >= 8 and e.max() <= 48
    assert np.array_equal(e, fi.batch_edges(0, 4000))
    assert not np.array_equal(e, fi.batch_edges(1, 4000))
    counts = np.bincount(e - 8, minlength=41)
    assert counts.min() > 0.6 * 4000 / 41 and counts.max() < 1.4 * 4000 / 41
    assert fi.system_seed(0, 0) != fi.system_seed(0, 1)


def test_arrivals_poisson_and_lognormal_edges():
    t, e = fi.arrivals(3, 20000, 2000.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 2000.0) < 0.03 / 2000.0        # exponential mean 1/rate
    assert abs(gaps.std() - 1 / 2000.0) < 0.05 / 2000.0          # and standard deviation 1/rate
    assert e.min() >= 16 and e.max() <= 96
    assert abs(np.median(np.log(e)) - 0.5 * np.log(16 * 96)) < 0.05
