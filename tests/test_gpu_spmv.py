"""CSR product on the GPU against the oracle (through the C ABI)."""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
from gpu_util import cg_mod, dev_csr, handle, spmv_tol
from pins import load_paper_example

pytestmark = pytest.mark.gpu


def gpu_spmv(h, x):
    import torch
    cg = cg_mod()
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    yd = torch.full_like(xd, float("nan"))
    cg.cg_spmv(h, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_paper_example_exact():
    """Sec. 2.3 matrix: integer products are exact in any summation order."""
    g, A1, A0 = load_paper_example()
    for A in (A1, A0):
        with handle(A) as h:
            for p in g["products"]:
                y = gpu_spmv(h, np.array(p["x"], dtype=np.float64))
                assert np.array_equal(y, np.array(p["Ax"], dtype=np.float64))


@pytest.mark.parametrize("N", [16, 5])
def test_laplace7(N):
    A = fi.laplace7(N)
    x = fi.uniform(N, 3, A.n)
    with handle(A) as h:
        y = gpu_spmv(h, x)
    ref = oracle.spmv(A, x)
    assert np.all(np.abs(y - ref) <= spmv_tol(A, x))


@pytest.mark.parametrize("N,seed", [(24, 2), (7, 3), (1, 4), (2, 5)])
def test_q1(N, seed):
    A = fi.q1(N, 1.0, seed)
    x = fi.uniform(seed, 3, A.n)
    with handle(A) as h:
        y = gpu_spmv(h, x)
    ref = oracle.spmv(A, x)
    assert np.all(np.abs(y - ref) <= spmv_tol(A, x))


def test_q1_n64_full():
    """The 64^3 workload, every row."""
    A = fi.q1(64, 1.0, 0)
    x = fi.xstar(0, A.n)
    with handle(A) as h:
        y = gpu_spmv(h, x)
    ref = oracle.spmv(A, x)
    assert np.all(np.abs(y - ref) <= spmv_tol(A, x))


def test_q1_n160_sampled_rows():
    """The 160^3 workload (109M entries) in the bench's configuration: sampled
    rows recomputed one by one by the oracle, plus every chunk boundary row."""
    import torch
    A = fi.q1(160, 1.0, 0)
    x = fi.xstar(0, A.n)
    with handle(A) as h:
        y = gpu_spmv(h, x)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.integers(0, A.n, 20000), [0, 1, A.n - 2, A.n - 1],
                                     np.arange(0, A.n, 4096)]))
    ref = oracle.spmv_rows(A, x, rows)
    sc = oracle.spmv_rows(fi.CSR(A.row_ptr, A.col_idx, np.abs(A.val), A.n), np.abs(x), rows)
    assert np.all(np.abs(y[rows] - ref) <= 1e-12 * sc)
    assert np.all(np.isfinite(y))
    del A
    torch.cuda.empty_cache()


@pytest.mark.parametrize("seed", [1, 2])
def test_irregular_rows(seed):
    """Empty rows, rows longer than a warp, longer than a shared-memory stage
    (streamed by the whole CTA), and warp-per-row chunks; integer data -> exact."""
    A = fi.random_csr(12000, seed, 0, 30, empty_frac=0.15,
                      long_rows=(40, 100, 300, 5000, 9000, 11000), integer=True)
    x = np.round(fi.uniform(seed, 5, A.n, -9, 9))
    with handle(A) as h:
        y = gpu_spmv(h, x)
    assert np.array_equal(y, oracle.spmv(A, x))   # integer sums are exact on both sides
    Af = fi.random_csr(6000, seed + 10, 0, 80, empty_frac=0.1, long_rows=(9000, 12000))
    xf = fi.uniform(seed, 6, Af.n)
    with handle(Af) as h:
        yf = gpu_spmv(h, xf)
    assert np.all(np.abs(yf - oracle.spmv(Af, xf)) <= spmv_tol(Af, xf))


def test_long_rows_only():
    """Rows averaging > 48 entries: warp-per-row chunks everywhere."""
    A = fi.random_csr(700, 9, 60, 200, empty_frac=0.0)
    x = fi.uniform(9, 1, A.n)
    with handle(A) as h:
        y = gpu_spmv(h, x)
    assert np.all(np.abs(y - oracle.spmv(A, x)) <= spmv_tol(A, x))


def test_all_empty_and_single_row():
    A = fi.CSR(np.zeros(11, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0), 10)
    with handle(A) as h:
        y = gpu_spmv(h, np.ones(10))
    assert np.array_equal(y, np.zeros(10))
    B = fi.dense_to_csr(np.array([[3.5]]))
    with handle(B) as h:
        assert gpu_spmv(h, np.array([2.0]))[0] == 7.0


def test_empty_matrix_is_noop():
    import torch
    cg = cg_mod()
    A = fi.CSR(np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0), 0)
    with handle(A) as h:
        x = torch.zeros(0, dtype=torch.float64, device="cuda")
        cg.cg_spmv(h, x, x)


def test_one_based_device_input():
    A = fi.q1(9, 1.0, 8)
    A1 = fi.to_one_based(A)
    x = fi.uniform(8, 2, A.n)
    with handle(A1) as h:
        y1 = gpu_spmv(h, x)
    with handle(A) as h:
        y0 = gpu_spmv(h, x)
    assert np.array_equal(y0, y1)
    assert np.all(np.abs(y0 - oracle.spmv(A1, x)) <= spmv_tol(A, x))


def test_host_arrays_and_determinism():
    cg = cg_mod()
    A = fi.q1(20, 1.0, 6)
    x = fi.uniform(6, 2, A.n)
    h1 = cg.cg_create(A.row_ptr, A.col_idx, A.val)   # host (numpy) CSR
    y1 = gpu_spmv(h1, x)
    y2 = gpu_spmv(h1, x)
    h1.close()
    with handle(A) as h2:
        y3 = gpu_spmv(h2, x)
    assert np.array_equal(y1, y2) and np.array_equal(y1, y3)


def test_invalid_device_csr_rejected():
    cg = cg_mod()
    A = fi.laplace7(4)
    rp, ci, va = dev_csr(A)
    ci[3] = A.n  # out of range
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(rp, ci, va)
    assert e.value.status == cg.CG_EINVAL


def test_rows_longer_than_the_ring():
    """Rows of 8193 .. 39000 entries (longer than a chunk, some longer than the
    whole shared-memory ring) next to short rows; integer data -> exact."""
    A = fi.random_csr(40000, 3, 0, 20, empty_frac=0.1, long_rows=(17000, 30000, 39000, 8193, 8192), integer=True)
    x = np.round(fi.uniform(3, 5, A.n, -9, 9))
    with handle(A) as h:
        y = gpu_spmv(h, x)
        y2 = gpu_spmv(h, x)
    assert np.array_equal(y, oracle.spmv(A, x))
    assert np.array_equal(y, y2)
