"""Dot product, vector addition and element-wise product on the GPU against the oracle."""
import math

import numpy as np
import pytest

import fe_inputs as fi
import oracle
from gpu_util import cg_mod, handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    with handle(fi.laplace7(4)) as hh:
        yield hh


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()


# paper sizes (Sec. 5.2 tables): 1e4, 2e6, 5e6 for the vector ops; 101,168 .. 1,587,808 for dot
@pytest.mark.parametrize("n", [0, 1, 7, 10_000, 101_168, 1_587_808, 5_000_000])
def test_dot(h, n):
    import torch
    cg = cg_mod()
    x, y = fi.uniform(n + 1, 1, n), fi.uniform(n + 1, 2, n)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    cg.cg_dot(h, _cuda(x), _cuda(y), out, n=n)
    got = out.item()
    ref = oracle.dot(x, y)
    scale = float(np.sum(np.abs(x * y)))
    # both are within (terms per partial sum + tree depth) * u * sum|x y| of the exact value
    assert abs(got - ref) <= 1e-12 * max(scale, 1e-300) + (0.0 if n else 0.0)
    if n:
        exact = math.fsum((x * y).tolist())
        assert abs(got - exact) <= 1e-12 * scale
    # deterministic: same bits on a second call
    out2 = torch.zeros_like(out)
    cg.cg_dot(h, _cuda(x), _cuda(y), out2, n=n)
    assert out2.item() == got
    # the host-result call runs the same kernel: the same bits
    assert cg.cg_dot_host(h, _cuda(x), _cuda(y), n=n) == got


def test_dot_integers_exact(h):
    import torch
    cg = cg_mod()
    n = 3_000_001
    x = np.round(fi.uniform(5, 1, n, -1000, 1000))
    y = np.round(fi.uniform(5, 2, n, -1000, 1000))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cg.cg_dot(h, _cuda(x), _cuda(y), out)
    assert out.item() == float(np.sum(x.astype(np.int64) * y.astype(np.int64)))


@pytest.mark.parametrize("n", [1, 3, 10_000, 2_000_000, 5_000_000])
@pytest.mark.parametrize("offset", [0, 1])
def test_axpy(h, n, offset):
    """offset 1 makes the vectors 8-byte but not 16-byte aligned (scalar path)."""
    import torch
    cg = cg_mod()
    a = -0.731
    x, y = fi.uniform(n, 3, n + 1), fi.uniform(n, 4, n + 1)
    xd, yd = _cuda(x), _cuda(y)
    cg.cg_axpy(h, a, xd[offset:], yd[offset:], n=n)
    got = yd.cpu().numpy()
    ref = oracle.axpy(a, x[offset:offset + n], y[offset:offset + n])
    # FMA (one rounding) against a*x + y (two roundings)
    tol = 2 * 2.0 ** -53 * (np.abs(a * x[offset:offset + n]) + np.abs(y[offset:offset + n]))
    assert np.all(np.abs(got[offset:offset + n] - ref) <= tol)
    assert np.array_equal(got[:offset], y[:offset])           # untouched outside the range
    assert np.array_equal(got[offset + n:], y[offset + n:])


def test_axpy_integers_exact(h):
    cg = cg_mod()
    n = 1_000_003
    x, y = np.round(fi.uniform(1, 1, n, -99, 99)), np.round(fi.uniform(1, 2, n, -99, 99))
    yd = _cuda(y)
    cg.cg_axpy(h, 3.0, _cuda(x), yd)
    assert np.array_equal(yd.cpu().numpy(), 3.0 * x + y)


@pytest.mark.parametrize("n", [1, 5, 10_000, 2_000_000, 5_000_000])
@pytest.mark.parametrize("offset", [0, 1])
def test_ewmul(h, n, offset):
    import torch
    cg = cg_mod()
    x, y = fi.uniform(n, 5, n + 1), fi.uniform(n, 6, n + 1)
    z = torch.full((n + 1,), 7.0, dtype=torch.float64, device="cuda")
    cg.cg_ewmul(h, _cuda(x)[offset:], _cuda(y)[offset:], z[offset:], n=n)
    got = z.cpu().numpy()
    # a single rounded product: bitwise equal to the oracle
    assert np.array_equal(got[offset:offset + n], oracle.ewmul(x[offset:offset + n], y[offset:offset + n]))


def test_ewmul_in_place(h):
    cg = cg_mod()
    x = fi.uniform(1, 1, 1001)
    xd = _cuda(x)
    cg.cg_ewmul(h, xd, xd, xd)
    assert np.array_equal(xd.cpu().numpy(), x * x)
