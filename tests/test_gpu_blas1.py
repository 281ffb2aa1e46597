"""Dot product, vector addition and element-wise product on the GPU against
the oracle, through the handle-free calls of the C ABI."""
import math

import numpy as np
import pytest

import fe_inputs as fi
import oracle
from gpu_util import cg_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    """The vector calls take no handle; the fixture only keeps the tests' signatures."""
    return None


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()


# paper sizes (Sec. 5.2 tables): 1e4, 2e6, 5e6 for the vector ops; 101,168 .. 1,587,808 for dot; around the
# streamed kernel's threshold (32768) and its chunk (2048), a ragged tail past the last whole chunk, and the
# benchmark's 6.4e7
@pytest.mark.parametrize("n", [0, 1, 7, 10_000, 32_767, 32_768, 32_768 + 2047, 101_168, 1_587_808, 5_000_000,
                               64_000_000])
def test_dot(h, n):
    import torch
    cg = cg_mod()
    x, y = fi.uniform(n + 1, 1, n), fi.uniform(n + 1, 2, n)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    cg.cg_dot(_cuda(x), _cuda(y), out, n=n)
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
    cg.cg_dot(_cuda(x), _cuda(y), out2, n=n)
    assert out2.item() == got
    # the host-result call runs the same kernel: the same bits
    assert cg.cg_dot_host(_cuda(x), _cuda(y), n=n) == got


def test_dot_integers_exact(h):
    import torch
    cg = cg_mod()
    n = 3_000_001
    x = np.round(fi.uniform(5, 1, n, -1000, 1000))
    y = np.round(fi.uniform(5, 2, n, -1000, 1000))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cg.cg_dot(_cuda(x), _cuda(y), out)
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
    cg.cg_axpy(a, xd[offset:], yd[offset:], n=n)
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
    cg.cg_axpy(3.0, _cuda(x), yd)
    assert np.array_equal(yd.cpu().numpy(), 3.0 * x + y)


@pytest.mark.parametrize("n", [1, 5, 10_000, 2_000_000, 5_000_000])
@pytest.mark.parametrize("offset", [0, 1])
def test_ewmul(h, n, offset):
    import torch
    cg = cg_mod()
    x, y = fi.uniform(n, 5, n + 1), fi.uniform(n, 6, n + 1)
    z = torch.full((n + 1,), 7.0, dtype=torch.float64, device="cuda")
    cg.cg_ewmul(_cuda(x)[offset:], _cuda(y)[offset:], z[offset:], n=n)
    got = z.cpu().numpy()
    # a single rounded product: bitwise equal to the oracle
    assert np.array_equal(got[offset:offset + n], oracle.ewmul(x[offset:offset + n], y[offset:offset + n]))


def test_ewmul_in_place(h):
    cg = cg_mod()
    x = fi.uniform(1, 1, 1001)
    xd = _cuda(x)
    cg.cg_ewmul(xd, xd, xd)
    assert np.array_equal(xd.cpu().numpy(), x * x)


@pytest.mark.parametrize("n", [40_000, 3_000_001])
def test_dot_unaligned_falls_back_within_tolerance(n):
    """x and y 8-byte but not 16-byte aligned take the grid-stride kernel: the
    same sum within the rounding bound, deterministic."""
    import torch
    cg = cg_mod()
    x, y = fi.uniform(n, 31, n + 1), fi.uniform(n, 32, n + 1)
    xd, yd = _cuda(x), _cuda(y)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    cg.cg_dot(xd[1:], yd[1:], out[0:1], n=n)
    cg.cg_dot(xd[1:], yd[1:], out[1:2], n=n)
    ref = oracle.dot(x[1:], y[1:])
    scale = float(np.sum(np.abs(x[1:] * y[1:])))
    got = out.cpu().numpy()
    assert got[0] == got[1]
    assert abs(got[0] - ref) <= 1e-12 * scale


def test_blas1_on_a_side_stream_and_release():
    """The calls queue on the given stream; per-stream scratch; release frees it
    and the next call allocates again."""
    import torch
    cg = cg_mod()
    n = 2_000_003
    x, y = fi.uniform(9, 1, n), fi.uniform(9, 2, n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xd, yd = _cuda(x), _cuda(y)
        zd = torch.empty_like(xd)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cg.cg_dot(xd, yd, out, stream=s)
    cg.cg_ewmul(xd, yd, zd, stream=s)
    cg.cg_axpy(2.0, xd, zd, stream=s)
    s.synchronize()
    assert abs(out.item() - oracle.dot(x, y)) <= 1e-12 * float(np.sum(np.abs(x * y)))
    # z = x*y (one rounding, bitwise the oracle's), then z += 2x with one FMA
    # against the oracle's two roundings
    want = oracle.axpy(2.0, x, oracle.ewmul(x, y))
    assert np.all(np.abs(zd.cpu().numpy() - want) <= 2 * 2.0 ** -53 * (2 * np.abs(x) + np.abs(x * y)))
    v1 = cg.cg_dot_host(xd, yd, stream=s)
    cg.cg_blas_release()
    v2 = cg.cg_dot_host(xd, yd, stream=s)
    assert v1 == v2 == out.item()


def test_fp64_peak_probe():
    """The probe reports a positive rate below the FP64 issue limit of the
    device (2 FMAs per SM per clock at the maximum SM clock, with margin)."""
    import torch
    cg = cg_mod()
    g = cg.cg_probe_fp64_peak(torch.cuda.current_device())
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    assert 0 < g
    assert g <= 2 * 2 * props.multi_processor_count * 2.2e9 / 1e9 * 1.5


def test_dot_on_the_per_thread_default_stream_from_two_threads():
    """cudaStreamPerThread (handle value 2) names a different stream in every
    host thread; each thread gets its own scratch, so concurrent dot products
    on it from two threads give their own correct sums."""
    import threading
    import torch
    cg = cg_mod()
    n = 3_000_000
    data = [(fi.uniform(40 + t, 1, n), fi.uniform(40 + t, 2, n)) for t in range(2)]
    dev = [(_cuda(x), _cuda(y)) for x, y in data]
    torch.cuda.synchronize()
    got = [[], []]

    def work(t):
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(20):
            got[t].append(cg.cg_dot_host(dev[t][0], dev[t][1], stream=2))
        cg.cg_dot(dev[t][0], dev[t][1], out, stream=2)
        torch.cuda.synchronize()
        got[t].append(out.item())

    th = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for t, (x, y) in enumerate(data):
        ref = oracle.dot(x, y)
        assert len(got[t]) == 21 and len(set(got[t])) == 1, set(got[t])
        assert abs(got[t][0] - ref) <= 1e-12 * float(np.sum(np.abs(x * y)))
