"""cg_dot_noalloc: the dot product for callers that cannot allocate GPU memory.

Some callers cannot call cudaMalloc when they need a result: code that runs
under a fixed memory budget with no allocation after start-up, code called
from inside another allocator, or latency-critical loops that cannot take
cudaMalloc's device synchronisation.  cg_dot allocates its scratch on its first
call for each stream; cg_dot_noalloc takes raw device pointers and keeps its
scratch in a fixed array inside the library.  These tests call it through the C ABI and
compare it with cg_dot on two calls in a row.  The file is named to be
collected last, so a run stopping at the first failure has run everything
else first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import fe_inputs as fi
from gpu_util import cg_mod

pytestmark = pytest.mark.gpu

MAX_N = 16384 * 256 * 8  # capacity of the fixed scratch, in elements


def _cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()


@pytest.mark.parametrize("n", [1, 1000, 101_168, 1_587_808, 5_000_000])
def test_noalloc_matches_cg_dot_twice(n):
    import torch
    cg = cg_mod()
    x, y = fi.uniform(n, 11, n), fi.uniform(n, 12, n)
    xd, yd = _cuda(x), _cuda(y)
    scale = float(np.sum(np.abs(x * y)))
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    cg.cg_dot(xd, yd, ref)
    torch.cuda.synchronize()
    got = []
    for _ in range(2):  # two calls in a row share (and must clean) the scratch
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        cg.cg_dot_noalloc(xd, yd, out)
        torch.cuda.synchronize()
        got.append(out.item())
    for g in got:
        assert abs(g - ref.item()) <= 1e-12 * scale
    assert got[0] == got[1]  # deterministic


def test_noalloc_empty_and_capacity():
    import torch
    cg = cg_mod()
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    cg.cg_dot_noalloc(z, z, out, n=0)
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # beyond the fixed scratch: refused before any work, with a message
    rc = cg.lib.cg_dot_noalloc(MAX_N + 1, z.data_ptr(), z.data_ptr(), out.data_ptr(), None)
    assert rc == cg.CG_EINVAL
    assert "exceeds" in cg.last_error()
