"""Batched and served solves on the GPU, through the C ABI (cg_batch_*).

Every system of a batch is checked against the oracle like a single solve
(true residual <= tol, solution within 1e-8 of the oracle run for the same
number of steps, stopping step within max(2, 1%) of the oracle's).  The batch
machinery itself is checked by properties that hold for any correct runtime:
a system gives the same bits alone and in any mix, in one launch or over
many rounds (its state carried between launches), with one CTA or a group of
CTAs within tolerance of each other; admission respects the memory budget;
malformed and oversized requests are refused without disturbing the rest.
"""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
from gpu_util import cg_mod, hub_matrix, iters_close, kappa_estimate

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _system(N, seed, kind="q1"):
    A = fi.q1(N, 1.0, seed) if kind == "q1" else fi.laplace7(N)
    xs = fi.xstar(seed, A.n)
    b = oracle.spmv(A, xs)
    return A, b


def _request(A, b, host=True, tag=0, tol=TOL, maxit=None):
    import torch
    cg = cg_mod()
    if host:
        rp, ci, va = A.row_ptr.astype(np.int32), A.col_idx.astype(np.int32), A.val.astype(np.float64)
        bb, x = b.copy(), np.zeros(A.n)
    else:
        rp, ci, va = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col_idx, A.val))
        bb, x = torch.from_numpy(b).cuda(), torch.zeros(A.n, dtype=torch.float64, device="cuda")
    return cg.Request(rp, ci, va, bb, x, tol=tol, maxit=maxit, index_base=getattr(A, "index_base", 0), tag=tag)


def _wait_all(bt, tickets, limit_ms=120000):
    res = bt.wait_all(tickets, limit_ms)
    assert all(r.done for r in res), "a request did not finish within the limit"
    return res


def _wait1(bt, ticket, limit_ms=120000):
    return _wait_all(bt, [ticket], limit_ms)[0]


def _x(req):
    x = req.x
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def _check_vs_oracle(A, b, res, x):
    cg = cg_mod()
    assert res.done and res.status == cg.CG_OK, res
    assert res.relres <= TOL
    # the true residual recomputed by the oracle's product
    tr = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert tr <= 1.0000001 * TOL
    ref = oracle.cg(A, b, tol=TOL, maxit=10 * A.n)
    assert iters_close(res.iters, ref.iters), (res.iters, ref.iters)
    same = oracle.cg(A, b, tol=0.0, maxit=res.iters, force_iters=res.iters)
    assert np.linalg.norm(x - same.x) <= 1e-8 * np.linalg.norm(same.x)


def test_batch_matches_oracle_per_system():
    cg = cg_mod()
    systems = [_system(N, 10 + N) for N in (2, 3, 5, 8, 12)] + [_system(6, 0, "lap")]
    with cg.Batch() as bt:
        reqs = [_request(A, b, host=(i % 2 == 0), tag=i) for i, (A, b) in enumerate(systems)]
        tickets = bt.submit(reqs)
        results = _wait_all(bt, tickets)
        st = bt.stats()
    assert st["graph"] == 1, "rounds should replay a captured CUDA graph"
    # a few kB of vectors: the row pointers keep the default L2 policy
    assert st["rounds_stream_rows"] == 0
    for (A, b), req, res in zip(systems, reqs, results):
        assert res.tag == req.tag
        _check_vs_oracle(A, b, res, _x(req))


@pytest.mark.parametrize("validate", [True, False])
def test_one_based_input_from_host_and_device(validate):
    """One-based CSR (the paper's IA/JA/AA indexing) from host and from device
    memory, with and without the library's validation: rebased on admission,
    so the same bits as the zero-based request."""
    cg = cg_mod()
    A, b = _system(7, 31)
    B = fi.to_one_based(A)
    with cg.Batch(validate=validate) as bt:
        reqs = [_request(A, b, host=True), _request(B, b, host=True), _request(B, b, host=False)]
        res = _wait_all(bt, bt.submit(reqs))
    _check_vs_oracle(A, b, res[0], _x(reqs[0]))
    for k in (1, 2):
        assert res[k].status == cg.CG_OK and res[k].iters == res[0].iters, res[k]
        assert np.array_equal(_x(reqs[k]), _x(reqs[0]))


def test_alone_and_in_a_mix_give_the_same_bits():
    cg = cg_mod()
    A, b = _system(10, 77)
    others = [_system(N, 200 + N) for N in (4, 7, 9, 13, 6)]
    with cg.Batch() as bt:
        r_alone = _request(A, b)
        t = bt.submit([r_alone])[0]
        ra = _wait1(bt, t)
        mix = [_request(*s) for s in others[:2]] + [_request(A, b)] + [_request(*s) for s in others[2:]]
        tm = bt.submit(mix)
        rm = _wait_all(bt, tm)
    assert ra.status == cg.CG_OK and rm[2].status == cg.CG_OK
    assert ra.iters == rm[2].iters
    assert np.array_equal(_x(r_alone), _x(mix[2]))


def test_rounds_resume_exactly():
    """Advancing every system a few steps per launch (state saved and
    reloaded between launches) gives the bits of one launch per system."""
    cg = cg_mod()
    systems = [_system(N, 300 + N) for N in (5, 9, 11)]
    outs = {}
    for chunk in (0, 7):
        with cg.Batch(chunk_iters=chunk) as bt:
            reqs = [_request(A, b) for A, b in systems]
            res = _wait_all(bt, bt.submit(reqs))
            outs[chunk] = (reqs, res, bt.stats())
    (r0, s0, st0), (r7, s7, st7) = outs[0], outs[7]
    assert st7["rounds"] > st0["rounds"]
    for a, b_, ra, rb in zip(r0, r7, s0, s7):
        assert ra.status == rb.status == cg.CG_OK
        assert ra.iters == rb.iters
        assert rb.rounds >= ra.iters // 7
        assert np.array_equal(_x(a), _x(b_))


@pytest.mark.parametrize("group", [2, 5])
def test_groups_of_ctas(group):
    """A system shared by a group of CTAs (own group barrier, per-group sums)."""
    cg = cg_mod()
    systems = [_system(14, 400), _system(17, 401), _system(6, 402)]
    with cg.Batch(group_override=group) as bt:
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
    for (A, b), req, r in zip(systems, reqs, res):
        assert r.group == group
        _check_vs_oracle(A, b, r, _x(req))


def test_groups_with_chunks_resume_exactly():
    cg = cg_mod()
    A, b = _system(15, 500)
    xs = []
    for chunk in (0, 5):
        with cg.Batch(group_override=3, chunk_iters=chunk) as bt:
            req = _request(A, b)
            r = _wait1(bt, bt.submit([req])[0])
            assert r.status == cg.CG_OK
            xs.append((_x(req).copy(), r.iters))
    assert xs[0][1] == xs[1][1] and np.array_equal(xs[0][0], xs[1][0])


def test_budget_admission_and_release():
    """A budget that holds about two systems at a time: every request still
    completes, in rounds, and the arena never exceeds the budget."""
    cg = cg_mod()
    systems = [_system(12, 600 + i) for i in range(6)]
    A0 = systems[0][0]
    per = 12 * A0.nnz + 4 * A0.nnz + 80 * A0.n + 64 * 1024
    with cg.Batch(budget_bytes=int(2.2 * per), chunk_iters=20) as bt:
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
        st = bt.stats()
    assert st["bytes_peak"] <= st["budget_bytes"]
    assert st["bytes_in_use"] == 0 and st["resident"] == 0 and st["pending"] == 0
    for (A, b), req, r in zip(systems, reqs, res):
        _check_vs_oracle(A, b, r, _x(req))
    # admission waited for memory: some request was admitted after another finished
    assert max(r.admit_ms for r in res) >= min(r.done_ms for r in res)


def test_oversized_and_malformed_requests():
    cg = cg_mod()
    A, b = _system(8, 700)
    with cg.Batch(budget_bytes=1 << 20) as bt:
        big = _request(*_system(20, 701))
        with pytest.raises(cg.CGError) as e:
            bt.submit([big])
        assert e.value.status == cg.CG_ENOMEM
        bad = _request(A, b)
        bad.col_idx = bad.col_idx.copy()
        bad.col_idx[5] = A.n + 3          # column out of range
        good = _request(*_system(3, 702))
        t_bad, t_good = bt.submit([bad, good])
        r_bad, r_good = _wait1(bt, t_bad), _wait1(bt, t_good)
    assert r_bad.done and r_bad.status == cg.CG_EINVAL
    assert r_good.status == cg.CG_OK and r_good.relres <= TOL


def test_empty_system_and_zero_rhs():
    cg = cg_mod()
    A, _ = _system(4, 800)
    empty = fi.CSR(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), 0)
    with cg.Batch() as bt:
        r_empty = _request(empty, np.zeros(0))
        r_zero = _request(A, np.zeros(A.n))
        r_zero.x[:] = 5.0  # overwritten: x0 = 0 and b = 0 give x = 0
        res = _wait_all(bt, bt.submit([r_empty, r_zero]))
    assert res[0].status == cg.CG_OK and res[0].iters == 0
    assert res[1].status == cg.CG_OK and res[1].iters == 0 and np.all(_x(r_zero) == 0.0)


def test_mixed_precision_batch():
    cg = cg_mod()
    systems = [_system(N, 900 + N) for N in (6, 10, 16)]
    with cg.Batch(precision=cg.CG_PREC_MIXED) as bt:
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
    for (A, b), req, r in zip(systems, reqs, res):
        assert r.status == cg.CG_OK and r.relres <= TOL
        x = _x(req)
        assert np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b) <= 1.0000001 * TOL
        ref = oracle.cg_mixed(A, b, tol=TOL)
        assert ref.status == oracle.OK
        # both are within kappa * 1e-10 of the exact solution
        kap = kappa_estimate(A, b)
        assert np.linalg.norm(x - ref.x) <= 2.0 * kap * TOL * np.linalg.norm(ref.x)


def test_batch_of_256_uneven_systems_sampled():
    """The 256-system workload (edges uniform in [8, 48], own densities and
    right-hand side per system) in one batch: every system converges; a
    sample is checked against the oracle's product."""
    cg = cg_mod()
    edges = fi.batch_edges(0, 256)
    reqs, systems = [], []
    for i, N in enumerate(edges):
        sd = fi.system_seed(0, i)
        A = fi.q1(int(N), 1.0, sd)
        b = oracle.spmv(A, fi.xstar(sd, A.n))
        systems.append((A, b))
        reqs.append(_request(A, b, tag=i))
    with cg.Batch(precision=cg.CG_PREC_MIXED) as bt:
        res = _wait_all(bt, bt.submit(reqs))
        st = bt.stats()
    assert st["completed"] == 256
    assert all(r.status == cg.CG_OK and r.relres <= TOL for r in res)
    # p, q, r (FP64), the FP32 copy of p and the row pointers of the systems
    # of a round outgrow 4/7 of the L2: the row pointers are streamed
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    if 7 * 32 * sum(A.n for A, _ in systems) > 4 * l2:
        assert st["rounds_stream_rows"] >= 1, st
    assert st["rounds_stream_rows"] <= st["rounds"]
    for i in range(0, 256, 37):
        A, b = systems[i]
        x = _x(reqs[i])
        assert np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b) <= 1.0000001 * TOL


@pytest.mark.parametrize("group", [1, 3])
def test_batch_row_longer_than_the_ring(group):
    """A system with a row of 27,000 entries (longer than the 16,384-entry
    shared-memory ring) beside a Q1 system in one batch, on one CTA and on a
    group of three: every system matches the oracle at equal iterations."""
    cg = cg_mod()
    H = hub_matrix(30, 72)
    systems = [(H, oracle.spmv(H, fi.xstar(72, H.n))), _system(12, 73)]
    with cg.Batch(group_override=group) as bt:
        reqs = [_request(A, b, tag=i) for i, (A, b) in enumerate(systems)]
        res = _wait_all(bt, bt.submit(reqs))
    for (A, b), req, r in zip(systems, reqs, res):
        assert r.group == group
        _check_vs_oracle(A, b, r, _x(req))


def test_groups_beyond_one_wave():
    """More group ranks than the grid has CTAs: later groups are taken by
    CTAs that finish earlier group tasks (in one launch), and every system
    still matches the oracle."""
    cg = cg_mod()
    systems = [_system(13 + i, 1000 + i) for i in range(4)]
    with cg.Batch(group_override=100) as bt:
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
        st = bt.stats()
    assert st["rounds"] == 1
    for (A, b), req, r in zip(systems, reqs, res):
        assert r.group == min(100, st["nblocks"])
        _check_vs_oracle(A, b, r, _x(req))


@pytest.mark.parametrize("variant", ["fp64", "mixed_jacobi"])
def test_served_request_joins_running_rounds_with_the_same_bits(variant):
    """Continuous batching: a request submitted while other systems are part
    way through their solves (rounds of a few steps) is admitted at a later
    round, overlaps them on the device, and gives exactly the bits it gives
    when it runs alone."""
    import time
    cg = cg_mod()
    A, b = _system(11, 1200)
    others = [_system(N, 1210 + N) for N in (18, 20, 22)]
    opts = {} if variant == "fp64" else {"precision": cg.CG_PREC_MIXED, "preconditioner": cg.CG_PRECOND_JACOBI}
    with cg.Batch(chunk_iters=4, **opts) as bt:
        r_alone = _request(A, b)
        ra = _wait1(bt, bt.submit([r_alone])[0])
        r0 = bt.stats()["rounds"]
        reqs = [_request(*s) for s in others]
        tick = bt.submit(reqs)
        t0 = time.time()
        while bt.stats()["rounds"] < r0 + 3 and time.time() - t0 < 60:
            time.sleep(0.001)
        late = _request(A, b)
        tl = bt.submit([late])[0]
        res = _wait_all(bt, tick + [tl])
    rl = res[-1]
    assert ra.status == rl.status == cg.CG_OK
    assert rl.iters == ra.iters and np.array_equal(_x(r_alone), _x(late))
    # it joined while the others were running and finished among them
    assert rl.admit_ms > min(r.admit_ms for r in res[:-1])
    assert rl.admit_ms < max(r.done_ms for r in res[:-1])
    for (S, bs), req, r in zip(others, reqs, res[:-1]):
        if variant == "fp64":
            _check_vs_oracle(S, bs, r, _x(req))
        else:
            assert r.status == cg.CG_OK and r.relres <= TOL
            assert np.linalg.norm(bs - oracle.spmv(S, _x(req))) <= TOL * np.linalg.norm(bs) * 1.0000001


def test_autotuned_group_model():
    """The autotuner measures the group-size cost model on the GPU; the model
    is positive and self-consistent, a large system gets a larger group than
    a small one, and solves still match the oracle."""
    cg = cg_mod()
    with cg.Batch(autotune=True) as bt:
        st = bt.stats()
        assert st["autotuned"] == 1
        assert st["cta_bytes_per_s"] > 1e9 and st["group_cta_bytes_per_s"] > 1e9
        assert st["step_overhead_s"] >= 0 and st["group_step_overhead_s"] >= 0
        g_small = bt.group_for(fi.q1(8, 1.0, 1).row_ptr)
        g_big = bt.group_for(fi.q1(48, 1.0, 1).row_ptr)
        assert 1 <= g_small <= g_big <= st["nblocks"]
        systems = [_system(N, 1300 + N) for N in (6, 12)]
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
    for (A, b), req, r in zip(systems, reqs, res):
        _check_vs_oracle(A, b, r, _x(req))


def test_autotuned_step_shapes():
    """The autotuner also measures, for each bucket of row lengths, which step
    shape (one lane, two lanes or a warp per row) the product runs fastest
    with on this GPU.  The table holds only shapes the rows allow; systems
    solved with it match the oracle; a system gives the same bits alone and
    in a mix on the tuned object (the table depends on the object, not the mix)."""
    cg = cg_mod()
    with cg.Batch(autotune=True) as bt:
        st = bt.stats()
        assert st["shape_tuned"] == 1
        kinds = st["step_kind"]
        assert all(k in (0, 1) for k in kinds[:4]) and all(k in (1, 2) for k in kinds[4:]), kinds
        systems = [_system(N, 1500 + N) for N in (5, 9, 13)] + [_system(7, 1507, "lap7")]
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
        A1, b1 = systems[1]
        alone = _request(A1, b1)
        _wait1(bt, bt.submit([alone])[0])
    for (A, b), req, r in zip(systems, reqs, res):
        _check_vs_oracle(A, b, r, _x(req))
    assert np.array_equal(_x(alone), _x(reqs[1]))


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_forced_step_shapes(shape):
    """Every step shape (1: the built-in one lane per row up to 32 entries and
    two lanes up to 64; 2: two lanes per row; 3: a warp per row) solves Q1
    systems, a 7-point Laplacian and an irregular SPD system with rows of 14
    to 37 entries to the oracle's result at equal steps; the stats report the shape."""
    cg = cg_mod()
    irregular = fi.random_spd(300, 77, density=0.08)
    xs = fi.xstar(77, irregular.n)
    systems = [_system(6, 1601), _system(11, 1602), _system(9, 1603, "lap7"),
               (irregular, oracle.spmv(irregular, xs))]
    with cg.Batch(step_shape=shape, autotune=True) as bt:
        st = bt.stats()
        assert st["shape_tuned"] == 0
        want = {1: [0, 0, 0, 0, 1, 1], 2: [1] * 6, 3: [2] * 6}[shape]
        assert st["step_kind"] == want
        reqs = [_request(A, b) for A, b in systems]
        res = _wait_all(bt, bt.submit(reqs))
    for (A, b), req, r in zip(systems, reqs, res):
        _check_vs_oracle(A, b, r, _x(req))


def test_destroy_with_work_in_flight():
    """Destroying a batch object while requests are queued and running
    returns after the round in flight; a new batch object then works."""
    cg = cg_mod()
    systems = [_system(N, 1400 + N) for N in (10, 14, 18, 22)]
    bt = cg.Batch(chunk_iters=3, budget_bytes=64 << 20)
    reqs = [_request(A, b) for A, b in systems * 3]
    bt.submit(reqs)
    bt.close()
    A, b = systems[0]
    with cg.Batch() as bt2:
        r = _request(A, b)
        res = _wait1(bt2, bt2.submit([r])[0])
    _check_vs_oracle(A, b, res, _x(r))
