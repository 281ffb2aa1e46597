"""Multi-process replica logic of the benchmark, on CPU with the gloo backend.

The path does not shard a system across GPUs: with N processes every rank
solves its own independently seeded system and the job's rate is all ranks'
solves over the slowest rank's time.  These tests run that host logic with
two gloo ranks (no GPU): distinct systems per rank, the max-over-ranks time,
and the whole-job rate; each rank's solve is the oracle's, as a stand-in for
the device solve, so that the replicas' results can be checked too.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import fe_inputs as fi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    import oracle

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    seed = bench.replica_seed(7, rank)
    A = fi.q1(4, 1.0, seed)
    xs = fi.xstar(seed, A.n)
    b = oracle.spmv(A, xs)
    res = oracle.cg(A, b, tol=1e-10, maxit=10 * A.n)
    dist.barrier()
    t_local = 1.0 + rank          # rank r "took" 1 + r seconds
    t_max = bench.max_over_ranks(t_local, dist, torch.device("cpu"))
    rate = bench.whole_job_rate(10, world, t_max)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), b=b, x=res.x, xs=xs, status=res.status,
             relres=res.relres_true, t_max=t_max, rate=rate)
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    # every rank solved its own system
    assert not np.array_equal(out[0]["b"], out[1]["b"])
    for o in out:
        assert int(o["status"]) == 0 and float(o["relres"]) <= 1e-10
        assert np.linalg.norm(o["x"] - o["xs"]) <= 1e-6 * np.linalg.norm(o["xs"])
        # the slowest rank's time, and all ranks' solves over it
        assert float(o["t_max"]) == 2.0
        assert float(o["rate"]) == pytest.approx(10 * world / 2.0)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.whole_job_rate(20, 1, 4.0) == 5.0
    assert bench.replica_seed(3, 0) == 3 and bench.replica_seed(3, 1) == 4
