"""bench.py's multi-rank plumbing on CPU (gloo, world size 2): each rank
solves its own instance (replicas), the job value is all ranks' units over
the slowest rank's time; the reference arm runs on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "CPMDP_BENCH_BACKEND": "gloo"})
    import bench
    r, w, local, pg = bench.dist_setup(world)
    assert (r, w, local) == (rank, world, rank)
    units, ms = bench.aggregate(pg, 1000.0 * (rank + 1), 10.0 + 5.0 * rank)
    out.put((rank, units, ms))
    pg.barrier()
    pg.destroy_process_group()


def test_aggregate_sum_units_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, units, ms in res:
        assert units == 3000.0 and ms == 15.0


def test_reference_arm_other_ranks_do_nothing():
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) == 0


def test_small_case_cpu_oracles_report():
    """The 10 x 10 CPU-oracle timings bench.py reports beside the GPU solve:
    every field present and positive, the one-core run restores the
    oracle's thread count."""
    import bench
    from oracle import cpfactor as oc
    oc.build()
    before = oc.threads()
    out = bench.small_10x10_cpu(reps=1)
    for k in ("tabular_vi_ms", "tabular_pi_ms", "cp_factor_vi_ms", "cp_factor_vi_ms_one_core"):
        assert out[k] > 0
    assert out["cp_factor_threads"] == before == oc.threads()
