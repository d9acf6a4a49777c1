"""The multi-GPU path of bench.py is replicas only (one independent problem
sequence per rank, no collective on the data path): its host logic, the
process group, the barriers around the timed region and the maximum of the
ranks' times, run here as two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), RK_BENCH_BACKEND="gloo")
    import bench
    import torch.distributed as dist
    w, r, loc = bench.dist_init()
    bench.barrier(w)
    t = bench.max_over_ranks(w, 1.5 * (r + 1))
    bench.barrier(w)
    q.put((r, w, loc, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == ws for o in out)
    assert all(o[3] == 3.0 for o in out)  # every rank sees the slowest rank's time


def test_replicas_solve_different_sequences():
    """Weak scaling: rank r > 0 draws its right-hand sides from its own seed,
    so the replicas are independent problems of the same shape."""
    import numpy as np
    from problems import make_config
    a = make_config(1, size=6)
    b = make_config(1, size=6, seed=20150113 + 1 + 1000 * 1)
    assert a.coef.shape == b.coef.shape and not np.array_equal(a.rhs(0), b.rhs(0))


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(workload="channel128", precond="subdomain", steps=1, warmup=3, gpus=2)
    bench.run_reference(args, 2, 1)  # rank 1: no work, no output
    assert capsys.readouterr().out == ""
