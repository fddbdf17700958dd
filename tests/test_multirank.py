"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
each rank draws its own batch from a disjoint seed range (no data-path
collective), the job time is the maximum over ranks, and the whole-job rate
is all ranks' units over that time."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        rhs = 3
        pb = wl.varcoef_random_rhs(n=1, W=2, n_rhs=rhs, seed0=bench.shard_seed0(rank, rhs))
        x = np.linspace(0.1, 0.9, 4)
        f = np.stack([fr(x, x, x) for fr in pb.f])
        got = [None] * ws
        dist.all_gather_object(got, f)
        ms = bench.reduce_max_ms(10.0 + 5.0 * rank, ws, "cpu")
        rate = bench.weak_scaling_rate(ws, 1_000_000, ms)
        if rank == 0:
            out.put((got, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, ms, rate = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # disjoint shards: the ranks' right-hand sides differ, and rank 1's are the
    # ones a single rank would draw after rank 0's (seeds 20260 + 3 .. + 5)
    assert not np.allclose(got[0], got[1])
    ref = wl.varcoef_random_rhs(n=1, W=2, n_rhs=6, seed0=20260)
    x = np.linspace(0.1, 0.9, 4)
    np.testing.assert_allclose(got[1], np.stack([fr(x, x, x) for fr in ref.f[3:]]), rtol=0, atol=0)
    assert ms == 15.0
    assert rate == 2 * 1_000_000 / 15e-3 / 1e9
