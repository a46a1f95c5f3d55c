"""The N > 1 path of bench.py on CPU: two gloo ranks check that each rank gets its own
disorder realisation (weak scaling, no data-path collective) and that the reported
time is the max over ranks of the timed region."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import numpy as np
    import torch.distributed as dist

    import bench
    import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_env()
        seed = bench.rank_seed(bench.CFG["seed"], r)
        h = wl.fields(bench.CFG["L"], bench.CFG["W"], seed)
        t_local = 1.0 + 0.5 * r  # rank 1 is the slow one
        t_max = bench.reduce_max(t_local, dist, "cpu")
        rate = bench.whole_job_rate(16 * 5, w, t_max)
        # gather what each rank saw (test plumbing only)
        got = [None] * world
        dist.all_gather_object(got, dict(w=w, r=r, lr=lr, seed=seed, h=h.tolist(), t_max=t_max, rate=rate))
        if r == 0:
            out.put(got)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    import bench
    assert [g["r"] for g in got] == [0, 1] and all(g["w"] == 2 for g in got)
    assert got[0]["seed"] == bench.CFG["seed"]  # rank 0 runs the named workload itself
    assert got[0]["seed"] != got[1]["seed"] and got[0]["h"] != got[1]["h"]
    assert all(g["t_max"] == pytest.approx(1.5) for g in got)  # the slowest rank sets the time
    assert all(g["rate"] == pytest.approx(2 * 16 * 5 / 1.5) for g in got)


def test_single_rank_helpers_without_process_group():
    import bench
    assert bench.reduce_max(3.25) == 3.25
    assert bench.rank_seed(1, 0) == 1
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
