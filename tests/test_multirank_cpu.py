"""The N > 1 host path of bench.py on CPU: two gloo ranks.

Ranks run replicas of the evaluation on their own positions; only the
elapsed time (max over ranks) and the work (sum over ranks) are exchanged.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [3.0, 5.0][rank]
        units = [100.0, 250.0][rank]
        t, u = bench.aggregate_over_ranks(elapsed, units, dist)
        seeds = {bench.rank_seed(rank, s) for s in range(4)}
        q.put((rank, t, u, sorted(seeds)))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_distinct_inputs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, u, _ in out:
        assert t == 5.0 and u == 350.0
    assert not set(out[0][3]) & set(out[1][3])  # ranks never evaluate the same positions


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_over_ranks(2.5, 7, None) == (2.5, 7.0)
