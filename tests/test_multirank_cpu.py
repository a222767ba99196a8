"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2).

The method shards only by independent problems: every rank evaluates its
own meshes (or a replica of the workload) and the only collectives are the
timing's max over ranks, the sum of the points processed and the broadcast
of the autotuned configuration.  These helpers are exercised here with two
gloo ranks; the GPU data path itself has no collective.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + rank, device="cpu")
        choice = bench.broadcast_choice({"p": 8, "leaf_size": 128} if rank == 0 else None)
        t = torch.tensor([100.0 * (rank + 1)], dtype=torch.float64)
        dist.all_reduce(t)
        out.put((rank, slowest, choice, float(t.item())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing_and_choice():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, choice, total in res:
        assert slowest == 11.0                       # max over ranks
        assert choice == {"p": 8, "leaf_size": 128}  # rank 0's pick everywhere
        assert total == 300.0                        # points summed over ranks


def test_shard_by_work_covers_and_balances():
    import bench
    rng = np.random.default_rng(0)
    work = rng.choice([3072, 6260, 21888, 33140, 121344, 140660], size=64)
    for world in (1, 2, 4, 8):
        parts = bench.shard_by_work(work, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))                          # every mesh exactly once
        loads = [work[p].sum() for p in map(np.array, parts)]
        assert max(loads) - min(loads) <= work.max()            # longest-first bound
    assert bench.max_over_ranks(3.5, device="cpu") == 3.5       # one rank: unchanged
    assert bench.broadcast_choice({"a": 1}) == {"a": 1}
