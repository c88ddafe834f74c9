"""Multi-GPU host logic on the CPU: images sharded over ranks, timings reduced over a gloo
process group (world size 2, two processes), and the least-loaded serving dispatcher."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2108_10209_gb300 import dispatch


def test_shard_partitions_items():
    items = list(range(11))
    parts = [dispatch.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert parts[0] == [0, 3, 6, 9] and parts[2] == [2, 5, 8]
    with pytest.raises(ValueError):
        dispatch.shard(items, 3, 3)


def test_least_loaded_balances_and_releases():
    d = dispatch.LeastLoaded(2)
    assert d.assign("a", 10.0) == 0
    assert d.assign("b", 3.0) == 1
    assert d.assign("c", 3.0) == 1      # GPU 1 still lighter (3 < 10)
    assert d.assign("d", 5.0) == 1      # 6 < 10
    assert d.assign("e", 1.0) == 0      # 11 > 10
    assert d.done("a") == 0
    assert d.assign("f", 2.0) == 0      # GPU 0 now holds 1
    assert d.load == [3.0, 11.0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = dispatch.shard(list(range(7)), rank, world)
    secs = 1.5 + rank  # rank 1 is the slower one
    tmax, n = dispatch.aggregate(secs, len(mine))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, tmax, n))


def test_two_rank_gloo_sharding_and_timing():
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
    (r0, m0, t0, n0), (r1, m1, t1, n1) = res
    assert sorted(m0 + m1) == list(range(7)) and not set(m0) & set(m1)
    assert t0 == t1 == 2.5          # the job's time is the slowest rank's
    assert n0 == n1 == 7            # images over all ranks


def test_aggregate_without_group_is_local():
    assert dispatch.aggregate(3.0, 4) == (3.0, 4)
