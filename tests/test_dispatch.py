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


class _FakeStatus:
    def __init__(self, state):
        self.state = state


class _FakeError(RuntimeError):
    def __init__(self, code):
        super().__init__(code)
        self.code = code


class _FakeCtx:
    """Stands in for n2f.Context on one device: jobs finish when the test says so."""

    def __init__(self, dev):
        self.dev, self.next, self.state, self.closed = dev, 100 * (dev + 1), {}, False
        self.cancelled = []

    def submit(self, image, p=None):
        self.next += 1
        self.state[self.next] = 1  # RUNNING
        return self.next

    submit_u16 = submit

    def poll(self, cid):
        if cid not in self.state:
            raise _FakeError(-4)
        return _FakeStatus(self.state[cid])

    def wait(self, cid, timeout_ms=-1):
        return 0 if self.state[cid] >= 2 else -5

    def result(self, cid, shape):
        if self.state[cid] < 2:
            raise _FakeError(-3)
        del self.state[cid]
        return ("out", self.dev, cid, shape)

    def history(self, cid):
        return [0.5], 1

    def cancel(self, cid):
        self.cancelled.append(cid)
        return 0

    def close(self):
        self.closed = True


def test_multi_context_assigns_by_pixels_and_releases_on_completion():
    import numpy as np
    ctxs = {}

    def make(dev):
        ctxs[dev] = _FakeCtx(dev)
        return ctxs[dev]

    m = dispatch.MultiContext([3, 5], make_context=make)
    big, small = np.zeros((64, 64)), np.zeros((16, 16))
    a = m.submit(big)            # 4096 px -> device 3
    b = m.submit(small)          # device 5 (0 < 4096)
    c = m.submit(small)          # device 5 (256 < 4096)
    d = m.submit_u16(big)        # device 5 (512 < 4096)
    assert [m.device_of(j) for j in (a, b, c, d)] == [3, 5, 5, 5]
    assert m.load() == [4096.0, 4608.0]
    # not finished: a result is refused and nothing is released
    with pytest.raises(_FakeError):
        m.result(a, big.shape)
    assert m.load() == [4096.0, 4608.0] and m.history(b) == ([0.5], 1)
    # device 3's job finishes: the poll that sees it final returns its work
    g, cid = m.jobs[a]
    ctxs[3].state[cid] = 2
    assert m.poll(a).state == 2 and m.load() == [0.0, 4608.0]
    assert m.result(a, big.shape)[:2] == ("out", 3)
    assert a not in m.jobs
    e = m.submit(big)            # device 3 is the lighter one again
    assert m.device_of(e) == 3
    # a cancel goes to the job's own device; a failed result releases the job
    assert m.cancel(c) == 0 and ctxs[5].cancelled == [m.jobs[c][1]]
    ctxs[5].state[m.jobs[c][1]] = 4
    assert m.wait(c) == 0 and m.load() == [4096.0, 4352.0]
    m.close()
    assert ctxs[3].closed and ctxs[5].closed


def test_multi_context_submit_failure_returns_the_work():
    class Refusing(_FakeCtx):
        def submit(self, image, p=None):
            raise _FakeError(-2)

    import numpy as np
    m = dispatch.MultiContext([0], make_context=Refusing)
    with pytest.raises(_FakeError):
        m.submit(np.zeros((8, 8)))
    assert m.load() == [0.0] and not m.jobs
    with pytest.raises(ValueError):
        dispatch.MultiContext([], make_context=Refusing)
