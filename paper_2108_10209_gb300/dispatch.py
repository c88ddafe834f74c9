"""Host-side multi-GPU logic. Noise2Fast jobs are independent images, so several GPUs are used
by giving each rank (one process per GPU) its own share of the images; no tensor of a job ever
crosses GPUs. The only collective is the reduction of the timing over ranks."""
from __future__ import annotations

import heapq


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` out of `world` ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return [it for i, it in enumerate(items) if i % world == rank]


def aggregate(local_seconds: float, local_images: int, group=None):
    """(max seconds over ranks, images over all ranks) via torch.distributed (any backend).
    With no process group initialised, the local values are returned."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_seconds), int(local_images)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    n = torch.tensor([float(local_images)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(n, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), int(round(n.item()))


class LeastLoaded:
    """Assigns arriving jobs to the GPU with the least outstanding work (pixels x expected
    epochs); ties go to the lowest index. `done` returns a job's work to its GPU."""

    def __init__(self, n_gpus: int):
        self.load = [0.0] * n_gpus
        self.heap = [(0.0, g) for g in range(n_gpus)]
        self.where = {}

    def assign(self, job_id, work: float) -> int:
        while True:
            load, g = heapq.heappop(self.heap)
            if load == self.load[g]:
                break
        self.load[g] += work
        heapq.heappush(self.heap, (self.load[g], g))
        self.where[job_id] = (g, work)
        return g

    def done(self, job_id):
        g, work = self.where.pop(job_id)
        self.load[g] -= work
        heapq.heappush(self.heap, (self.load[g], g))
        return g


class MultiContext:
    """Serving front end over several GPUs in one process: one library context per device (each
    with its own scheduler, HBM budget and slots), every arriving image assigned on arrival to
    the device with the least outstanding work (LeastLoaded; work = pixels x planes, the
    per-epoch cost; the epochs a job will take are not known in advance), its status, history
    and result fetched from that device. A job's work is returned to its device once a final
    state is seen (poll, wait or result). Images are independent, so no data crosses devices.

    make_context(device) builds a context object with the methods of n2f.Context (submit,
    submit_u16, poll, wait, result, history, cancel, close); the default builds n2f.Context
    with **ctx_kw."""

    FINAL = (2, 3, 4)  # N2F_DONE, N2F_FAILED, N2F_CANCELED

    def __init__(self, devices, make_context=None, **ctx_kw):
        if not devices:
            raise ValueError("at least one device")
        if make_context is None:
            from . import n2f

            def make_context(dev):
                return n2f.Context(device=dev, **ctx_kw)
        self.devices = list(devices)
        self.ctxs = [make_context(d) for d in self.devices]
        self.sched = LeastLoaded(len(self.devices))
        self.jobs = {}  # front-end id -> (context index, the context's job id)
        self.next_id = 1

    def _add(self, work, submit):
        jid = self.next_id
        g = self.sched.assign(jid, float(work))
        try:
            cid = submit(self.ctxs[g])
        except Exception:
            self.sched.done(jid)
            raise
        self.next_id += 1
        self.jobs[jid] = (g, cid)
        return jid

    @staticmethod
    def _work(shape):
        n = 1
        for s in shape:
            n *= int(s)
        return n

    def submit(self, image, p=None) -> int:
        return self._add(self._work(image.shape), lambda c: c.submit(image, p))

    def submit_u16(self, image, p=None) -> int:
        return self._add(self._work(image.shape), lambda c: c.submit_u16(image, p))

    def device_of(self, jid) -> int:
        return self.devices[self.jobs[jid][0]]

    def _release(self, jid):
        if jid in self.sched.where:
            self.sched.done(jid)

    def poll(self, jid):
        g, cid = self.jobs[jid]
        st = self.ctxs[g].poll(cid)
        if st.state in self.FINAL:
            self._release(jid)
        return st

    def wait(self, jid, timeout_ms: int = -1) -> int:
        g, cid = self.jobs[jid]
        rc = self.ctxs[g].wait(cid, timeout_ms)
        if rc == 0:
            self._release(jid)
        return rc

    def result(self, jid, shape):
        """The job's output; the job is released from its device and this front end unless the
        call failed with EAGAIN (still running) or EINVAL (a wrong size: nothing released)."""
        g, cid = self.jobs[jid]
        try:
            out = self.ctxs[g].result(cid, shape)
        except Exception as e:
            if getattr(e, "code", None) not in (-3, -1):  # N2F_EAGAIN, N2F_EINVAL
                self._forget(jid)
            raise
        self._forget(jid)
        return out

    def _forget(self, jid):
        self._release(jid)
        self.jobs.pop(jid, None)

    def history(self, jid):
        g, cid = self.jobs[jid]
        return self.ctxs[g].history(cid)

    def cancel(self, jid) -> int:
        g, cid = self.jobs[jid]
        return self.ctxs[g].cancel(cid)

    def load(self):
        """Outstanding work per device, in the order of `devices`."""
        return list(self.sched.load)

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
