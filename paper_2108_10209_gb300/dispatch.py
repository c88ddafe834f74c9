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
