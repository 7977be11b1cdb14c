"""Host-side sharding of independent images over ranks (one GPU per rank).

The despeckling path has no exchange between images, so a multi-GPU run
splits the batch and needs no collective on the data path; the only
collective is the timing reduction of the benchmark.
"""
from __future__ import annotations


def shard_images(sizes, world: int, rank: int):
    """Indices of the images rank `rank` processes: greedy longest-first
    assignment by pixel count (deterministic: ties go to the lower rank)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += sizes[i][0] * sizes[i][1]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def global_rate(pixels_local: float, ms_local: float, group=None):
    """Whole-job Mpixel/s: all ranks' pixels over the slowest rank's time."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.tensor([float(pixels_local), float(ms_local)], dtype=torch.float64, device=dev)
        px = t[:1].clone()
        ms = t[1:].clone()
        dist.all_reduce(px, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(ms, op=dist.ReduceOp.MAX, group=group)
        return float(px[0]) / (float(ms[0]) / 1e3) / 1e6, float(ms[0])
    return pixels_local / (ms_local / 1e3) / 1e6, ms_local
