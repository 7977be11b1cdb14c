"""Host-side sharding over ranks (one GPU per rank).

The despeckling path has no exchange between images, so a multi-GPU run
splits the batch and needs no collective on the data path; the only
collective of inference is the timing reduction of the benchmark.  Data-
parallel training (Sec. 3.2, the loss of Eq. learning summed over samples)
has one real exchange per step: the sum of the ranks' parameter gradients
(allreduce_gradients).  One image too large for one GPU splits into row
bands (band_rows) that need no exchange either: each rank runs the whole
cascade on its band plus 2R T ghost rows per side.
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


def band_rows(H: int, world: int, rank: int, ksize: int, T: int):
    """Row band of an H-row image for rank `rank` of `world`.

    Returns (own0, own1, g0, g1): the rank owns rows [own0, own1) (contiguous,
    sizes differing by at most one) and computes rows [g0, g1), its band plus
    2R T ghost rows on each side, clamped to the image (R = ksize // 2).  One
    stage of Eq. diffusionprocessfinal reads u_{t-1} at most 2R rows away (K,
    then K^T), and a band's cut edge acts as a symmetric border that is wrong
    only within 2R rows of the cut; after T stages the wrong rows reach 2R T
    rows in, all of them ghosts.  So every owned row comes out exactly as from
    the whole image, with no exchange between ranks during the cascade.
    """
    if world < 1 or not (0 <= rank < world) or H < 1 or ksize < 1 or T < 0:
        raise ValueError("bad band request")
    base, extra = divmod(H, world)
    own0 = rank * base + min(rank, extra)
    own1 = own0 + base + (1 if rank < extra else 0)
    ghost = 2 * (ksize // 2) * T
    return own0, own1, max(0, own0 - ghost), min(H, own1 + ghost)


def gather_bands(rows, H: int, group=None):
    """Assembles the ranks' owned rows (this rank's `rows`, [own1 - own0][W],
    band_rows order) into the whole image on every rank (one all_gather of
    equal-size padded bands)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return rows
    world = dist.get_world_size(group)
    cap = -(-H // world)
    pad = torch.zeros((cap,) + tuple(rows.shape[1:]), dtype=rows.dtype, device=rows.device)
    pad[:rows.shape[0]] = rows
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    base, extra = divmod(H, world)
    return torch.cat([parts[r][:base + (1 if r < extra else 0)] for r in range(world)])


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


def allreduce_gradients(tensors, group=None) -> None:
    """Sums the .grad of every tensor over the ranks, in place (one flat
    all-reduce of T (N_k k^2 + N_k N_rbf + 1) values).  With each rank's loss
    summing its own samples, the result is the gradient of the whole batch's
    loss, identical on every rank.  No-op without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return
    grads = [t.grad for t in tensors if t.grad is not None]
    if not grads:
        return
    flat = torch.cat([g.reshape(-1) for g in grads])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for g in grads:
        n = g.numel()
        g.copy_(flat[off:off + n].view_as(g))
        off += n
