"""Multi-rank host logic on CPU (gloo, world size 2): image sharding and the
whole-job rate reduction that bench.py uses with one process per GPU."""
import dataclasses
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1702_07482_gb300.shard import global_rate, shard_images


def test_shard_partitions_and_balances():
    sizes = [(256 + 37 * i % 700, 300 + 53 * i % 650) for i in range(64)]
    for world in (1, 2, 3, 8):
        parts = [shard_images(sizes, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(sizes[i][0] * sizes[i][1] for i in p) for p in parts]
        biggest = max(h * w for h, w in sizes)
        assert max(loads) - min(loads) <= biggest
    with pytest.raises(ValueError):
        shard_images(sizes, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [(512, 512), (256, 1024), (300, 700), (1000, 260), (512, 300)]
    mine = shard_images(sizes, world, rank)
    px = sum(sizes[i][0] * sizes[i][1] for i in mine)
    ms = 10.0 + 5.0 * rank            # rank 1 is the slower one
    rate, ms_max = global_rate(px, ms)
    q.put((rank, sorted(mine), rate, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_rate_uses_all_pixels_and_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    total = 512 * 512 + 256 * 1024 + 300 * 700 + 1000 * 260 + 512 * 300
    assert sorted(out[0][1] + out[1][1]) == [0, 1, 2, 3, 4]
    for _, _, rate, ms_max in out:
        assert ms_max == 15.0
        assert rate == pytest.approx(total / 15e-3 / 1e6)


def _grad_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_1702_07482_gb300.shard import allreduce_gradients
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # three parameter tensors shaped as one 3x3x4, T = 2 model; rank-dependent gradients
    shapes = [(2, 4, 3, 3), (2, 4, 63), (2,)]
    ts = []
    for k, sh in enumerate(shapes):
        t = torch.zeros(sh, requires_grad=True)
        t.grad = torch.full(sh, float(rank + 1)) * (k + 1) + torch.arange(t.numel()).view(sh)
        ts.append(t)
    allreduce_gradients(ts)
    q.put((rank, [t.grad.clone() for t in ts]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gradient_allreduce_sums_and_agrees():
    """The data-parallel exchange of training: after allreduce_gradients every
    rank holds the sum of both ranks' gradients, bit for bit the same."""
    import torch
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shapes = [(2, 4, 3, 3), (2, 4, 63), (2,)]
    for k, sh in enumerate(shapes):
        n = int(np.prod(sh))
        want = (1 + 2) * (k + 1) + 2 * torch.arange(n).view(sh).float()
        assert torch.equal(out[0][k], want) and torch.equal(out[1][k], want)


def test_allreduce_is_noop_without_process_group():
    import torch
    from paper_1702_07482_gb300.shard import allreduce_gradients
    t = torch.zeros(3, requires_grad=True)
    t.grad = torch.tensor([1.0, 2.0, 3.0])
    allreduce_gradients([t])
    assert torch.equal(t.grad, torch.tensor([1.0, 2.0, 3.0]))


def test_band_rows_partition():
    from paper_1702_07482_gb300.shard import band_rows
    for H in (1, 7, 37, 100, 513):
        for world in (1, 2, 3, 8):
            for ks, T in ((3, 2), (7, 5)):
                bands = [band_rows(H, world, r, ks, T) for r in range(world)]
                owned = [row for o0, o1, _, _ in bands for row in range(o0, o1)]
                assert owned == list(range(H))
                sizes = [o1 - o0 for o0, o1, _, _ in bands]
                assert max(sizes) - min(sizes) <= 1
                ghost = 2 * (ks // 2) * T
                for o0, o1, g0, g1 in bands:
                    assert g0 == max(0, o0 - ghost) and g1 == min(H, o1 + ghost)
    with pytest.raises(ValueError):
        band_rows(10, 2, 2, 3, 1)


def _band_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1702_07482_gb300.shard import band_rows, gather_bands
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    results = []
    for (H, W, ks, nk, T) in ((37, 23, 3, 4, 3), (41, 19, 5, 4, 2)):
        p = synth.params(T, ks, nk, seed=11 + ks)
        _, f = synth.single_image(H, W, 1, 7, index=ks)
        own0, own1, g0, g1 = band_rows(H, world, rank, ks, T)
        band = oracle.forward(f[g0:g1].copy(), p)[-1][own0 - g0:own1 - g0]
        whole = gather_bands(torch.from_numpy(np.ascontiguousarray(band)), H).numpy()
        results.append(whole)
    q.put((rank, results))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_bands_reproduce_the_whole_image(world):
    """One image split into row bands with 2R T ghost rows, each band run alone
    through the FP64 oracle and the owned rows gathered over gloo ranks, equals
    the oracle's whole-image result exactly: the cascade needs no exchange."""
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k, (H, W, ks, nk, T) in enumerate(((37, 23, 3, 4, 3), (41, 19, 5, 4, 2))):
        p = synth.params(T, ks, nk, seed=11 + ks)
        _, f = synth.single_image(H, W, 1, 7, index=ks)
        ref = oracle.forward(f, p)[-1]
        for r in range(world):
            np.testing.assert_array_equal(out[r][k], ref)
        # and the ghosts are needed: one row fewer on each side changes the result
        ghost = 2 * (ks // 2) * T - 1
        cut = H // 2
        short = oracle.forward(f[max(0, cut - ghost):].copy(), p)[-1][min(cut, ghost):]
        assert not np.array_equal(short[0], ref[cut])


# Data-parallel training on the oracle: a batch of 4 crops, loss
# L = sum_s 1/2 |u_T^s - clean^s|^2 (Eq. learning), split 2 + 2 over the ranks.
_DP = dict(H=20, W=23, ks=3, nk=4, T=2, n=4, cfg=41)


def _dp_case():
    import synth
    d = _DP
    p = synth.params(d["T"], d["ks"], d["nk"], seed=synth.seed_for(d["cfg"], 0, "params"))
    pairs = [synth.single_image(d["H"], d["W"], 1, d["cfg"], index=s) for s in range(d["n"])]
    return p, pairs


def _crop_grads(p, clean, f):
    import oracle
    u = oracle.forward(f, p)
    _, gk, gw, gl = oracle.backward(f, p, u, u[-1] - clean)
    return gk, gw, gl


def _dp_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_1702_07482_gb300.shard import allreduce_gradients
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, pairs = _dp_case()
    mine = range(rank * _DP["n"] // world, (rank + 1) * _DP["n"] // world)
    acc = None
    for s in mine:   # this rank's loss sums its own crops
        g = _crop_grads(p, *pairs[s])
        acc = list(g) if acc is None else [a + b for a, b in zip(acc, g)]
    ts = []
    for a in acc:
        t = torch.zeros(a.shape, dtype=torch.float64, requires_grad=True)
        t.grad = torch.from_numpy(np.ascontiguousarray(a))
        ts.append(t)
    allreduce_gradients(ts)
    q.put((rank, [t.grad.numpy().copy() for t in ts]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_oracle_gradients_sum_to_the_whole_batch_gradient():
    """Each gloo rank takes the oracle gradient (filters, RBF weights, lambda)
    of its half of the batch; after allreduce_gradients both ranks hold the
    oracle gradient of the whole batch's loss (to FP64 rounding) and agree bit
    for bit.  The loss-sum convention is pinned by a finite difference of the
    whole-batch loss in one lambda."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = dict(q.get(timeout=300) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, pairs = _dp_case()
    whole = None
    for s in range(_DP["n"]):
        g = _crop_grads(p, *pairs[s])
        whole = list(g) if whole is None else [a + b for a, b in zip(whole, g)]
    for k in range(3):
        np.testing.assert_array_equal(out[0][k], out[1][k])
        np.testing.assert_allclose(out[0][k], whole[k], rtol=1e-12,
                                   atol=1e-12 * np.abs(whole[k]).max())

    def loss(lam1):
        lam = p.lam.copy()
        lam[1] = lam1
        pp = dataclasses.replace(p, lam=lam)
        return sum(0.5 * float(((oracle.forward(f, pp)[-1] - c) ** 2).sum()) for c, f in pairs)

    h = 1e-4 * p.lam[1]
    fd = (loss(p.lam[1] + h) - loss(p.lam[1] - h)) / (2 * h)
    assert abs(fd - out[0][2][1]) <= 1e-6 * max(1.0, abs(fd))
