"""Tile staging by bulk tensor copies (TMA) against the symmetric gather.

The fused stage kernels stage each haloed u_{t-1} tile with one
cp.async.bulk.tensor box copy (start column rounded down to 16 bytes), then
mirror the zero-filled out-of-image part of the box in shared memory.  The
staged values, and so every output bit, must equal those of the element-wise
symmetric gather (TNRD_TMA=0).  Sizes cover images smaller than one tile (the
halo reflects more than once), odd widths (start columns at every residue mod
4, and odd start columns, which the float2 row reads of the column-pair
kernels cannot use: those tiles fall back to the gather), ragged tails and
several images per call (the tensor map's third dimension).
"""
import os

import numpy as np
import pytest
import torch

from _cases import TOL_U_FP32, case


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


SIZES = [(7, 7, 7, 48, 2, 1), (13, 40, 7, 48, 2, 2), (97, 65, 7, 48, 2, 1),
         (133, 27, 5, 24, 2, 1), (64, 35, 3, 4, 3, 3), (150, 301, 7, 48, 2, 1),
         (40, 257, 5, 24, 1, 2), (200, 131, 7, 48, 1, 1)]


def _run(p, f, kernel, tma, keep=True):
    from paper_1702_07482_gb300 import ops
    old = {k: os.environ.get(k) for k in ("TNRD_FUSED_KERNEL", "TNRD_TMA")}
    os.environ["TNRD_FUSED_KERNEL"] = kernel
    os.environ["TNRD_TMA"] = "1" if tma else "0"
    try:
        m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
        ft = torch.tensor(f, dtype=torch.float32, device="cuda")
        out = ops.forward(m, ft, keep_stages=keep)
        torch.cuda.synchronize()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", ["lane", "pair", "pair2", "pair4", "pair8"])
@pytest.mark.parametrize("H,W,ks,nk,T,N", SIZES)
def test_tma_staging_matches_gather_bit_for_bit(kernel, H, W, ks, nk, T, N):
    from paper_1702_07482_gb300 import binding as B
    B.load()
    p, f = case(H, W, ks, nk, T, L=1, N=N, cfg=301 + H + 3 * W)
    a = _run(p, f, kernel, tma=True)
    b = _run(p, f, kernel, tma=False)
    assert B.tnrd_device_status() == 0
    assert not torch.isnan(a[..., :W]).any()
    assert torch.equal(a[..., :W], b[..., :W])


@pytest.mark.gpu
def test_tma_staging_matches_oracle():
    import oracle
    p, f = case(61, 77, 7, 48, 2, L=1, N=1, cfg=399)
    for kernel in ("lane", "pair", "pair2"):
        got = _run(p, f, kernel, tma=True, keep=False)[0, :, :77].double().cpu().numpy()
        ref = oracle.forward(f[0], p)[-1]
        assert np.abs(got - ref).max() <= TOL_U_FP32


@pytest.mark.gpu
@pytest.mark.parametrize("schedule", ["stages", "pairs"])
def test_batched_stage_schedule_tma_matches_gather(schedule):
    """Per-stage batched plans (one-column and column-pair tiles): tiles of every
    image staged from per-image tensor maps of f, u and the inter-stage buffer
    give the gather's bits."""
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    sizes = [(97, 65, 0), (40, 300, 1), (7, 7, 0), (133, 27, 1), (256, 201, 0)]
    params = [synth.params(3, 7, 48, seed=synth.seed_for(170, s, "params")) for s in range(2)]
    models = [ops.Model.create(q.filters, q.rbf_w, q.lam) for q in params]
    fts, uts, imgs = [], [], []
    for i, (H, W, s) in enumerate(sizes):
        _, f = synth.single_image(H, W, 1, 170, index=i)
        ft = ops.to_pitched(torch.tensor(f, dtype=torch.float32, device="cuda"))[0]
        ut = torch.full_like(ft, float("nan"))
        fts.append(ft)
        uts.append(ut)
        imgs.append(B.tnrd_image(ft.data_ptr(), ut.data_ptr(), H, W, ft.shape[-1], s))
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for tma in ("1", "0"):
        os.environ["TNRD_BATCH_SCHEDULE"] = schedule
        os.environ["TNRD_TMA"] = tma
        try:
            plan = B.Plan(imgs, [m.params() for m in models])
        finally:
            del os.environ["TNRD_BATCH_SCHEDULE"]
            del os.environ["TNRD_TMA"]
        assert plan.launches == 3
        for u in uts:
            u.fill_(float("nan"))
        plan.forward(stream)
        torch.cuda.synchronize()
        assert plan.status() == 0
        outs.append([u.clone() for u in uts])
        plan.close()
    assert B.tnrd_device_status() == 0
    for (H, W, s), a, b in zip(sizes, *outs):
        assert not torch.isnan(a[:, :W]).any()
        assert torch.equal(a[:, :W], b[:, :W])


def test_kernel_query_names_the_staging():
    """Host-only: the fused stage reports TMA staging by default and the gather
    with TNRD_TMA=0."""
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    q = synth.params(2, 7, 48, seed=3)
    prm = ops.Model.create(q.filters, q.rbf_w, q.lam, device="cpu").params()
    assert B.tnrd_forward_kernel(prm, 1, 512, 512, B.ALGO["fused"]).endswith("tma staging")
    os.environ["TNRD_TMA"] = "0"
    try:
        assert B.tnrd_forward_kernel(prm, 1, 512, 512, B.ALGO["fused"]).endswith("gather staging")
    finally:
        del os.environ["TNRD_TMA"]


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", ["lane", "pair2"])
def test_copy_wait_runs_out_and_reports(kernel):
    """A tile copy whose wait runs out (tnrd_stage_wait_test: the mbarrier armed
    for more bytes than the copy brings): every tile records TNRD_ERR_TIMEOUT and
    writes nothing, no GPU fault, and the context stays usable -- the next call
    matches the oracle with status OK."""
    import oracle
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    H, W = 40, 60
    p, f = case(H, W, 7, 48, 1, L=1, N=1, cfg=391)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    assert B.tnrd_device_status() in (0, 4)          # clears the word
    old = os.environ.get("TNRD_FUSED_KERNEL")
    os.environ["TNRD_FUSED_KERNEL"] = kernel
    try:
        out = torch.full((1, H, ops.pitch_for(W)), float("nan"), device="cuda")
        B.tnrd_stage_wait_test(200_000, True)
        try:
            ops.forward(m, ft, out=out)
            torch.cuda.synchronize()
        finally:
            B.tnrd_stage_wait_test(1 << 31, False)
        assert B.tnrd_device_status() == 4           # TNRD_ERR_TIMEOUT
        assert torch.isnan(out[..., :W]).all()       # no tile wrote its outputs
        good = ops.forward(m, ft)[0, :, :W].double().cpu().numpy()
        torch.cuda.synchronize()
        assert B.tnrd_device_status() == 0
    finally:
        if old is None:
            os.environ.pop("TNRD_FUSED_KERNEL", None)
        else:
            os.environ["TNRD_FUSED_KERNEL"] = old
    assert np.abs(good - oracle.forward(f[0], p)[-1]).max() <= TOL_U_FP32
