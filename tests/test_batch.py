"""GPU tests of the persistent batched forward (tnrd_plan_create /
tnrd_batch_forward) over images of different sizes and parameter sets."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from _cases import TOL_U_FP32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


SIZES = [(97, 65, 1, 0), (40, 300, 2, 1), (133, 27, 4, 0), (7, 7, 8, 1), (64, 64, 1, 1),
         (256, 200, 2, 0)]


def _make(T=3, sizes=SIZES, cfg=160):
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    params = [synth.params(T, 7, 48, seed=synth.seed_for(cfg, s, "params")).astype(np.float32)
              .astype(np.float64) for s in range(2)]
    models = [ops.Model.create(p.filters, p.rbf_w, p.lam) for p in params]
    fs, fts, uts, imgs = [], [], [], []
    for i, (H, W, L, s) in enumerate(sizes):
        _, f = synth.single_image(H, W, L, cfg, index=i)
        f = f.astype(np.float32).astype(np.float64)
        ft = ops.to_pitched(torch.tensor(f, dtype=torch.float32, device="cuda"))[0]
        ut = torch.full_like(ft, float("nan"))
        fs.append(f)
        fts.append(ft)
        uts.append(ut)
        imgs.append(B.tnrd_image(ft.data_ptr(), ut.data_ptr(), H, W, ft.shape[-1], s))
    return params, models, fs, fts, uts, imgs


def test_batch_matches_per_image_forward_bit_for_bit():
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    params, models, fs, fts, uts, imgs = _make()
    plan = B.Plan(imgs, [m.params() for m in models])
    stream = torch.cuda.current_stream().cuda_stream
    plan.forward(stream)
    torch.cuda.synchronize()
    assert plan.status() == 0
    # the persistent kernel walks tiles of the one-column-per-lane fused kernel
    os.environ["TNRD_FUSED_TH"] = str(plan.tile_height)
    os.environ["TNRD_FUSED_KERNEL"] = "lane"
    try:
        for (H, W, L, s), ft, ut in zip(SIZES, fts, uts):
            ref = ops.forward(models[s], ft.unsqueeze(0), W=W)[0]
            torch.cuda.synchronize()
            assert torch.equal(ut[:, :W], ref[:, :W])
    finally:
        del os.environ["TNRD_FUSED_TH"]
        del os.environ["TNRD_FUSED_KERNEL"]


def test_stage_schedule_matches_persistent_bit_for_bit():
    """One launch per stage over the plan's tile table gives the same bits as
    the persistent schedule (same tiles, same stage kernel body)."""
    from paper_1702_07482_gb300 import binding as B
    params, models, fs, fts, uts, imgs = _make(T=3, cfg=164)
    stream = torch.cuda.current_stream().cuda_stream
    plan = B.Plan(imgs, [m.params() for m in models])
    assert plan.launches == 1
    plan.forward(stream)
    torch.cuda.synchronize()
    first = [u.clone() for u in uts]
    os.environ["TNRD_BATCH_SCHEDULE"] = "stages"
    try:
        plan2 = B.Plan(imgs, [m.params() for m in models])
    finally:
        del os.environ["TNRD_BATCH_SCHEDULE"]
    assert plan2.launches == 3 and plan2.tile_height == plan.tile_height
    for u in uts:
        u.fill_(float("nan"))
    plan2.forward(stream)
    torch.cuda.synchronize()
    assert plan2.status() == 0
    for (H, W, L, s), a, b in zip(SIZES, first, uts):
        assert torch.equal(a[:, :W], b[:, :W])


def test_batch_matches_oracle_and_replays():
    from paper_1702_07482_gb300 import binding as B
    params, models, fs, fts, uts, imgs = _make(T=2, cfg=161)
    plan = B.Plan(imgs, [m.params() for m in models])
    stream = torch.cuda.current_stream().cuda_stream
    plan.forward(stream)
    torch.cuda.synchronize()
    first = [u.clone() for u in uts]
    for (H, W, L, s), f, u in zip(SIZES, fs, uts):
        ref = oracle.forward(f, params[s])[-1]
        assert np.abs(u[:, :W].double().cpu().numpy() - ref).max() <= TOL_U_FP32
    plan.forward(stream)     # graph replay: same bits
    torch.cuda.synchronize()
    for (H, W, L, sset), a, b in zip(SIZES, first, uts):
        assert torch.equal(a[:, :W], b[:, :W])


def test_wait_limit_zero_reports_timeout_then_recovers():
    from paper_1702_07482_gb300 import binding as B
    params, models, fs, fts, uts, imgs = _make(T=3, cfg=162)
    plan = B.Plan(imgs, [m.params() for m in models])
    stream = torch.cuda.current_stream().cuda_stream
    plan.set_wait_limit(0)            # every dependency wait gives up at once
    plan.forward(stream)
    torch.cuda.synchronize()
    assert plan.status() == 4         # TNRD_ERR_TIMEOUT, and the launch returned
    plan.set_wait_limit(2_000_000_000)
    plan.forward(stream)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for (H, W, L, s), f, u in zip(SIZES, fs, uts):
        ref = oracle.forward(f, params[s])[-1]
        assert np.abs(u[:, :W].double().cpu().numpy() - ref).max() <= TOL_U_FP32


def test_autotuned_plan_and_user_graph_capture():
    from paper_1702_07482_gb300 import binding as B
    params, models, fs, fts, uts, imgs = _make(T=2, cfg=163)
    plan = B.Plan(imgs, [m.params() for m in models], autotune=True)
    assert plan.tile_height in (16, 23, 30, 32, 37, 45)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.forward(s.cuda_stream)   # direct launch while captured
    for u in uts:
        u.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    for (H, W, L, sset), f, u in zip(SIZES, fs, uts):
        ref = oracle.forward(f, params[sset])[-1]
        assert np.abs(u[:, :W].double().cpu().numpy() - ref).max() <= TOL_U_FP32


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
def test_tensor_core_plan_matches_per_image_forward_and_oracle(algo):
    """A plan on the tensor cores (one launch per stage over every image's
    tiles, in a CUDA graph) computes each image exactly as tnrd_forward does
    with the same algorithm, and stays within the stated bound of the oracle."""
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    params, models, fs, fts, uts, imgs = _make(T=2, cfg=165)
    plan = B.Plan(imgs, [m.params() for m in models], algo=B.ALGO[algo])
    stream = torch.cuda.current_stream().cuda_stream
    plan.forward(stream)
    torch.cuda.synchronize()
    assert plan.status() == 0
    # tiles of 2 (TF32) or 3 (BF16) row blocks of 16 z rows, 2R = 6 of them halo
    assert plan.tile_height == 16 * {"tf32": 2, "bf16": 3}[algo] - 2 * 3
    tol = {"tf32": 0.02, "bf16": 0.2}[algo]
    for (H, W, L, s), f, ft, ut in zip(SIZES, fs, fts, uts):
        ref = ops.forward(models[s], ft.unsqueeze(0), W=W, algo=algo)[0]
        torch.cuda.synchronize()
        assert torch.equal(ut[:, :W], ref[:, :W])
        u_or = oracle.forward(f, params[s])[-1]
        assert np.abs(ut[:, :W].double().cpu().numpy() - u_or).max() <= tol
    first = [u.clone() for u in uts]
    plan.forward(stream)          # graph replay: same bits
    torch.cuda.synchronize()
    for (H, W, L, s), a, b in zip(SIZES, first, uts):
        assert torch.equal(a[:, :W], b[:, :W])


def test_pair_schedule_matches_per_image_pair_kernel_and_oracle():
    """The column-pair schedule (one launch per stage over tiles of 64 - 2R
    columns on two-CTA clusters): each image equals tnrd_forward's column-pair
    kernel at the same tile height bit for bit, stays within the FP32 bound of
    the oracle, and repeats its bits on a graph replay."""
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    params, models, fs, fts, uts, imgs = _make(T=3, cfg=166)
    stream = torch.cuda.current_stream().cuda_stream
    os.environ["TNRD_BATCH_SCHEDULE"] = "pairs"
    try:
        plan = B.Plan(imgs, [m.params() for m in models])
    finally:
        del os.environ["TNRD_BATCH_SCHEDULE"]
    assert plan.launches == 3 and plan.tile_width == 64 - 2 * 3
    plan.forward(stream)
    torch.cuda.synchronize()
    assert plan.status() == 0
    first = [u.clone() for u in uts]
    env = {"TNRD_FUSED_KERNEL": "pair2", "TNRD_FUSED_TH": str(plan.tile_height),
           "TNRD_FUSED_ROWS": "uniform"}
    os.environ.update(env)
    try:
        for (H, W, L, s), f, ft, ut in zip(SIZES, fs, fts, uts):
            ref = ops.forward(models[s], ft.unsqueeze(0), W=W)[0]
            torch.cuda.synchronize()
            assert torch.equal(ut[:, :W], ref[:, :W])
            u_or = oracle.forward(f, params[s])[-1]
            assert np.abs(ut[:, :W].double().cpu().numpy() - u_or).max() <= TOL_U_FP32
    finally:
        for k in env:
            del os.environ[k]
    plan.forward(stream)
    torch.cuda.synchronize()
    for (H, W, L, s), a, b in zip(SIZES, first, uts):
        assert torch.equal(a[:, :W], b[:, :W])
