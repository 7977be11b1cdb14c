"""The one-launch cascade of small images (fused_pairc_cascade): all T stages of
a batch of images too small to fill the GPU in one launch, the column-pair walk
on clusters of four or eight CTAs per tile, a grid-wide barrier between stages.
It must give exactly the bits of the per-stage launches of the same kernel
(TNRD_CASCADE=0), for both ping-pong parities and with all stages kept, match
the FP64 oracle, and report a barrier wait that runs out without hanging."""
import os

import numpy as np
import pytest
import torch

import oracle
from _cases import TOL_U_FP32, case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _forward(p, f, keep, cascade, kernel=None):
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    env = {"TNRD_CASCADE": None if cascade else "0", "TNRD_FUSED_KERNEL": kernel}
    old = {k: os.environ.get(k) for k in env}
    try:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
        ft = torch.tensor(f, dtype=torch.float32, device="cuda")
        N, H, W = f.shape
        name = B.tnrd_forward_kernel(m.params(), N, H, W, B.ALGO["fused"])
        u = ops.forward(m, ft, keep_stages=keep)
        torch.cuda.synchronize()
        assert B.tnrd_device_status() == 0
        return u[..., :W].clone(), name
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("keep", [False, True])
@pytest.mark.parametrize("H,W,ks,nk,T,N,kernel", [
    (128, 128, 5, 24, 5, 1, None),       # the 128^2 workload: four-CTA clusters
    (128, 128, 5, 24, 4, 1, "pair8"),    # eight-CTA clusters, even T
    (97, 65, 7, 48, 3, 2, None),         # two images, ragged
    (64, 35, 3, 4, 2, 1, "pair4"),
    (40, 70, 7, 48, 6, 1, "pair4"),
])
def test_cascade_equals_per_stage_launches(H, W, ks, nk, T, N, kernel, keep):
    p, f = case(H, W, ks, nk, T, N=N, cfg=600 + H + W + T)
    got, name = _forward(p, f, keep, True, kernel)
    ref, name0 = _forward(p, f, keep, False, kernel)
    assert name.startswith("fused_pairc_cascade"), name
    assert not name0.startswith("fused_pairc_cascade"), name0
    assert torch.equal(got, ref)


def test_cascade_matches_oracle_every_stage():
    p, f = case(128, 128, 5, 24, 5, N=1, cfg=611)
    got, name = _forward(p, f, True, True)
    assert name.startswith("fused_pairc_cascade"), name
    ref = oracle.forward(f[0], p)
    err = np.abs(got[:, 0].double().cpu().numpy() - ref).max(axis=(1, 2))
    assert np.all(err <= TOL_U_FP32), err


def test_cascade_barrier_wait_runs_out_and_reports():
    """A zero wait limit (tnrd_stage_wait_test) makes the grid barriers' waits
    run out: the launch still ends (every wait bounded, every CTA passes every
    cluster barrier), TNRD_ERR_TIMEOUT is reported, and the next call is right."""
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    p, f = case(128, 128, 5, 24, 5, N=1, cfg=612)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    assert B.tnrd_device_status() in (0, 4)          # clears the word
    assert B.tnrd_forward_kernel(m.params(), 1, 128, 128, B.ALGO["fused"]).startswith(
        "fused_pairc_cascade")
    B.tnrd_stage_wait_test(0, False)
    try:
        ops.forward(m, ft)
        torch.cuda.synchronize()
    finally:
        B.tnrd_stage_wait_test(1 << 31, False)
    assert B.tnrd_device_status() == 4               # TNRD_ERR_TIMEOUT
    good = ops.forward(m, ft)[0, :, :128].double().cpu().numpy()
    torch.cuda.synchronize()
    assert B.tnrd_device_status() == 0
    assert np.abs(good - oracle.forward(f[0], p)[-1]).max() <= TOL_U_FP32
