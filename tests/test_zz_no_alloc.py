"""tnrd_forward_noalloc: the forward cascade for callers that cannot allocate
device memory (hosts that own all device memory and forbid a library from
calling cudaMalloc, or real-time loops where an allocation may stall or fail).
It keeps the image between stages in a scratch array built into the library
instead of a caller workspace and runs the same kernels with the same tiling
as tnrd_forward, so its results must equal tnrd_forward's bit for bit.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from _cases import case


def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    return binding


def _noalloc_vs_forward(B, m, ft, N, H, W, P, stream):
    import torch
    from paper_1702_07482_gb300 import ops
    ref = ops.forward(m, ft, keep_stages=False, algo="fused", W=W)
    got = torch.full_like(ft, float("nan"))
    B.tnrd_forward_noalloc(m.params(), N, H, W, P, ft, got, stream)
    torch.cuda.synchronize()
    assert torch.isfinite(got[..., :W]).all()
    assert torch.equal(got[..., :W], ref[..., :W])


@pytest.mark.gpu
def test_noalloc_matches_forward_on_two_calls_in_a_row():
    import torch
    from paper_1702_07482_gb300 import ops
    B = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    # two different inputs (odd and even stage counts: the scratch holds the
    # image between stages in both ping-pong parities), one call each, back to
    # back: the second call must not see anything the first left in the scratch
    for cfg, (H, W, N, T) in ((130, (96, 70, 2, 3)), (131, (61, 129, 1, 4))):
        p, f = case(H, W, 7, 48, T, N=N, cfg=cfg)
        m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
        ft = ops.to_pitched(torch.tensor(f, dtype=torch.float32, device="cuda"))
        _noalloc_vs_forward(B, m, ft, N, H, W, ft.shape[-1], stream)


@pytest.mark.gpu
def test_noalloc_at_its_size_limit_and_one_row_beyond():
    import torch
    from paper_1702_07482_gb300 import ops
    B = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    # exactly TNRD_NOALLOC_MAX_FLOATS: one 2048 x 2048 image, pitch 2048
    S = 2048
    assert S * S == B.NOALLOC_MAX_FLOATS
    p, f = case(S, S, 7, 48, 2, cfg=132)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    _noalloc_vs_forward(B, m, ft, 1, S, S, S, stream)
    # one row more is rejected before anything is launched: u keeps its canary
    f2 = torch.ones((1, S + 1, S), dtype=torch.float32, device="cuda")
    u2 = torch.full_like(f2, 12345.0)
    with pytest.raises(RuntimeError, match="scratch"):
        B.tnrd_forward_noalloc(m.params(), 1, S + 1, S, S, f2, u2, stream)
    torch.cuda.synchronize()
    assert bool((u2 == 12345.0).all())


def test_noalloc_rejects_a_batch_larger_than_its_scratch():
    B = _lib()
    L = B.load()
    p = B.tnrd_params()
    p.T, p.ksize, p.nfilt, p.nrbf = 3, 7, 48, 63
    p.rbf_mu0, p.rbf_delta, p.rbf_gamma = -310.0, 10.0, 10.0
    p.filters = p.rbf_w = p.lambda_ = 0x1000
    H = W = 2048
    N = B.NOALLOC_MAX_FLOATS // (H * W) + 1
    st = L.tnrd_forward_noalloc(ctypes.byref(p), N, H, W, W, ctypes.c_void_p(0x10000),
                                ctypes.c_void_p(0x2000000), None)
    assert st == 1
    assert "scratch" in B.last_error()
