"""tnrd_forward_noalloc: the forward cascade for callers that cannot allocate
device memory (hosts that own all device memory and forbid a library from
calling cudaMalloc, or real-time loops where an allocation may stall or fail).
It keeps the image between stages in a scratch array built into the library
instead of a caller workspace, so its results must equal tnrd_forward's.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from _cases import TOL_U_FP32, case


def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.gpu
def test_noalloc_matches_forward_on_two_calls_in_a_row():
    import torch
    from paper_1702_07482_gb300 import ops
    B = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    # two different inputs, one call each, back to back: the second call must
    # not see anything the first left in the shared scratch
    for cfg, (H, W, N, T) in ((130, (96, 70, 2, 3)), (131, (61, 129, 1, 4))):
        p, f = case(H, W, 7, 48, T, N=N, cfg=cfg)
        m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
        ft = ops.to_pitched(torch.tensor(f, dtype=torch.float32, device="cuda"))
        P = ft.shape[-1]
        ref = ops.forward(m, ft, keep_stages=False, algo="fused", W=W)
        got = torch.full_like(ft, float("nan"))
        B.tnrd_forward_noalloc(m.params(), N, H, W, P, ft, got, stream)
        torch.cuda.synchronize()
        a = got[..., :W].double().cpu().numpy()
        r = ref[..., :W].double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.abs(a - r).max() <= TOL_U_FP32


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
