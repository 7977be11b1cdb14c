"""GPU: one image split into row bands (shard.band_rows), each band run alone
with its 2R T ghost rows through the fused stage (ops.forward_band), gives the
whole image's result.  Each pixel's sums run in the same order whatever tile
computes it, so with one kernel variant for all shapes (the one-column kernel)
the assembled bands equal the whole-image forward bit for bit; the default
choice (which may pick another variant per band) stays within the FP32
tolerance of the whole image."""
import os

import numpy as np
import pytest
import torch

from _cases import TOL_U_FP32, case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _bands(m, ft, world, ops):
    parts = []
    for r in range(world):
        rows, o0, o1 = ops.forward_band(m, ft, world, r)
        parts.append(rows)
    return torch.cat(parts)


@pytest.mark.parametrize("world", [2, 3, 5])
@pytest.mark.parametrize("H,W,ks,nk,T", [(200, 150, 7, 48, 2), (131, 77, 5, 24, 3)])
def test_bands_equal_whole_image(world, H, W, ks, nk, T):
    from paper_1702_07482_gb300 import ops
    p, f = case(H, W, ks, nk, T, L=1, N=1, cfg=611 + H)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    ft = torch.tensor(f[0], dtype=torch.float32, device="cuda")
    old = os.environ.get("TNRD_FUSED_KERNEL")
    os.environ["TNRD_FUSED_KERNEL"] = "lane"
    try:
        whole = ops.forward(m, ft)[:, :W]
        got = _bands(m, ft, world, ops)
    finally:
        if old is None:
            os.environ.pop("TNRD_FUSED_KERNEL", None)
        else:
            os.environ["TNRD_FUSED_KERNEL"] = old
    torch.cuda.synchronize()
    assert got.shape == whole.shape
    assert torch.equal(got, whole)
    # default kernel choice per band: within the FP32 bound of the whole image
    got2 = _bands(m, ft, world, ops)
    torch.cuda.synchronize()
    assert (got2 - whole).abs().max().item() <= TOL_U_FP32
