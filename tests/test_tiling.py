"""Row tilings of the fused forward stage: runtime tile heights below the
compiled one, and short border tile rows (the first and last tile rows 2R
shorter, so that every tile walks th + 4R steps).

Each output pixel's sums run in the same order whatever tile computes it, so
every tiling must give the same bits; one tiling per case is also checked
against the FP64 oracle.  Heights include the smallest image that allows short
border rows (H = 2 te + th), ragged last tiles, a last interior tile shifted
back onto its neighbour, and several images per call.
"""
import os

import numpy as np
import pytest
import torch

from _cases import TOL_U_FP32, case

ENV = ("TNRD_FUSED_KERNEL", "TNRD_FUSED_TH", "TNRD_FUSED_ROWS")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _run(p, f, **env):
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    old = {k: os.environ.get(k) for k in ENV}
    for k in ENV:
        os.environ.pop(k, None)
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
        N, H, W = f.shape
        name = B.tnrd_forward_kernel(m.params(), N, H, W, B.ALGO["fused"])
        ft = torch.tensor(f, dtype=torch.float32, device="cuda")
        out = ops.forward(m, ft)
        torch.cuda.synchronize()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out[..., :W], name


# (H, W, N): 99 = 2 * 31 + 37 (short rows just allowed at th 37), 100, 150
# (ragged), 241 (last interior tile shifted back), 3 images of 77 x 50.
SIZES = [(99, 70, 1), (100, 129, 1), (150, 61, 1), (241, 90, 1), (77, 50, 3)]


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", ["lane", "pair", "pair2", "pair8"])
@pytest.mark.parametrize("H,W,N", SIZES)
def test_row_tilings_give_the_same_bits(kernel, H, W, N):
    p, f = case(H, W, 7, 48, 2, L=1, N=N, cfg=501 + H + W)
    ref, _ = _run(p, f, TNRD_FUSED_KERNEL=kernel, TNRD_FUSED_TH=37, TNRD_FUSED_ROWS="uniform")
    for th in (16, 23, 33, 37, 45):
        for rows in ("uniform", "short"):
            got, name = _run(p, f, TNRD_FUSED_KERNEL=kernel, TNRD_FUSED_TH=th, TNRD_FUSED_ROWS=rows)
            assert torch.equal(got, ref), name
    from paper_1702_07482_gb300 import binding as B
    assert B.tnrd_device_status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", ["lane", "pair2"])
def test_short_border_rows_match_oracle(kernel):
    import oracle
    p, f = case(130, 90, 7, 48, 2, L=1, N=1, cfg=560)
    got, name = _run(p, f, TNRD_FUSED_KERNEL=kernel, TNRD_FUSED_TH=33, TNRD_FUSED_ROWS="short")
    assert "border rows 27" in name
    ref = oracle.forward(f[0], p)[-1]
    assert np.abs(got[0].double().cpu().numpy() - ref).max() <= TOL_U_FP32


@pytest.mark.gpu
def test_512_image_tiling_is_one_wave():
    """The 512 x 512 workload: 33-row tiles with 27-row border rows, 16 tile
    rows x 9 tile columns x 2 CTAs = 288 CTAs, one per slot of 152 SMs."""
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    q = synth.params(2, 7, 48, seed=3)
    prm = ops.Model.create(q.filters, q.rbf_w, q.lam).params()
    if torch.cuda.get_device_properties(0).multi_processor_count < 144:
        pytest.skip("fewer than 144 SMs")
    name = B.tnrd_forward_kernel(prm, 1, 512, 512, B.ALGO["fused"])
    assert name.startswith("fused_pair2_fwd<7,48,37> tiles 33x58 (border rows 27)"), name


@pytest.mark.parametrize("N,H,W", [(1, 512, 512), (32, 180, 180), (16, 2048, 2048), (1, 128, 128),
                                   (1, 97, 65), (1, 7, 7), (4, 512, 512), (3, 1000, 333)])
@pytest.mark.parametrize("ks,nk", [(7, 48), (5, 24), (3, 4)])
def test_tiling_choice_host_only(N, H, W, ks, nk):
    """Host-only (no GPU): the row tiling named by tnrd_forward_kernel keeps the
    runtime tile height within the compiled one, uses short border rows only
    where the image holds two of them and a full interior tile (te = th - 2R),
    and honours the overrides."""
    import re
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    q = synth.params(1, ks, nk, seed=5)
    prm = ops.Model.create(q.filters, q.rbf_w, q.lam, device="cpu").params()
    R = ks // 2
    old = {k: os.environ.pop(k, None) for k in ENV}
    try:
        name = B.tnrd_forward_kernel(prm, N, H, W, B.ALGO["fused"])
        m = re.match(r"(fused_stage_fwd|fused_pair[248]_fwd|fused_pair_fwd)<(\d+),(\d+),(\d+)> "
                     r"tiles (\d+)x(\d+)(?: \(border rows (\d+)\))?, (tma|gather) staging$", name)
        assert m, name
        kth, th, tw = int(m.group(4)), int(m.group(5)), int(m.group(6))
        assert (int(m.group(2)), int(m.group(3))) == (ks, nk)
        assert 2 * R < th <= kth
        assert tw == (32 if m.group(1) == "fused_stage_fwd" else 64) - 2 * R
        if m.group(7):
            te = int(m.group(7))
            assert te == th - 2 * R and H >= 2 * te + th
        for rows in ("uniform", "short"):
            os.environ["TNRD_FUSED_ROWS"] = rows
            os.environ["TNRD_FUSED_TH"] = str(kth)
            n2 = B.tnrd_forward_kernel(prm, N, H, W, B.ALGO["fused"])
            te2 = re.search(r"border rows (\d+)", n2)
            if rows == "uniform" or H < 2 * (kth - 2 * R) + kth:
                assert te2 is None, n2
                assert f"tiles {kth}x" in n2, n2
            else:
                assert te2 and int(te2.group(1)) == kth - 2 * R, n2
    finally:
        for k in ENV:
            os.environ.pop(k, None)
        for k, v in old.items():
            if v is not None:
                os.environ[k] = v


@pytest.mark.parametrize("N,H,W,want", [(16, 2048, 2048, "fused_pair2_fwd"),
                                        (32, 180, 180, "fused_stage_fwd"),
                                        (1, 512, 512, "fused_pair2_fwd"),
                                        (1, 128, 128, "fused_pair4_fwd")])
def test_kernel_choice_host_only(N, H, W, want):
    """Host-only: the kernel tnrd_forward picks where it was measured -- the
    two-CTA pair kernel on wide images (16 x 2048^2: 318.8 against 284.4
    Mpixel/s), one column per lane on the 180-wide training crops (127.4 against
    122.6), four-CTA clusters of 12-row tiles on the 128^2, 5x5x24 image (259.8
    against 212.0 with 17 rows and 223.6 on eight-CTA clusters).  (Without a GPU
    the one-launch cascade is never chosen: its co-residency check needs one.)"""
    import synth
    from paper_1702_07482_gb300 import binding as B
    from paper_1702_07482_gb300 import ops
    ks, nk = (5, 24) if H == 128 else (7, 48)
    q = synth.params(1, ks, nk, seed=5)
    prm = ops.Model.create(q.filters, q.rbf_w, q.lam, device="cpu").params()
    old = {k: os.environ.pop(k, None) for k in ENV}
    try:
        assert B.tnrd_forward_kernel(prm, N, H, W, B.ALGO["fused"]).startswith(want)
    finally:
        for k, v in old.items():
            if v is not None:
                os.environ[k] = v
