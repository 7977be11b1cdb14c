"""GPU parity of the quality indexes (tnrd_quality, Sec. 4) with the FP64
oracle (oracle/quality.py, pinned in tests/test_quality_oracle.py).  The GPU
forms every per-pixel quantity in FP32 and sums 4 pixels per thread in FP32
(relative error about 1e-7 per partial), the partials in FP64: relative
agreement 1e-6 (absolute 1e-9 near zero).  The SSIM window statistics are FP32,
centred (sums of w (x - mx)(y - my) over 121 terms): MSSIM agrees to 1e-5
absolute."""
import numpy as np
import pytest
import torch

import synth
from oracle import quality as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _triplet(H, W, seed, N=1):
    refs, imgs, noisys = [], [], []
    for n in range(N):
        clean, f = synth.single_image(H, W, 2, 600 + seed, index=n)
        g = np.random.Generator(np.random.PCG64(seed * 10 + n))
        img = clean * (1 + 0.05 * g.standard_normal(clean.shape))   # a "despeckled" result
        img = np.maximum(img, 0.5)
        refs.append(clean)
        imgs.append(img)
        noisys.append(f)
    c = lambda a: np.stack(a).astype(np.float32).astype(np.float64)
    return c(refs), c(imgs), c(noisys)


def _gpu(ref, img, noisy, peak=255.0):
    from paper_1702_07482_gb300 import ops
    t = lambda a: None if a is None else torch.tensor(a, dtype=torch.float32, device="cuda")
    out = ops.quality(t(img), t(ref), t(noisy), peak)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _cmp(got, ref):
    names = ("psnr", "mssim", "ec", "ri_mean", "ri_var", "cv")
    for k, name in enumerate(names):
        a, b = got[k], ref[name]
        if np.isnan(b):
            assert np.isnan(a), name
        elif name == "mssim":
            assert abs(a - b) <= 1e-5, (name, a, b)
        else:
            assert a == pytest.approx(b, rel=1e-6, abs=1e-9), (name, a, b)


@pytest.mark.parametrize("H,W,N", [(64, 64, 1), (97, 130, 2), (33, 40, 1), (11, 11, 1),
                                   (200, 75, 1)])
def test_indexes_match_oracle(H, W, N):
    ref, img, noisy = _triplet(H, W, H + W, N)
    got = _gpu(ref, img, noisy)
    for n in range(N):
        _cmp(got[n], Q.indexes(ref[n], img[n], noisy[n]))


def test_small_images_and_missing_inputs():
    ref, img, noisy = _triplet(10, 30, 3)
    got = _gpu(ref, img, noisy)[0]
    assert np.isnan(got[1])                      # no 11 x 11 window fits
    rim, riv = Q.ratio_image_stats(noisy[0], img[0])
    ref_idx = {"psnr": Q.psnr(ref[0], img[0]), "mssim": np.nan,
               "ec": Q.edge_correlation(ref[0], img[0]), "ri_mean": rim, "ri_var": riv,
               "cv": Q.coefficient_of_variation(img[0])}
    _cmp(got, ref_idx)
    no_ref = _gpu(None, img, noisy)[0]
    assert np.all(np.isnan(no_ref[:3])) and np.all(np.isfinite(no_ref[3:]))
    no_noisy = _gpu(ref, img, None)[0]
    assert np.all(np.isnan(no_noisy[3:5])) and np.isfinite(no_noisy[5])


def test_identical_images_and_repeatable_bits():
    ref, img, noisy = _triplet(90, 70, 4)
    got = _gpu(ref, ref, noisy)[0]
    assert got[1] == pytest.approx(1.0, abs=1e-6) and got[2] == pytest.approx(1.0, abs=1e-6)
    assert np.isinf(got[0])
    a = _gpu(ref, img, noisy)
    b = _gpu(ref, img, noisy)
    np.testing.assert_array_equal(a, b)


def test_indexes_of_a_despeckled_cascade_output():
    """The indexes of a TRDMD forward result on the 512^2 L=1 workload shape
    (sampled by the same oracle definitions)."""
    import oracle
    from paper_1702_07482_gb300 import ops
    from _cases import case
    p, f = case(128, 128, 7, 48, 3, cfg=610)
    clean = synth.single_image(128, 128, 1, 610, index=0)[0].astype(np.float32).astype(np.float64)
    m = ops.Model.create(p.filters, p.rbf_w, p.lam)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    u = ops.forward(m, ft)[..., :128]
    torch.cuda.synchronize()
    un = u.double().cpu().numpy()
    got = _gpu(clean[None], un, f)[0]
    _cmp(got, Q.indexes(clean, un[0], f[0]))
