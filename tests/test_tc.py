"""GPU tests of the tensor-core stage (TNRD_ALGO_TC_TF32): filter bank and
adjoint as tcgen05 GEMMs with TF32 operands, phi and the prox in FP32.

TF32 keeps 10 mantissa bits, so this path is not held to the FP32 bound.  Its
stated accuracy against the FP64 oracle, asserted here: max |u_gpu - u_oracle|
<= 2.0 on the [0, 255] scale for every stage, and PSNR(u_T vs oracle) >= 55 dB.
"""
import numpy as np
import pytest
import torch

import oracle
from _cases import case, crop_window

pytestmark = pytest.mark.gpu

TOL_TF32_MAXABS = 2.0
TOL_TF32_PSNR = 55.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _run(p, f, algo="tf32", keep=True):
    from paper_1702_07482_gb300 import binding, ops
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda")
    u = ops.forward(m, ft, keep_stages=keep, algo=algo)
    torch.cuda.synchronize()
    assert binding.tnrd_device_status() == 0
    return u[..., :f.shape[-1]].double().cpu().numpy()


def _psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10 * np.log10(255.0 ** 2 / max(mse, 1e-30))


@pytest.mark.parametrize("H,W,ks,nk,T,N", [
    (128, 128, 7, 48, 5, 1),
    (97, 65, 7, 48, 2, 2),
    (7, 7, 7, 48, 2, 1),
    (64, 35, 3, 4, 2, 1),
    (50, 100, 5, 24, 3, 1),
    (45, 200, 7, 48, 1, 1),
])
def test_tf32_matches_oracle_within_stated_bound(H, W, ks, nk, T, N):
    p, f = case(H, W, ks, nk, T, N=N, cfg=180 + H)
    got = _run(p, f)
    ref = np.stack([oracle.forward(f[n], p) for n in range(N)], axis=1)
    np.testing.assert_array_equal(got[0], f)
    err = np.abs(got - ref).max(axis=(1, 2, 3))
    assert np.all(err <= TOL_TF32_MAXABS), err
    assert _psnr(got[-1], ref[-1]) >= TOL_TF32_PSNR


def test_tf32_repeatable_bits_and_final_only():
    p, f = case(80, 90, 7, 48, 3, cfg=190)
    a = _run(p, f, keep=True)
    b = _run(p, f, keep=False)
    c = _run(p, f, keep=False)
    np.testing.assert_array_equal(a[-1], b)
    np.testing.assert_array_equal(b, c)


def test_tf32_full_size_2048_T8_sampled_windows():
    """One 2048 x 2048 image of the mixed-precision workload (L=2, 7x7x48, T=8)
    in the launch the benchmark times; the oracle computes sampled pixels on
    crops the crop edge cannot reach (radius 2R T = 48)."""
    H = W = 2048
    T = 8
    p, f = case(H, W, 7, 48, T, L=2, cfg=5)
    got = _run(p, f, keep=False)[0]
    M = 2 * 3 * T
    g = np.random.Generator(np.random.PCG64(11))
    pts = [(0, 0), (2047, 2047), (0, 1024), (1500, 0), (3, 2044)]
    pts += [tuple(x) for x in g.integers(0, 2048, size=(6, 2))]
    errs = []
    for (y, x) in pts:
        y0, y1, x0, x1 = crop_window(H, W, y, x, M)
        ref = oracle.forward(f[0, y0:y1, x0:x1], p)[-1][y - y0, x - x0]
        errs.append(abs(got[y, x] - ref))
    assert max(errs) <= TOL_TF32_MAXABS, errs
