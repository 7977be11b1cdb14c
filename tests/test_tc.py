"""GPU tests of the tensor-core stages (TNRD_ALGO_TC_TF32, TNRD_ALGO_TC_BF16):
filter bank and adjoint as tcgen05 GEMMs with TF32 or BF16 operands and FP32
accumulation, phi and the prox in FP32.

Two kinds of check:

* Rounding model.  Each product of the two GEMMs is exact in FP32 (11 x 11 or
  8 x 8 significant bits), so the stage equals FP64 arithmetic on operands
  rounded the way the kernel rounds them -- u and the filters in the filter
  bank, phi's outputs and the filters in the adjoint (TF32: round to nearest,
  ties away; BF16: round to nearest even) -- up to FP32 accumulation and
  phi's FP32 evaluation.  One stage built from the oracle's primitives on the
  rounded operands must match the GPU within the FP32 bound, 1e-3.

* Stated accuracy against the FP64 oracle.  Rounding the operands to a
  relative precision eps moves z by about ||k|| |u| eps and, through phi' and
  the adjoint sum over N_k k^2 taps, u_t by a few eps |u|-weighted units; the
  FP64 emulation above gives max |du| = 0.0045 (TF32, eps = 2^-11) and 0.029
  (BF16, eps = 2^-8) for one 7x7x48 stage on a 64 x 64 L=1 image, and the
  prox contracts the error over later stages.  Asserted with a margin of
  about 4x: max |u_gpu - u_oracle| <= 0.02 (TF32) / 0.2 (BF16) on the
  [0, 255] scale for every stage, PSNR(u_T vs oracle) >= 100 dB / 85 dB.
"""
import numpy as np
import pytest
import torch

import oracle
from _cases import TOL_U_FP32, case, crop_window

pytestmark = pytest.mark.gpu

TOL = {"tf32": (0.02, 100.0), "bf16": (0.2, 85.0)}   # (max |du|, min PSNR dB)


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


def _round_tf32(x):
    """FP32 -> TF32, round to nearest with ties away from zero (10 fraction bits)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def _round_bf16(x):
    """FP32 -> BF16, round to nearest even (7 fraction bits)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


ROUND = {"tf32": _round_tf32, "bf16": _round_bf16}


def _rounded_stage(p, f, rnd):
    """One stage in FP64 on rounded GEMM operands, from the oracle's primitives."""
    u = np.asarray(f, np.float64)
    g = np.zeros_like(u)
    for i in range(p.nk):
        k = rnd(p.filters[0, i])
        z = oracle.conv(rnd(u), k)
        v = oracle.phi(z, p.rbf_w[0, i], p.mu0, p.delta, p.gamma)
        g += oracle.conv_adj(rnd(v), k)
    return oracle.prox(u - g, u, float(p.lam[0]))


def test_rounding_helpers_pinned():
    """The host-side roundings against torch's BF16 cast and hand-made ties."""
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -11), 255.3], np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(_round_bf16(x), ref)
    # TF32 ties go away from zero: 1 + 2^-11 -> 1 + 2^-10, -(1 + 2^-11) -> -(1 + 2^-10)
    assert _round_tf32(np.float32(1 + 2 ** -11)) == 1 + 2 ** -10
    assert _round_tf32(np.float32(-(1 + 2 ** -11))) == -(1 + 2 ** -10)
    assert _round_tf32(np.float32(1 + 2 ** -12)) == 1.0


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
@pytest.mark.parametrize("H,W,ks,nk", [(64, 64, 7, 48), (45, 70, 5, 24), (40, 33, 3, 4)])
def test_stage_equals_fp64_on_rounded_operands(algo, H, W, ks, nk):
    p, f = case(H, W, ks, nk, 1, N=1, cfg=170 + H + ks)
    got = _run(p, f, algo)[1, 0]
    ref = _rounded_stage(p, f[0], ROUND[algo])
    assert np.abs(got - ref).max() <= TOL_U_FP32


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
@pytest.mark.parametrize("H,W,ks,nk,T,N", [
    (128, 128, 7, 48, 5, 1),
    (97, 65, 7, 48, 2, 2),
    (7, 7, 7, 48, 2, 1),
    (64, 35, 3, 4, 2, 1),
    (50, 100, 5, 24, 3, 1),
    (45, 200, 7, 48, 1, 1),
])
def test_matches_oracle_within_stated_bound(algo, H, W, ks, nk, T, N):
    p, f = case(H, W, ks, nk, T, N=N, cfg=180 + H)
    got = _run(p, f, algo)
    ref = np.stack([oracle.forward(f[n], p) for n in range(N)], axis=1)
    np.testing.assert_array_equal(got[0], f)
    err = np.abs(got - ref).max(axis=(1, 2, 3))
    tol, psnr = TOL[algo]
    assert np.all(err <= tol), err
    assert _psnr(got[-1], ref[-1]) >= psnr


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
def test_repeatable_bits_and_final_only(algo):
    p, f = case(80, 90, 7, 48, 3, cfg=190)
    a = _run(p, f, algo, keep=True)
    b = _run(p, f, algo, keep=False)
    c = _run(p, f, algo, keep=False)
    np.testing.assert_array_equal(a[-1], b)
    np.testing.assert_array_equal(b, c)


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
def test_full_size_2048_T8_sampled_windows(algo):
    """One 2048 x 2048 image of the mixed-precision workload (L=2, 7x7x48, T=8)
    in the launch the benchmark times; the oracle computes sampled pixels on
    crops the crop edge cannot reach (radius 2R T = 48)."""
    H = W = 2048
    T = 8
    p, f = case(H, W, 7, 48, T, L=2, cfg=5)
    got = _run(p, f, algo, keep=False)[0]
    M = 2 * 3 * T
    g = np.random.Generator(np.random.PCG64(11))
    pts = [(0, 0), (2047, 2047), (0, 1024), (1500, 0), (3, 2044)]
    pts += [tuple(x) for x in g.integers(0, 2048, size=(6, 2))]
    errs = []
    for (y, x) in pts:
        y0, y1, x0, x1 = crop_window(H, W, y, x, M)
        ref = oracle.forward(f[0, y0:y1, x0:x1], p)[-1][y - y0, x - x0]
        errs.append(abs(got[y, x] - ref))
    assert max(errs) <= TOL[algo][0], errs


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
@pytest.mark.parametrize("nb", ["2", "3"])
def test_both_tile_heights_within_bound(algo, nb, monkeypatch):
    """Tiles of 2 and 3 row blocks (TNRD_TC_NB; the defaults are 2 for TF32, 3 for
    BF16) on a ragged multi-tile image: every stage within the stated bound."""
    monkeypatch.setenv("TNRD_TC_NB", nb)
    p, f = case(101, 83, 7, 48, 2, N=1, cfg=197)
    got = _run(p, f, algo)
    ref = oracle.forward(f[0], p)[:, None]
    err = np.abs(got - ref).max(axis=(1, 2, 3))
    assert np.all(err <= TOL[algo][0]), err
