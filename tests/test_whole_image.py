"""Whole-image parity at the benchmark configurations: every pixel of every
stage u_1 .. u_T of the GPU cascade against the FP64 oracle (Eq. diffusion with
the stage of Eq. diffusionprocessfinal), in the launch configurations the
benchmark times.

* 512 x 512, L = 1, 7x7x48, T = 5, plain FP32 (the fused stage kernel that
  tnrd_forward picks for one image of this size: column pairs on two-CTA
  clusters, short border tile rows): max |du| <= 1e-3 on [0, 255].
* 1024 x 1024, L = 2, 7x7x48, T = 8, tensor-core stages (TF32 and BF16 operands,
  FP32 accumulation, phi and prox in FP32): the stated bounds max |du| <= 0.02
  (TF32) / 0.2 (BF16) for every stage and PSNR(u_T) >= 100 / 85 dB; split TF32
  operands (three products): the FP32 bound 1e-3 and PSNR >= 130 dB.
* 512 x 512, T = 5 with split TF32 operands: the FP32 bound at every stage.

The oracle runs once per image (all cores; about 10 s and 1 min on 16 cores)."""
import numpy as np
import pytest
import torch

import oracle
from _cases import TOL_U_FP32, case

pytestmark = pytest.mark.gpu

TOL_TC = {"tf32": (0.02, 100.0), "bf16": (0.2, 85.0),   # (max |du|, min PSNR dB)
          "tf32x3": (TOL_U_FP32, 130.0)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _gpu_stages(p, f, algo):
    from paper_1702_07482_gb300 import binding, ops
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    ft = ops.to_pitched(torch.tensor(f, dtype=torch.float32, device="cuda"))
    u = ops.forward(m, ft, keep_stages=True, algo=algo, W=f.shape[-1])
    torch.cuda.synchronize()
    assert binding.tnrd_device_status() == 0
    return u[..., :f.shape[-1]].double().cpu().numpy()[:, 0]


def _psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10 * np.log10(255.0 ** 2 / max(mse, 1e-30))


def test_whole_512_T5_fp32_every_stage():
    p, f = case(512, 512, 7, 48, 5, L=1, cfg=2)
    got = _gpu_stages(p, f, "fused")
    ref = oracle.forward(f[0], p)
    np.testing.assert_array_equal(got[0], f[0])
    err = np.abs(got - ref).max(axis=(1, 2))
    assert np.all(err <= TOL_U_FP32), err


@pytest.fixture(scope="module")
def _case_1024():
    p, f = case(1024, 1024, 7, 48, 8, L=2, cfg=5)
    return p, f, oracle.forward(f[0], p)


@pytest.mark.parametrize("algo", ["tf32", "bf16", "tf32x3"])
def test_whole_1024_T8_tensor_core_every_stage(algo, _case_1024):
    p, f, ref = _case_1024
    got = _gpu_stages(p, f, algo)
    np.testing.assert_array_equal(got[0], f[0])
    err = np.abs(got - ref).max(axis=(1, 2))
    tol, psnr = TOL_TC[algo]
    assert np.all(err <= tol), err
    assert _psnr(got[-1], ref[-1]) >= psnr


def test_whole_512_T5_split_tf32_every_stage():
    p, f = case(512, 512, 7, 48, 5, L=1, cfg=2)
    got = _gpu_stages(p, f, "tf32x3")
    ref = oracle.forward(f[0], p)
    np.testing.assert_array_equal(got[0], f[0])
    err = np.abs(got - ref).max(axis=(1, 2))
    assert np.all(err <= TOL_U_FP32), err
