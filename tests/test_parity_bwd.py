"""GPU parity of the backward kernels (tnrd_backward through the C ABI) with
the FP64 oracle's gradients, which tests/test_oracle.py pins to central finite
differences.

Tolerance per gradient group (filters of a stage, RBF weights of a stage,
lambda, dL/du_0): relative L2 error <= 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
from _cases import case

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1702_07482_gb300 import binding, build
    build.build()
    binding.load()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _gpu_grads(p, f, clean, algo="fused", bwd_algo="fused"):
    from paper_1702_07482_gb300 import ops
    m = ops.Model.create(p.filters, p.rbf_w, p.lam, p.mu0, p.delta, p.gamma)
    W = f.shape[-1]
    fp = ops.to_pitched(torch.tensor(f, dtype=torch.float32, device="cuda"))
    u_all = ops.forward(m, fp, keep_stages=True, algo=algo, W=W)
    ct = ops.to_pitched(torch.tensor(clean, dtype=torch.float32, device="cuda"))
    eT = (u_all[-1] - ct).contiguous()
    g0, gk, gw, gl = ops.backward(m, fp, u_all, eT, want_grad_u0=True, W=W, algo=bwd_algo)
    torch.cuda.synchronize()
    c = lambda t: t.double().cpu().numpy()
    return c(u_all[..., :W]), c(g0[..., :W]), c(gk), c(gw), c(gl)


def _oracle_grads(p, f, clean, u_gpu=None):
    """Oracle gradients of L = sum_n 1/2 |u_T - clean|^2 over the batch."""
    gk = np.zeros_like(p.filters)
    gw = np.zeros_like(p.rbf_w)
    gl = np.zeros_like(p.lam)
    g0 = []
    for n in range(f.shape[0]):
        u_all = oracle.forward(f[n], p)
        e0, k, w, l = oracle.backward(f[n], p, u_all, u_all[-1] - clean[n])
        gk += k
        gw += w
        gl += l
        g0.append(e0)
    return np.stack(g0), gk, gw, gl


def _check(p, f, clean, algo="fused", tol=TOL_GRAD, bwd_algo="fused"):
    _, g0, gk, gw, gl = _gpu_grads(p, f, clean, algo, bwd_algo)
    r0, rk, rw, rl = _oracle_grads(p, f, clean)
    errs = {"u0": _rel(g0, r0), "lam": _rel(gl, rl)}
    for t in range(p.T):
        errs[f"k{t}"] = _rel(gk[t], rk[t])
        errs[f"w{t}"] = _rel(gw[t], rw[t])
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"relative L2 errors above {tol}: {bad}"
    return errs


def test_fd_instance_32x32_3x3x4_T2():
    """The finite-difference instance of the oracle pins (32x32, 3x3x4, T=2)."""
    p, f = case(32, 32, 3, 4, 2, cfg=93)
    p.rbf_w *= 3.0
    clean = np.stack([_clean(32, 32, 93)])
    _check(p, f, clean)


def _clean(H, W, cfg, n=0):
    import synth
    c, _ = synth.single_image(H, W, 1, cfg, index=n)
    return c.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("H,W,ks,nk,T,N", [
    (40, 53, 7, 48, 2, 2),
    (37, 29, 5, 24, 3, 1),
    (70, 33, 7, 48, 1, 1),
])
def test_gradients_match_oracle(H, W, ks, nk, T, N):
    p, f = case(H, W, ks, nk, T, N=N, cfg=140 + H)
    clean = np.stack([_clean(H, W, 140 + H, n) for n in range(N)])
    _check(p, f, clean)


def test_batch_gradient_is_sum_of_image_gradients():
    from paper_1702_07482_gb300 import ops
    p, f = case(45, 45, 7, 48, 2, N=3, cfg=150)
    clean = np.stack([_clean(45, 45, 150, n) for n in range(3)])
    _, _, gk, gw, gl = _gpu_grads(p, f, clean)
    sk, sw, sl = 0, 0, 0
    for n in range(3):
        _, _, k, w, l = _gpu_grads(p, f[n:n + 1], clean[n:n + 1])
        sk, sw, sl = sk + k, sw + w, sl + l
    assert _rel(gk, sk) <= 1e-5 and _rel(gw, sw) <= 1e-5 and _rel(gl, sl) <= 1e-5


def test_repeatable_bits():
    p, f = case(50, 41, 7, 48, 2, cfg=151)
    clean = np.stack([_clean(50, 41, 151)])
    a = _gpu_grads(p, f, clean)
    b = _gpu_grads(p, f, clean)
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)


def test_autograd_matches_backward():
    from paper_1702_07482_gb300 import autograd
    p, f = case(33, 40, 7, 48, 2, cfg=152)
    clean = _clean(33, 40, 152)
    dev = "cuda"
    k = torch.tensor(p.filters, dtype=torch.float32, device=dev, requires_grad=True)
    w = torch.tensor(p.rbf_w, dtype=torch.float32, device=dev, requires_grad=True)
    beta = torch.tensor(np.log(p.lam), dtype=torch.float32, device=dev, requires_grad=True)
    ft = torch.tensor(f[0], dtype=torch.float32, device=dev)
    ct = torch.tensor(clean, dtype=torch.float32, device=dev)
    u = autograd.trdmd(ft, k, w, beta.exp())
    loss = 0.5 * ((u - ct) ** 2).sum()
    loss.backward()
    r0, rk, rw, rl = _oracle_grads(p, f, clean[None])
    assert _rel(k.grad.double().cpu().numpy(), rk) <= TOL_GRAD
    assert _rel(w.grad.double().cpu().numpy(), rw) <= TOL_GRAD
    # Eq. derv5: dL/dbeta = lam dL/dlam
    assert _rel(beta.grad.double().cpu().numpy(), p.lam * rl) <= TOL_GRAD


def test_full_size_180_crop_T5():
    """One 180x180 crop of the training workload, 7x7x48, T=5 (the batch of
    32 differs only in how many such crops are summed)."""
    p, f = case(180, 180, 7, 48, 5, cfg=4)
    clean = np.stack([_clean(180, 180, 4)])
    _check(p, f, clean)


# Mixed-precision training: the forward's filter bank and adjoint on the tensor
# cores (TF32 or BF16 operands, FP32 accumulation), the backward FP32.  The
# gradients are those of the cascade at the checkpoints the forward wrote, so
# they inherit the forward's error.
TOL_GRAD_TC = {"tf32": 1e-3, "bf16": 1e-2}


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
def test_tensor_core_forward_gradients_180_crop_T5(algo):
    p, f = case(180, 180, 7, 48, 5, cfg=4)
    clean = np.stack([_clean(180, 180, 4)])
    _check(p, f, clean, algo, TOL_GRAD_TC[algo])


@pytest.mark.parametrize("algo", ["tf32", "bf16"])
def test_tensor_core_forward_gradients_ragged_batch(algo):
    p, f = case(61, 90, 7, 48, 3, N=2, cfg=161)
    clean = np.stack([_clean(61, 90, 161, n) for n in range(2)])
    _check(p, f, clean, algo, TOL_GRAD_TC[algo])


def test_autograd_tensor_core_forward():
    """autograd.trdmd(algo="tf32") gives the gradients of ops.forward(tf32) +
    ops.backward, bit for bit (same kernels, same order)."""
    from paper_1702_07482_gb300 import autograd
    p, f = case(64, 64, 7, 48, 2, cfg=162)
    clean = _clean(64, 64, 162)
    dev = "cuda"
    k = torch.tensor(p.filters, dtype=torch.float32, device=dev, requires_grad=True)
    w = torch.tensor(p.rbf_w, dtype=torch.float32, device=dev, requires_grad=True)
    lam = torch.tensor(p.lam, dtype=torch.float32, device=dev, requires_grad=True)
    u = autograd.trdmd(torch.tensor(f[0], dtype=torch.float32, device=dev), k, w, lam,
                       algo="tf32")
    (0.5 * ((u - torch.tensor(clean, dtype=torch.float32, device=dev)) ** 2).sum()).backward()
    _, _, gk, gw, gl = _gpu_grads(p, f, clean[None], "tf32")
    np.testing.assert_array_equal(k.grad.double().cpu().numpy(), gk)
    np.testing.assert_array_equal(w.grad.double().cpu().numpy(), gw)
    np.testing.assert_array_equal(lam.grad.double().cpu().numpy(), gl)


# The backward's adjoint on the tensor cores (tc_bwd_adj): split TF32 keeps the
# FP32 bound with every other kernel FP32 (and with the split-TF32 forward);
# TF32 operands in both directions stay within 1e-3 too.
@pytest.mark.parametrize("H,W,ks,nk,T,N", [
    (40, 53, 7, 48, 2, 2),
    (37, 29, 5, 24, 3, 1),
    (70, 33, 7, 48, 1, 1),
    (45, 61, 3, 4, 2, 1),
])
def test_tensor_core_adjoint_gradients(H, W, ks, nk, T, N):
    p, f = case(H, W, ks, nk, T, N=N, cfg=170 + H)
    clean = np.stack([_clean(H, W, 170 + H, n) for n in range(N)])
    _check(p, f, clean, "fused", TOL_GRAD, "tf32x3")


@pytest.mark.parametrize("algo", ["tf32x3", "tf32"])
def test_tensor_core_training_step_180_crop_T5(algo):
    p, f = case(180, 180, 7, 48, 5, cfg=4)
    clean = np.stack([_clean(180, 180, 4)])
    _check(p, f, clean, algo, TOL_GRAD, algo)


def test_tensor_core_adjoint_repeatable_and_close_to_cuda_core():
    """tc_bwd_adj gives the same bits on repeated calls, and with split TF32
    the gradients of the CUDA-core adjoint within FP32 rounding."""
    p, f = case(90, 77, 7, 48, 2, N=2, cfg=175)
    clean = np.stack([_clean(90, 77, 175, n) for n in range(2)])
    a = _gpu_grads(p, f, clean, "fused", "tf32x3")
    b = _gpu_grads(p, f, clean, "fused", "tf32x3")
    c = _gpu_grads(p, f, clean, "fused", "fused")
    for x, y, z in zip(a[1:], b[1:], c[1:]):
        np.testing.assert_array_equal(x, y)
        assert _rel(x, z) <= 1e-5
