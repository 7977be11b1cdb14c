"""torch.autograd binding of the TRDMD cascade.

`TNRDFunction.apply(f, filters, rbf_w, lam, mu0, delta, gamma, data_term,
proj_c, algo)` runs the forward cascade (tnrd_forward, keeping u_0..u_T as
checkpoints) and, in backward, the library's gradient kernels (tnrd_backward).
`algo` picks the forward's stage kernels: "fused" (FP32), "tf32x3" (the
tensor-core filter bank and adjoint at FP32 accuracy), or "tf32" / "bf16"
(tensor-core filter bank and adjoint with TF32 / BF16 operands); `bwd_algo` the
backward's ("fused", or "tf32x3" / "tf32": its adjoint on the tensor cores;
by default "tf32x3" after a "tf32x3" forward and "fused" otherwise).  The
backward differentiates the cascade at the checkpoints the forward wrote.  The noisy input f
is data: it gets no gradient.  Training lambda through lam = exp(beta) (Sec.
3.2, Eq. derv5) is plain torch: pass beta.exp() as `lam`.
"""
from __future__ import annotations

import torch

from . import binding as B
from . import ops


class TNRDFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, filters, rbf_w, lam, mu0=-310.0, delta=10.0, gamma=10.0, data_term=0,
                proj_c=1.0, algo="fused", bwd_algo=None):
        model = ops.Model(filters.detach().contiguous(), rbf_w.detach().contiguous(),
                          lam.detach().contiguous(), float(mu0), float(delta), float(gamma),
                          int(data_term), float(proj_c))
        W = f.shape[-1]
        fp = ops.to_pitched(f.detach())
        u_all = ops.forward(model, fp, keep_stages=True, algo=algo, W=W)
        ctx.model = model
        ctx.W = W
        ctx.bwd_algo = bwd_algo or ("tf32x3" if algo == "tf32x3" else "fused")
        ctx.save_for_backward(fp, u_all)
        out = u_all[-1][..., :W]
        return out if f.dim() == 3 else out[0]

    @staticmethod
    def backward(ctx, grad_out):
        fp, u_all = ctx.saved_tensors
        W = ctx.W
        g = grad_out if grad_out.dim() == 3 else grad_out.unsqueeze(0)
        gp = ops.to_pitched(g.contiguous().float())
        if gp.shape[-1] != fp.shape[-1]:
            gp = torch.nn.functional.pad(gp, (0, fp.shape[-1] - gp.shape[-1]))
        _, gk, gw, gl = ops.backward(ctx.model, fp, u_all, gp, want_grad_u0=False, W=W,
                                     algo=ctx.bwd_algo)
        return None, gk, gw, gl, None, None, None, None, None, None, None


def trdmd(f, filters, rbf_w, lam, mu0=-310.0, delta=10.0, gamma=10.0, data_term=0, proj_c=1.0,
          algo="fused", bwd_algo=None):
    """u_T of the T-stage cascade, differentiable in filters, rbf_w and lam
    (data_term as tnrd_data_term: 0 despeckling prox, 1 Gaussian, 2 projection;
    algo the forward's stage kernels: "fused", "tf32x3", "tf32" or "bf16";
    bwd_algo the backward's, see TNRDFunction)."""
    return TNRDFunction.apply(f, filters, rbf_w, lam, mu0, delta, gamma, data_term, proj_c,
                              algo, bwd_algo)
