"""Torch-facing calls of the TRDMD library: marshal tensors, call the C ABI.

PyTorch supplies device memory and streams only; every arithmetic step of the
stage runs in libtnrd.so's kernels.  Images are float32 [N][H][W] (or [H][W])
CUDA tensors; rows are padded to a multiple of 4 floats when W is not.
"""
from __future__ import annotations

import dataclasses

import torch

from . import binding as B


@dataclasses.dataclass
class Model:
    """Parameters of a T-stage TRDMD model, held as device float32 tensors.

    filters [T][nfilt][ks][ks], rbf_w [T][nfilt][nrbf], lam [T] (lambda_t >= 0);
    RBF centres mu_j = mu0 + j * delta, width gamma; data_term 0 (despeckling
    prox), 1 (TNRD Gaussian reaction) or 2 (explicit step with projection at
    proj_c), as tnrd_data_term.
    """
    filters: torch.Tensor
    rbf_w: torch.Tensor
    lam: torch.Tensor
    mu0: float = -310.0
    delta: float = 10.0
    gamma: float = 10.0
    data_term: int = 0
    proj_c: float = 1.0

    @staticmethod
    def create(filters, rbf_w, lam, mu0=-310.0, delta=10.0, gamma=10.0, device="cuda",
               data_term=0, proj_c=1.0):
        t = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
        return Model(t(filters), t(rbf_w), t(lam), float(mu0), float(delta), float(gamma),
                     int(data_term), float(proj_c))

    @property
    def T(self):
        return self.filters.shape[0]

    @property
    def nfilt(self):
        return self.filters.shape[1]

    @property
    def ksize(self):
        return self.filters.shape[2]

    @property
    def nrbf(self):
        return self.rbf_w.shape[2]

    def params(self) -> B.tnrd_params:
        return B.make_params(self)


def pitch_for(W: int) -> int:
    return (W + 3) // 4 * 4


def to_pitched(x: torch.Tensor) -> torch.Tensor:
    """[N][H][W] float32 CUDA tensor -> contiguous [N][H][pitch] (copy only if needed)."""
    if x.dim() == 2:
        x = x.unsqueeze(0)
    N, H, W = x.shape
    P = pitch_for(W)
    if P == W and x.is_contiguous() and x.dtype == torch.float32:
        return x
    out = torch.zeros((N, H, P), dtype=torch.float32, device=x.device)
    out[:, :, :W] = x
    return out


def workspace_size(model: Model, N, H, W, pitch, keep_stages, algo="fused", op=B.OP_FORWARD):
    return B.tnrd_workspace_size(op, model.params(), N, H, W, pitch, int(keep_stages),
                                 B.ALGO[algo])


def forward(model: Model, f: torch.Tensor, keep_stages: bool = False, algo: str = "fused",
            out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
            W: int | None = None) -> torch.Tensor:
    """Runs the T-stage cascade from u_0 = f.

    Returns u_T as [N][H][pitch] (keep_stages False) or all u_0..u_T as
    [T+1][N][H][pitch] (keep_stages True).  `W` is the true width when f is
    already pitched.
    """
    squeeze = f.dim() == 2
    if W is None:
        W = f.shape[-1]
        fp = to_pitched(f)
    else:
        fp = f if f.dim() == 3 else f.unsqueeze(0)
    N, H, P = fp.shape
    p = model.params()
    shape = (model.T + 1, N, H, P) if keep_stages else (N, H, P)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=fp.device)
    ws_bytes = B.tnrd_workspace_size(B.OP_FORWARD, p, N, H, W, P, int(keep_stages), B.ALGO[algo])
    if workspace is None and ws_bytes:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=fp.device)
    stream = torch.cuda.current_stream(fp.device).cuda_stream
    B.tnrd_forward(p, N, H, W, P, fp, out, int(keep_stages), B.ALGO[algo], workspace,
                   ws_bytes, stream)
    if squeeze and not keep_stages:
        return out[0]
    return out


def forward_band(model: Model, f: torch.Tensor, world: int, rank: int, algo: str = "fused"):
    """u_T of this rank's row band of one image f ([H][W] float32 CUDA), from
    the cascade on the band plus its ghost rows (shard.band_rows).  Returns
    (rows [own1 - own0][W], own0, own1).  No exchange between ranks."""
    from .shard import band_rows
    H, W = f.shape[-2], f.shape[-1]
    own0, own1, g0, g1 = band_rows(H, world, rank, model.ksize, model.T)
    if own1 <= own0:
        return f.new_empty((0, W)), own0, own1
    u = forward(model, f[..., g0:g1, :].contiguous(), algo=algo)
    return u[..., own0 - g0:own1 - g0, :W].reshape(own1 - own0, W), own0, own1


def backward(model: Model, f: torch.Tensor, u_stages: torch.Tensor, grad_uT: torch.Tensor,
             want_grad_u0: bool = True, W: int | None = None, workspace=None,
             algo: str = "fused"):
    """Gradients (grad_u0, grad_filters, grad_rbf_w, grad_lambda) given dL/du_T.

    f [N][H][pitch], u_stages [T+1][N][H][pitch], grad_uT [N][H][pitch].  algo
    "fused": every kernel on the CUDA cores; "tf32x3" / "tf32": the adjoint
    dL/du_{t-1} = d + sum_i K_i^T c_i on the tensor cores (split TF32 for FP32
    accuracy, or TF32).
    """
    N, H, P = f.shape
    if W is None:
        W = P
    p = model.params()
    dev = f.device
    g_u0 = torch.empty((N, H, P), dtype=torch.float32, device=dev) if want_grad_u0 else None
    g_k = torch.empty_like(model.filters)
    g_w = torch.empty_like(model.rbf_w)
    g_l = torch.empty_like(model.lam)
    ws_bytes = B.tnrd_workspace_size(B.OP_BACKWARD, p, N, H, W, P, 1, B.ALGO[algo])
    if workspace is None and ws_bytes:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    B.tnrd_backward(p, N, H, W, P, f, u_stages, grad_uT, g_u0, g_k, g_w, g_l,
                    B.ALGO[algo], workspace, ws_bytes, stream)
    return g_u0, g_k, g_w, g_l


def quality(img: torch.Tensor, ref: torch.Tensor | None = None, noisy: torch.Tensor | None = None,
            peak: float = 255.0, W: int | None = None) -> torch.Tensor:
    """Quality indexes of Sec. 4 (tnrd_quality) of images [N][H][W] (or pitched
    [N][H][pitch] with W given): a float64 CUDA tensor [N][6] whose columns are
    binding.QUALITY_NAMES (psnr, mssim, ec, ri_mean, ri_var, cv).  ref and
    noisy are optional (their indexes are NaN without them)."""
    if img.dim() == 2:
        img = img.unsqueeze(0)
        ref = None if ref is None else ref.unsqueeze(0)
        noisy = None if noisy is None else noisy.unsqueeze(0)
    W = img.shape[-1] if W is None else W
    imgp = img if (W is not None and img.shape[-1] % 4 == 0) else to_pitched(img)
    pitch = imgp.shape[-1]
    pad = lambda t: None if t is None else (t if t.shape[-1] == pitch else to_pitched(t))
    refp, noisyp = pad(ref), pad(noisy)
    N, H = imgp.shape[0], imgp.shape[1]
    out = torch.empty((N, B.QUALITY_COUNT), dtype=torch.float64, device=img.device)
    nb = B.tnrd_quality_workspace_size(N, H, W)
    ws = torch.empty(nb, dtype=torch.uint8, device=img.device)
    B.tnrd_quality(refp, imgp.contiguous(), noisyp, N, H, W, pitch, peak, out, ws, nb,
                   torch.cuda.current_stream(img.device).cuda_stream)
    return out
