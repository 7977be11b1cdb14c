"""Training loop of TRDMD models (Sec. 3.2, Eqs. learning and iterstep).

The parameters Theta_t = {lambda_t, phi_i^t, k_i^t} of all stages minimise the
loss of Eq. learning, sum_s 1/2 |u_T^s - u_gt^s|^2, over a set of
(noisy, clean) pairs.  As in the paper (and TNRD, on which Sec. 3.2 builds)
the stages are first trained greedily -- stage t alone on the loss of u_t,
with stages 1 .. t-1 fixed at their greedy values -- and then jointly on the
loss of u_T.  Gradients come from the library's backward kernels through
`autograd.trdmd`; this module only holds the parameterisation and the
optimiser loop:

* lambda_t = exp(beta_t) (Eq. derv5), so lambda stays positive;
* k_i = theta_i - mean(theta_i): zero-mean filters (Sec. 2.2.1) without a
  constraint, the projection differentiated by torch;
* phi_i's RBF weights w_ij trained directly.

Optimisers: torch's Adam or L-BFGS (the paper's choice for TNRD-type models).
Every forward and backward stage runs in libtnrd.so; torch only updates the
few thousand parameters.  Under torch.distributed each rank passes its own
crops, and the parameter gradients are summed over the ranks after every
backward (one all-reduce), so all ranks take the same step.
"""
from __future__ import annotations

import dataclasses

import torch

from . import autograd
from .shard import allreduce_gradients


@dataclasses.dataclass
class Params:
    """Unconstrained trainable parameters of a T-stage model."""
    theta: torch.Tensor    # [T][nfilt][ks][ks]  filters before the zero-mean projection
    w: torch.Tensor        # [T][nfilt][nrbf]    RBF weights
    beta: torch.Tensor     # [T]                 log lambda
    mu0: float = -310.0
    delta: float = 10.0
    gamma: float = 10.0
    data_term: int = 0       # tnrd_data_term of the model
    proj_c: float = 1.0

    @staticmethod
    def from_model(filters, rbf_w, lam, mu0=-310.0, delta=10.0, gamma=10.0, device="cuda",
                   data_term=0, proj_c=1.0):
        t = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).clone().contiguous()
        lam_t = t(lam)
        if torch.any(lam_t <= 0):
            raise ValueError("lambda must be positive (lambda = exp(beta))")
        return Params(t(filters).requires_grad_(), t(rbf_w).requires_grad_(),
                      lam_t.log().requires_grad_(), float(mu0), float(delta), float(gamma),
                      int(data_term), float(proj_c))

    @property
    def T(self) -> int:
        return self.theta.shape[0]

    def filters(self, stages=None) -> torch.Tensor:
        th = self.theta if stages is None else self.theta[stages]
        return th - th.mean(dim=(-2, -1), keepdim=True)

    def lam(self, stages=None) -> torch.Tensor:
        return (self.beta if stages is None else self.beta[stages]).exp()

    def weights(self, stages=None) -> torch.Tensor:
        return self.w if stages is None else self.w[stages]

    def tensors(self):
        return [self.theta, self.w, self.beta]

    def detached(self):
        """(filters, rbf_w, lam) as plain tensors, e.g. for ops.Model.create."""
        with torch.no_grad():
            return self.filters().clone(), self.w.detach().clone(), self.lam().clone()


def save(p: Params, path: str) -> None:
    """Writes the trainable parameters (theta, w, beta: the unconstrained
    values, so training resumes exactly) and the model constants to an .npz
    archive; one file per model (e.g. per number of looks L)."""
    import numpy as np
    np.savez(path, theta=p.theta.detach().cpu().numpy(), w=p.w.detach().cpu().numpy(),
             beta=p.beta.detach().cpu().numpy(),
             consts=np.array([p.mu0, p.delta, p.gamma, p.proj_c], dtype=np.float64),
             data_term=np.array(p.data_term, dtype=np.int64))


def load(path: str, device="cuda") -> Params:
    """Reads an archive written by save(): the same values, trainable again."""
    import numpy as np
    with np.load(path) as z:
        t = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).clone().requires_grad_()
        mu0, delta, gamma, proj_c = (float(v) for v in z["consts"])
        return Params(t(z["theta"]), t(z["w"]), t(z["beta"]), mu0, delta, gamma,
                      int(z["data_term"]), proj_c)


def loss_sum(u: torch.Tensor, clean: torch.Tensor) -> torch.Tensor:
    """Eq. learning: sum over samples and pixels of 1/2 (u - u_gt)^2."""
    return 0.5 * ((u - clean) ** 2).sum()


def cascade(p: Params, f: torch.Tensor, stages: int | None = None,
            algo: str = "fused") -> torch.Tensor:
    """u_t after the first `stages` stages (all T by default), differentiable;
    `algo` the forward's stage kernels ("fused", "tf32", "bf16")."""
    sl = slice(0, p.T if stages is None else stages)
    return autograd.trdmd(f, p.filters(sl).contiguous(), p.weights(sl).contiguous(),
                          p.lam(sl).contiguous(), p.mu0, p.delta, p.gamma, p.data_term,
                          p.proj_c, algo)


def _make_opt(tensors, optimizer: str, lr: float):
    if optimizer == "adam":
        return torch.optim.Adam(tensors, lr=lr)
    if optimizer == "lbfgs":
        return torch.optim.LBFGS(tensors, lr=lr, max_iter=1, history_size=20,
                                 line_search_fn="strong_wolfe")
    raise ValueError(f"unknown optimizer {optimizer!r}")


def _run(p: Params, f, clean, stages: int, steps: int, optimizer: str, lr: float,
         trainable_mask=None, history=None, tag=""):
    """`steps` optimiser iterations on the loss of u_stages.  trainable_mask[t]
    False freezes stage t (its gradient is zeroed before each update)."""
    opt = _make_opt(p.tensors(), optimizer, lr)
    npx = clean.numel()

    def closure():
        opt.zero_grad(set_to_none=False)
        loss = loss_sum(cascade(p, f, stages), clean)
        loss.backward()
        allreduce_gradients(p.tensors())     # data-parallel ranks: sum of the batch's gradients
        if trainable_mask is not None:
            with torch.no_grad():
                for g in (p.theta.grad, p.w.grad, p.beta.grad):
                    if g is not None:
                        g[~trainable_mask] = 0
        return loss

    for it in range(steps):
        loss = opt.step(closure)
        if history is not None:
            history.append((tag, it, float(loss.detach()) / npx * 2.0))   # per-pixel MSE
    return history


def fit(p: Params, f: torch.Tensor, clean: torch.Tensor, greedy_steps: int = 0,
        joint_steps: int = 0, optimizer: str = "adam", lr: float = 1e-3):
    """Greedy stage-wise training (greedy_steps iterations per stage), then
    joint training of all stages (joint_steps iterations).  f and clean are
    float32 CUDA tensors [N][H][W].  Returns the history as a list of
    (phase, iteration, per-pixel MSE before the update)."""
    if f.shape != clean.shape:
        raise ValueError("f and clean differ in shape")
    history = []
    if greedy_steps > 0:
        for t in range(1, p.T + 1):
            mask = torch.zeros(p.T, dtype=torch.bool, device=p.beta.device)
            mask[t - 1] = True
            _run(p, f, clean, t, greedy_steps, optimizer, lr, mask, history, f"greedy{t}")
    if joint_steps > 0:
        _run(p, f, clean, p.T, joint_steps, optimizer, lr, None, history, "joint")
    return history
