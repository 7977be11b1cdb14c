"""Seeded synthetic inputs for the TRDMD despeckling stage.

This module only draws inputs: clean piecewise-smooth images, Gamma speckle and
random stage parameters.  It holds none of the method's arithmetic, and both the
CUDA path and the FP64 oracle consume what it returns.

The paper trains and tests on natural-image crops (400 BSDS 256x256 crops, 68
test images; Sec. 4) and on real SAR scenes, none of which are available here.
These generators stand in for them with the shapes of the paper's workloads:

* clean image: a linear ramp plus random axis-aligned rectangles and ellipses of
  constant intensity in [1, 255] (piecewise smooth, strong edges), clamped to
  [1, 255];
* speckle: f = u * n with n i.i.d. Gamma(shape L, scale 1/L), i.e. mean 1
  (the multiplicative model of Eq. (mul));
* parameters per stage: k x k filters drawn N(0,1), projected to zero mean and
  unit L2 norm (zero-mean filters, Sec. 2.2.1); RBF weights N(0, 0.1^2);
  lambda_t = 0.5 t; RBF centres mu_j = -310 + 10 j, j = 0..62, width 10.

All draws use numpy's PCG64 generator seeded from an integer.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 1702_07482

RBF_MU0 = -310.0
RBF_DELTA = 10.0
RBF_GAMMA = 10.0
RBF_N = 63


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def clean_image(H: int, W: int, seed: int) -> np.ndarray:
    """Piecewise-smooth clean image in [1, 255], float64 [H][W]."""
    g = _rng(seed)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64),
                         np.arange(W, dtype=np.float64), indexing="ij")
    img = 40.0 + 60.0 * xx / max(W, 1) + 40.0 * yy / max(H, 1)
    n_shapes = int(np.ceil(20.0 * H * W / (256.0 * 256.0)))
    for s in range(n_shapes):
        cy = g.uniform(0, H)
        cx = g.uniform(0, W)
        hy = 0.5 * g.uniform(0.05, 0.40) * H
        hx = 0.5 * g.uniform(0.05, 0.40) * W
        val = g.uniform(1.0, 255.0)
        # only the shape's bounding box can hold pixels of the shape
        r0, r1 = max(0, int(np.floor(cy - hy)) - 1), min(H, int(np.ceil(cy + hy)) + 2)
        c0, c1 = max(0, int(np.floor(cx - hx)) - 1), min(W, int(np.ceil(cx + hx)) + 2)
        if r0 >= r1 or c0 >= c1:
            continue
        by, bx = yy[r0:r1, c0:c1], xx[r0:r1, c0:c1]
        if s % 2 == 0:
            m = (np.abs(by - cy) <= hy) & (np.abs(bx - cx) <= hx)
        else:
            m = ((by - cy) / hy) ** 2 + ((bx - cx) / hx) ** 2 <= 1.0
        img[r0:r1, c0:c1][m] = val
    return np.clip(img, 1.0, 255.0)


def gaussian_noise(clean: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Noisy observation f = clean + n, n ~ N(0, sigma^2) i.i.d. (the Gaussian
    denoising task of TNRD)."""
    return clean + _rng(seed).normal(0.0, float(sigma), size=clean.shape)


def speckle(clean: np.ndarray, L: float, seed: int) -> np.ndarray:
    """Noisy observation f = clean * n, n ~ Gamma(L, 1/L) i.i.d."""
    g = _rng(seed)
    n = g.gamma(shape=float(L), scale=1.0 / float(L), size=clean.shape)
    return clean * n


@dataclasses.dataclass
class Params:
    """Stage parameters of a T-stage cascade (float64 arrays)."""
    filters: np.ndarray   # [T][nk][ks][ks]
    rbf_w: np.ndarray     # [T][nk][nrbf]
    lam: np.ndarray       # [T]
    mu0: float = RBF_MU0
    delta: float = RBF_DELTA
    gamma: float = RBF_GAMMA
    dterm: int = 0          # data term: 0 despeckling prox, 1 Gaussian, 2 projection
    proj_c: float = 1.0     # floor of the projection variant

    @property
    def T(self) -> int:
        return self.filters.shape[0]

    @property
    def nk(self) -> int:
        return self.filters.shape[1]

    @property
    def ks(self) -> int:
        return self.filters.shape[2]

    @property
    def nrbf(self) -> int:
        return self.rbf_w.shape[2]

    def astype(self, dt) -> "Params":
        return Params(self.filters.astype(dt), self.rbf_w.astype(dt),
                      self.lam.astype(dt), self.mu0, self.delta, self.gamma, self.dterm,
                      self.proj_c)


def params(T: int, ks: int, nk: int, seed: int, nrbf: int = RBF_N,
           w_sigma: float = 0.1, lam_step: float = 0.5) -> Params:
    """Random stage parameters with zero-mean, unit-norm filters."""
    g = _rng(seed)
    k = g.standard_normal((T, nk, ks, ks))
    k -= k.mean(axis=(2, 3), keepdims=True)
    k /= np.sqrt((k * k).sum(axis=(2, 3), keepdims=True))
    w = g.normal(0.0, w_sigma, size=(T, nk, nrbf))
    lam = lam_step * np.arange(1, T + 1, dtype=np.float64)
    return Params(k, w, lam)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random array, for adjoint tests and loss gradients."""
    return _rng(seed).uniform(lo, hi, size=shape)


# ---------------------------------------------------------------------------
# The five workloads of the benchmark table, by shape.
# ---------------------------------------------------------------------------

def seed_for(cfg: int, index: int, kind: str = "image") -> int:
    off = {"image": 0, "noise": 200_000, "params": 500}[kind]
    return SEED_BASE + 1000 * cfg + off + index


def single_image(H: int, W: int, L: float, cfg: int, index: int = 0):
    """(clean, noisy) pair for one image of a workload."""
    c = clean_image(H, W, seed_for(cfg, index, "image"))
    f = speckle(c, L, seed_for(cfg, index, "noise"))
    return c, f


def uneven_batch(n: int, lo: int, hi: int, cfg: int = 3, looks=(1, 2, 4, 8)):
    """Sizes and look numbers of an uneven batch: side lengths U[lo, hi]
    drawn independently for H and W, looks cycling in equal groups."""
    g = _rng(seed_for(cfg, 0, "params") + 77)
    H = g.integers(lo, hi + 1, size=n)
    W = g.integers(lo, hi + 1, size=n)
    per = n // len(looks)
    L = np.array([looks[min(i // per, len(looks) - 1)] for i in range(n)])
    return [(int(h), int(w), int(l)) for h, w, l in zip(H, W, L)]
