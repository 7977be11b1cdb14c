"""Shared helpers of the tests: seeded cases, rounded once to float32 so that the
CUDA path and the FP64 oracle see bit-identical inputs."""
from __future__ import annotations

import numpy as np

import synth

# Tolerances (FP32 path vs FP64 oracle).  Values live on a [0, 255] scale
# (speckled inputs reach a few thousand); the bound is absolute on u.
TOL_U_FP32 = 1e-3


def case(H, W, ks, nk, T, L=1, N=1, cfg=100, seed_params=None):
    """(params, f[N][H][W]) with every value exactly representable in float32."""
    p = synth.params(T, ks, nk, seed=synth.seed_for(cfg, 0, "params") if seed_params is None
                     else seed_params)
    p = synth.Params(p.filters.astype(np.float32).astype(np.float64),
                     p.rbf_w.astype(np.float32).astype(np.float64),
                     p.lam.astype(np.float32).astype(np.float64))
    fs = []
    for n in range(N):
        _, f = synth.single_image(H, W, L, cfg, index=n)
        fs.append(f.astype(np.float32).astype(np.float64))
    return p, np.stack(fs)


def crop_window(H, W, y, x, M):
    """Rows/cols of the crop around (y, x) whose centre value the oracle can
    compute exactly: stage t changes values at most 2R away, so after T stages
    only pixels within M = 2RT of an artificial (non-image) crop edge differ."""
    y0, y1 = max(0, y - M), min(H, y + M + 1)
    x0, x1 = max(0, x - M), min(W, x + M + 1)
    return y0, y1, x0, x1
