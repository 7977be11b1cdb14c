"""FP64 oracle of the despeckling quality indexes (Sec. 4).

TEST INFRASTRUCTURE ONLY: plain numpy restatements of the index definitions
that the CUDA path (tnrd_quality) is checked against.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg use it.

The paper names the indexes and cites their sources without formulas; the
readings used here (also listed in the design notes):

* PSNR = 10 log10(peak^2 / MSE), peak = 255 for the [0, 255] scale.
* MSSIM (Wang, Bovik, Sheikh, Simoncelli 2004): local means, variances and
  covariance under an 11 x 11 Gaussian window (sigma = 1.5, weights summing to
  1), SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2))
  with C1 = (0.01 peak)^2, C2 = (0.03 peak)^2 and s^2 = E_w[x^2] - m^2; MSSIM is
  the mean over the windows that lie inside the image.
* EC (edge correlation): the correlation coefficient of the high-pass
  versions of the reference and the despeckled image, the high pass being the
  3 x 3 Laplacian [0 1 0; 1 -4 1; 0 1 0] with half-sample symmetric borders.
* Ratio image RI = f / u_hat (noisy over despeckled); RI_M its mean, RI_V its
  (population) variance.
* Coefficient of variation C = std / mean (population) of the despeckled image.
"""
from __future__ import annotations

import numpy as np

SSIM_WIN = 11
SSIM_SIGMA = 1.5
SSIM_K1 = 0.01
SSIM_K2 = 0.03


def gaussian_window(n: int = SSIM_WIN, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """n x n Gaussian weights exp(-(dy^2 + dx^2) / (2 sigma^2)), normalised to sum 1."""
    r = n // 2
    d = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def psnr(ref, img, peak: float = 255.0) -> float:
    ref = np.asarray(ref, np.float64)
    img = np.asarray(img, np.float64)
    mse = np.mean((ref - img) ** 2)
    return float(10.0 * np.log10(peak * peak / mse)) if mse > 0 else float("inf")


def ssim_map(x, y, peak: float = 255.0) -> np.ndarray:
    """SSIM of every window that lies inside the image, [H-10][W-10], by a
    direct sum over each window."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window()
    n = SSIM_WIN
    H, W = x.shape
    c1 = (SSIM_K1 * peak) ** 2
    c2 = (SSIM_K2 * peak) ** 2
    out = np.empty((H - n + 1, W - n + 1))
    for i in range(H - n + 1):
        for j in range(W - n + 1):
            px = x[i:i + n, j:j + n]
            py = y[i:i + n, j:j + n]
            mx = np.sum(w * px)
            my = np.sum(w * py)
            sx = np.sum(w * px * px) - mx * mx
            sy = np.sum(w * py * py) - my * my
            sxy = np.sum(w * px * py) - mx * my
            out[i, j] = ((2 * mx * my + c1) * (2 * sxy + c2)) / \
                ((mx * mx + my * my + c1) * (sx + sy + c2))
    return out


def mssim(x, y, peak: float = 255.0) -> float:
    return float(np.mean(ssim_map(x, y, peak)))


def laplacian(x) -> np.ndarray:
    """3 x 3 Laplacian with half-sample symmetric borders (edge pixel repeated)."""
    x = np.asarray(x, np.float64)
    p = np.pad(x, 1, mode="symmetric")
    return p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:] - 4.0 * p[1:-1, 1:-1]


def edge_correlation(ref, img) -> float:
    a = laplacian(ref)
    b = laplacian(img)
    a = a - a.mean()
    b = b - b.mean()
    return float(np.sum(a * b) / np.sqrt(np.sum(a * a) * np.sum(b * b)))


def ratio_image_stats(noisy, img):
    """(RI_M, RI_V) of RI = noisy / img."""
    ri = np.asarray(noisy, np.float64) / np.asarray(img, np.float64)
    m = ri.mean()
    return float(m), float(np.mean((ri - m) ** 2))


def coefficient_of_variation(img) -> float:
    x = np.asarray(img, np.float64)
    m = x.mean()
    return float(np.sqrt(np.mean((x - m) ** 2)) / m)


def indexes(ref, img, noisy, peak: float = 255.0) -> dict:
    """All indexes of one image, as tnrd_quality reports them."""
    rim, riv = ratio_image_stats(noisy, img)
    return {"psnr": psnr(ref, img, peak), "mssim": mssim(ref, img, peak),
            "ec": edge_correlation(ref, img), "ri_mean": rim, "ri_var": riv,
            "cv": coefficient_of_variation(img)}
