"""Pins of the quality-index oracle (oracle/quality.py, Sec. 4) against library
routines, closed forms and the ideal values the paper states."""
import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

import synth
from oracle import quality as Q


def _img(H, W, seed, lo=20.0, hi=230.0):
    return synth.random_field((H, W), seed, lo, hi)


def test_gaussian_window_is_scipy_window_outer_product():
    g = scipy.signal.windows.gaussian(11, 1.5)
    ref = np.outer(g, g)
    np.testing.assert_allclose(Q.gaussian_window(), ref / ref.sum(), rtol=1e-14)


def test_ssim_of_identical_images_is_one():
    x = _img(20, 23, 1)
    np.testing.assert_allclose(Q.ssim_map(x, x), 1.0, rtol=1e-14)
    assert Q.mssim(x, x) == pytest.approx(1.0, rel=1e-14)


def test_ssim_local_statistics_match_scipy_correlation():
    """The window statistics from scipy's 'valid' correlation give the same map."""
    x, y = _img(17, 19, 2), _img(17, 19, 3)
    w = Q.gaussian_window()
    corr = lambda a: scipy.signal.correlate2d(a, w, mode="valid")
    mx, my = corr(x), corr(y)
    sx, sy, sxy = corr(x * x) - mx ** 2, corr(y * y) - my ** 2, corr(x * y) - mx * my
    c1, c2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    ref = (2 * mx * my + c1) * (2 * sxy + c2) / ((mx ** 2 + my ** 2 + c1) * (sx + sy + c2))
    np.testing.assert_allclose(Q.ssim_map(x, y), ref, rtol=1e-12)


def test_ssim_of_a_shifted_image_is_the_luminance_term():
    """y = x + c leaves variances and covariance unchanged: SSIM reduces to
    (2 mx my + C1) / (mx^2 + my^2 + C1) per window."""
    x = _img(15, 15, 4)
    c = 17.0
    m = Q.ssim_map(x, x + c)
    w = Q.gaussian_window()
    mx = scipy.signal.correlate2d(x, w, mode="valid")
    my = mx + c
    c1 = (0.01 * 255) ** 2
    np.testing.assert_allclose(m, (2 * mx * my + c1) / (mx ** 2 + my ** 2 + c1), rtol=1e-12)


def test_ssim_is_symmetric_and_at_most_one():
    x, y = _img(16, 21, 5), _img(16, 21, 6)
    np.testing.assert_allclose(Q.ssim_map(x, y), Q.ssim_map(y, x), rtol=1e-12, atol=1e-12)
    assert Q.ssim_map(x, y).max() <= 1.0


def test_psnr_closed_form():
    x = _img(9, 13, 7)
    assert Q.psnr(x, x + 5.0) == pytest.approx(10 * np.log10(255.0 ** 2 / 25.0), rel=1e-14)


def test_laplacian_matches_scipy_reflect_convolution():
    x = _img(12, 9, 8)
    k = np.array([[0, 1, 0], [1, -4, 1], [0, 1, 0]], dtype=np.float64)
    np.testing.assert_allclose(Q.laplacian(x), scipy.ndimage.convolve(x, k, mode="reflect"),
                               rtol=1e-13, atol=1e-12)


def test_edge_correlation_invariances():
    x, y = _img(25, 30, 9), _img(25, 30, 10)
    assert Q.edge_correlation(x, x) == pytest.approx(1.0, rel=1e-14)
    assert Q.edge_correlation(x, 3.0 * x + 40.0) == pytest.approx(1.0, rel=1e-13)
    assert Q.edge_correlation(x, -x) == pytest.approx(-1.0, rel=1e-13)
    assert abs(Q.edge_correlation(x, y)) < 0.2      # independent fields


def test_ratio_image_of_single_look_amplitude_speckle():
    """RI = f / u for f = u n with n the single-look amplitude (Rayleigh) of
    unit mean: RI_M -> 1 and RI_V -> 4/pi - 1 (the ideal values of Sec. 4)."""
    g = np.random.Generator(np.random.PCG64(11))
    u = _img(400, 500, 12)
    n = g.rayleigh(scale=1.0, size=u.shape)
    n /= np.sqrt(np.pi / 2.0)                        # E[Rayleigh(1)] = sqrt(pi/2)
    m, v = Q.ratio_image_stats(u * n, u)
    se_m, se_v = np.sqrt((4 / np.pi - 1) / n.size), 3.0 / np.sqrt(n.size)
    assert abs(m - 1.0) < 5 * se_m
    assert abs(v - (4 / np.pi - 1)) < 5 * se_v


def test_coefficient_of_variation_closed_form():
    x = np.array([[10.0, 30.0], [10.0, 30.0]])       # mean 20, std 10
    assert Q.coefficient_of_variation(x) == pytest.approx(0.5, rel=1e-15)
    assert Q.coefficient_of_variation(np.full((3, 3), 7.0)) == 0.0
