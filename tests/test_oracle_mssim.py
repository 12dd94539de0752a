"""Pins of the oracle's MSSIM (Sec. 4.1 quality measure, Wang et al. 2004)."""
import numpy as np
import pytest

import synth_inputs as si

C1 = (0.01 * 255) ** 2
C2 = (0.03 * 255) ** 2


def test_identical_images_give_one(orc):
    img = si.ar1_image(48, 64, 0.9, 1)
    v, m = orc.mssim(img, img, want_map=True)
    assert m.shape == (38, 54)
    assert np.allclose(m, 1.0, atol=1e-12) and v == pytest.approx(1.0, abs=1e-12)


def test_constant_images_closed_form(orc):
    """Flat images a and b: zero variances, so SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    for a, b in ((10, 200), (128, 130), (0, 255)):
        x = np.full((20, 30), a, np.uint8)
        y = np.full((20, 30), b, np.uint8)
        v, _ = orc.mssim(x, y)
        assert v == pytest.approx((2 * a * b + C1) / (a * a + b * b + C1), rel=1e-12)


def test_matches_scipy_gaussian_filter(orc):
    """The same statistics from scipy's separable Gaussian filter (sigma 1.5, 11 taps:
    truncate 3.5 gives radius 5), taken on the positions where the window fits."""
    nd = pytest.importorskip("scipy.ndimage")
    x = si.ar1_image(64, 80, 0.9, 2).astype(np.float64)
    y = np.clip(x + np.random.default_rng(3).normal(0, 12, x.shape), 0, 255).round()
    f = lambda a: nd.gaussian_filter(a, 1.5, truncate=3.5, mode="constant")[5:-5, 5:-5]
    mx, my = f(x), f(y)
    vx, vy, cxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    ref = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    v, m = orc.mssim(x.astype(np.uint8), y.astype(np.uint8), want_map=True)
    assert np.max(np.abs(m - ref)) < 1e-9 and v == pytest.approx(ref.mean(), abs=1e-10)


def test_symmetric_and_below_one(orc):
    x = si.ar1_image(40, 40, 0.8, 4)
    y = si.ar1_image(40, 40, 0.8, 5)
    a, _ = orc.mssim(x, y)
    b, _ = orc.mssim(y, x)
    assert a == pytest.approx(b, abs=1e-14) and a < 1.0


def test_too_small_is_nan(orc):
    v, _ = orc.mssim(np.zeros((10, 40), np.uint8), np.zeros((10, 40), np.uint8))
    assert np.isnan(v)
