"""Pins of the oracle's losses (Eq. 3: L_rgb + lambda L_ssim)."""
import numpy as np
import pytest
from scipy.ndimage import convolve


def test_l1_closed_form(oracle):
    rng = np.random.default_rng(0)
    a, b = rng.uniform(size=(3, 5, 7)), rng.uniform(size=(3, 5, 7))
    L, g = oracle.l1(a, b)
    assert L == pytest.approx(np.abs(a - b).sum() / a.size)
    np.testing.assert_array_equal(g, np.sign(a - b) / a.size)


def test_ssim_of_identical_images_is_one(oracle):
    rng = np.random.default_rng(1)
    a = rng.uniform(size=(3, 20, 24))
    s, g = oracle.ssim(a, a)
    assert s == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(g, 0.0, atol=1e-12)


def test_ssim_window_and_moments_by_direct_convolution(oracle):
    """Window = normalised 11-tap Gaussian, sigma 1.5; local means by a direct
    2D zero-padded convolution with the outer-product window."""
    w = oracle.gaussian_window()
    ax = np.arange(11) - 5
    want = np.exp(-ax ** 2 / 4.5); want /= want.sum()
    np.testing.assert_allclose(w, want, rtol=1e-15)
    rng = np.random.default_rng(2)
    a = rng.uniform(size=(1, 17, 19))
    W2 = np.outer(w, w)
    np.testing.assert_allclose(oracle._filt(a, w)[0], convolve(a[0], W2, mode="constant"), atol=1e-14)


def test_ssim_gradient_by_differences(oracle):
    rng = np.random.default_rng(3)
    a = rng.uniform(size=(3, 13, 15))
    b = np.clip(a + rng.normal(0, 0.2, a.shape), 0, 1)
    s, g = oracle.ssim(a, b)
    h = 1e-6
    for _ in range(40):
        idx = tuple(rng.integers(0, n) for n in a.shape)
        ap, am = a.copy(), a.copy()
        ap[idx] += h; am[idx] -= h
        fd = (oracle.ssim(ap, b)[0] - oracle.ssim(am, b)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_dssim_loss_combination(oracle):
    rng = np.random.default_rng(4)
    a, b = rng.uniform(size=(3, 12, 12)), rng.uniform(size=(3, 12, 12))
    L, g = oracle.dssim_loss(a, b, 0.2)
    l1, g1 = oracle.l1(a, b)
    s, gs = oracle.ssim(a, b)
    assert L == pytest.approx(0.8 * l1 + 0.2 * (1 - s))
    np.testing.assert_allclose(g, 0.8 * g1 - 0.2 * gs)
