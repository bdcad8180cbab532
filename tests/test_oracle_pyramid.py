"""Pins of the FP64 pyramid oracle (CPU only)."""

import numpy as np
import scipy.ndimage as ndi

from oracle import pyramid as pm

B5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0])


def test_downsample_equals_nearest_correlation_then_subsample():
    rng = np.random.default_rng(7)
    for shape in [(1, 1), (3, 2), (8, 8), (17, 9), (20, 33)]:
        img = rng.random(shape)
        ref = ndi.correlate(img, np.outer(B5, B5) / 256.0, mode="nearest")[::2, ::2]
        np.testing.assert_allclose(pm.downsample(img), ref, rtol=0, atol=1e-15)


def _upsample_by_zero_stuffing(coarse, fine_shape):
    # Edge-pad the coarse image by 2, insert zeros between samples, filter with
    # [1,4,6,4,1]/8 along each axis (zero outside), crop the fine window.
    p = np.pad(coarse, 2, mode="edge")
    z = np.zeros((2 * p.shape[0], 2 * p.shape[1]))
    z[::2, ::2] = p
    taps = B5 / 8.0
    z = ndi.correlate1d(z, taps, axis=0, mode="constant", cval=0.0)
    z = ndi.correlate1d(z, taps, axis=1, mode="constant", cval=0.0)
    H, W = fine_shape
    return z[4:4 + H, 4:4 + W]


def test_upsample_equals_zero_stuffing_construction():
    rng = np.random.default_rng(8)
    for fine in [(2, 2), (3, 5), (8, 8), (17, 9), (24, 40)]:
        coarse = rng.random((pm.down_size(fine[0]), pm.down_size(fine[1])))
        np.testing.assert_allclose(pm.upsample(coarse, fine), _upsample_by_zero_stuffing(coarse, fine),
                                   rtol=0, atol=1e-15)


def test_ramps_interior():
    # Binomial downsample of f = x gives 2x; upsample of u[m] = m gives X/2 (away from borders).
    H, W = 24, 32
    ramp = np.tile(np.arange(W, dtype=np.float64), (H, 1))
    d = pm.downsample(ramp)
    np.testing.assert_allclose(d[:, 1:-1], np.tile(2.0 * np.arange(1, W // 2 - 1), (H // 2, 1)), atol=1e-13)
    coarse = np.tile(np.arange(16, dtype=np.float64), (12, 1))
    u = pm.upsample(coarse, (24, 32))
    np.testing.assert_allclose(u[:, 2:-2], np.tile(np.arange(2, 30) / 2.0, (24, 1)), atol=1e-13)


def test_constant_preserved_and_sizes():
    c = np.full((13, 7), 0.25)
    assert np.allclose(pm.downsample(c), 0.25, atol=1e-16, rtol=0)
    assert np.allclose(pm.upsample(c, (26, 13)), 0.25, atol=1e-16, rtol=0)
    w, h = 2560, 1536
    for _ in range(7):
        w, h = pm.down_size(w), pm.down_size(h)
    assert (w, h) == (20, 12)


def test_laplacian_collapse_reconstructs():
    rng = np.random.default_rng(9)
    img = rng.random((37, 45))
    g = pm.gaussian_pyramid(img, 5)
    assert [x.shape for x in g] == [(37, 45), (19, 23), (10, 12), (5, 6), (3, 3)]
    np.testing.assert_allclose(pm.collapse(pm.laplacian_pyramid(g)), img, rtol=0, atol=1e-14)
