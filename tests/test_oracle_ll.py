"""Pins of the FP64 local Laplacian oracle (CPU only)."""

import numpy as np
import scipy.ndimage as ndi

from oracle import local_laplacian as ll
from oracle import pyramid as pm
from paper_2012_07145_gb300 import synth

B5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0])


def test_remap_hand_values():
    # inside the band: g + sign(d) sigma (|d|/sigma)^alpha
    assert abs(ll.remap(0.55, 0.5, 0.1, 0.25, 1.0) - (0.5 + 0.1 * 0.5 ** 0.25)) < 1e-15
    assert abs(ll.remap(0.45, 0.5, 0.1, 0.25, 1.0) - (0.5 - 0.1 * 0.5 ** 0.25)) < 1e-15
    # outside: g + sign(d) (beta (|d| - sigma) + sigma)
    assert abs(ll.remap(0.9, 0.5, 0.1, 0.25, 0.5) - (0.5 + 0.5 * 0.3 + 0.1)) < 1e-15
    assert abs(ll.remap(0.1, 0.5, 0.1, 0.25, 0.5) - (0.5 - 0.5 * 0.3 - 0.1)) < 1e-15
    assert ll.remap(0.5, 0.5, 0.1, 0.25, 0.5) == 0.5
    # alpha = beta = 1 is the identity on both branches
    i = np.linspace(0, 1, 101)
    np.testing.assert_allclose(ll.remap(i, 3 / 7, 0.1, 1.0, 1.0), i, atol=1e-15, rtol=0)


def test_identity_parameters_return_the_input():
    img = synth.rgb_u16_gradient_noise(48, 40, seed=1)
    out = ll.local_laplacian(img, levels=4, k_levels=8, alpha=1.0, beta=1.0)
    assert np.array_equal(out, img)


def test_constant_image_is_unchanged_for_any_parameters():
    img = np.full((3, 16, 24), 30000, dtype=np.uint16)
    out = ll.local_laplacian(img, levels=4, alpha=0.25, beta=0.5)
    assert np.array_equal(out, img)


def test_tiny_sigma_is_the_linear_remap_closed_form():
    # sigma_r -> 0 makes r_k(i) = g_k + beta (i - g_k): every L_l[r_k] = beta L_l[gray], so
    # out_gray = beta * gray + (1 - beta) * (G_{J-1}[gray] upsampled through every level).
    beta = 0.4
    J = 4
    img = synth.rgb_u16_gradient_noise(40, 56, seed=2)
    out = ll.local_laplacian_float(img, levels=J, k_levels=8, sigma_r=1e-9, alpha=0.5, beta=beta)
    inp = img.astype(np.float64) / 65535.0
    gray = 0.299 * inp[0] + 0.587 * inp[1] + 0.114 * inp[2]
    g = pm.gaussian_pyramid(gray, J)
    up = g[-1]
    for l in range(J - 2, -1, -1):
        up = pm.upsample(up, g[l].shape)
    out_gray = beta * gray + (1.0 - beta) * up
    np.testing.assert_allclose(out, inp * (out_gray / gray)[None], rtol=0, atol=1e-7)


def _down(img):
    return ndi.correlate(img, np.outer(B5, B5) / 256.0, mode="nearest")[::2, ::2]


def _up(coarse, shape):
    p = np.pad(coarse, 2, mode="edge")
    z = np.zeros((2 * p.shape[0], 2 * p.shape[1]))
    z[::2, ::2] = p
    z = ndi.correlate1d(z, B5 / 8.0, axis=0, mode="constant")
    z = ndi.correlate1d(z, B5 / 8.0, axis=1, mode="constant")
    return z[4:4 + shape[0], 4:4 + shape[1]]


def test_two_level_filter_by_per_pixel_evaluation():
    # Independent per-pixel evaluation of a 2-level filter with a non-identity remap, built
    # on scipy-based down/upsampling instead of the oracle's pyramid module.
    K, sig, alpha, beta = 8, 0.1, 0.25, 1.0
    img = synth.rgb_u16_gradient_noise(10, 14, seed=3)
    inp = img.astype(np.float64) / 65535.0
    gray = 0.299 * inp[0] + 0.587 * inp[1] + 0.114 * inp[2]
    lap0 = []
    for k in range(K):
        r = ll.remap(gray, k / (K - 1), sig, alpha, beta)
        lap0.append(r - _up(_down(r), r.shape))
    residual = _down(gray)
    up_res = _up(residual, gray.shape)
    expect = np.zeros_like(inp)
    for y in range(gray.shape[0]):
        for x in range(gray.shape[1]):
            t = gray[y, x] * (K - 1)
            k0 = min(int(np.floor(t)), K - 2)
            f = t - k0
            lp = (1 - f) * lap0[k0][y, x] + f * lap0[k0 + 1][y, x]
            og = lp + up_res[y, x]
            for c in range(3):
                expect[c, y, x] = inp[c, y, x] * og / gray[y, x] if gray[y, x] > 0 else og
    got = ll.local_laplacian_float(img, levels=2, k_levels=K, sigma_r=sig, alpha=alpha, beta=beta)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13)


def test_quantize_rounds_half_to_even_and_clamps():
    x = np.array([-0.1, 0.0, 0.5 / 65535, 1.5 / 65535, 1.0, 1.2])
    assert ll.quantize_u16(x).tolist() == [0, 0, 0, 2, 65535, 65535]
