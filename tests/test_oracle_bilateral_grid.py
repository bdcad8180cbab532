"""Pins of the bilateral-grid oracle (CPU only)."""

import numpy as np

from oracle import bilateral_grid as ob


def _splat_brute(img, s, r):
    H, W = img.shape
    gz = ob.levels(r)
    GX, GY = ob.grid_size(W, H, s)
    g = np.zeros((GY, GX, gz, 2))
    inv_r = float(np.float32(1.0 / r))
    for gy in range(GY):
        for gx in range(GX):
            for j in range(s):
                for i in range(s):
                    x = min(max(gx * s + i - s // 2, 0), W - 1)
                    y = min(max(gy * s + j - s // 2, 0), H - 1)
                    v = float(np.float32(min(max(float(img[y, x]), 0.0), 1.0)))
                    z = int(np.floor(float(np.float32(v * inv_r + 0.5))))
                    z = min(max(z, 0), gz - 1)
                    g[gy, gx, z, 0] += v
                    g[gy, gx, z, 1] += 1.0
    return g


def test_splat_brute_force_and_counts():
    rng = np.random.default_rng(1)
    for (h, w, s, r) in [(5, 7, 2, 0.25), (9, 4, 4, 0.1), (1, 1, 2, 0.5), (13, 11, 3, 0.2)]:
        img = rng.random((h, w)).astype(np.float32) * 1.2 - 0.1     # some values outside [0, 1]
        g = ob.splat(img, s, r)
        np.testing.assert_allclose(g, _splat_brute(img, s, r), rtol=0, atol=1e-12)
        assert (g[..., 1].sum(axis=2) == s * s).all()             # every cell counts s^2 pixels


def test_range_level_is_decided_in_f32():
    # f32(0.35) * 10 + 0.5 = 3.99999994 exactly, which rounds to 4.0 in f32:
    # level 4 (an f64 evaluation would give 3)
    v = np.float32(0.35)
    assert np.floor(np.float64(v) * 10.0 + 0.5) == 3.0
    assert ob.range_level(np.array([v]), 0.1, 11)[0] == 4


def test_constant_image_is_preserved():
    img = np.full((37, 45), 0.37, dtype=np.float32)
    out = ob.bilateral_grid(img, 8, 0.1)
    np.testing.assert_allclose(out, np.float64(np.float32(0.37)), rtol=0, atol=1e-12)


def test_edge_far_apart_in_range_is_kept():
    # a step from 0.2 to 0.8: six range cells apart, beyond the blur's two, so
    # each side only averages itself and the edge survives exactly
    img = np.full((40, 64), 0.2, dtype=np.float32)
    img[:, 32:] = 0.8
    out = ob.bilateral_grid(img, 8, 0.1)
    np.testing.assert_allclose(out[:, :32], np.float64(np.float32(0.2)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out[:, 32:], np.float64(np.float32(0.8)), rtol=0, atol=1e-12)


def test_blur_axis_is_clamped_binomial():
    g = np.zeros((3, 4, 6, 2))
    g[1, 2, 0, 0] = 16.0                                           # an impulse at range level 0
    b = ob.blur_axis(g, 2)
    np.testing.assert_allclose(b[1, 2, :, 0], [11.0, 5.0, 1.0, 0.0, 0.0, 0.0])  # (1+4+6), (4+1), 1 at the clamped end
    assert b.sum() > 0 and b[..., 1].sum() == 0


def test_slice_of_a_linear_grid_is_the_linear_function():
    # trilinear interpolation reproduces a function linear in (x/s, y/s, v/r)
    H, W, s, r = 17, 23, 4, 0.25
    GX, GY = ob.grid_size(W, H, s)
    gz = ob.levels(r)
    gy, gx, gzz = np.meshgrid(np.arange(GY), np.arange(GX), np.arange(gz), indexing="ij")
    g = np.stack([0.5 + 0.1 * gx + 0.2 * gy + 0.3 * gzz, np.ones_like(gx, dtype=float)], axis=-1)
    img = np.random.default_rng(2).random((H, W)) * 0.999
    out = ob.slice_grid(g, img, s, r)
    ys, xs = np.mgrid[0:H, 0:W]
    exp = 0.5 + 0.1 * np.minimum(xs / s, GX - 1) + 0.2 * np.minimum(ys / s, GY - 1) + 0.3 * (img / r)
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-12)


def test_blur_is_the_separable_binomial_in_three_axes():
    # an impulse far from every edge spreads into b(y) b(x) b(z), b = [1,4,6,4,1]/16,
    # in the value channel only: the blur acts on all three grid axes
    g = np.zeros((9, 10, 11, 2))
    g[4, 5, 5, 0] = 1.0
    out = ob.blur(g)
    b = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0
    exp = np.zeros((9, 10, 11))
    exp[2:7, 3:8, 3:8] = b[:, None, None] * b[None, :, None] * b[None, None, :]
    np.testing.assert_allclose(out[..., 0], exp, rtol=0, atol=1e-15)
    assert not out[..., 1].any()
