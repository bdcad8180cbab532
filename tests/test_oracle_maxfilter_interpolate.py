"""Pins of the max-filter and interpolate oracles (CPU only)."""

import numpy as np
import scipy.ndimage as ndi

from oracle import interpolate as oi
from oracle import maxfilter as om


# ------------------------------------------------------------- max filter --
def _max_brute(img, rx, ry):
    H, W = img.shape
    out = np.empty_like(img)
    for y in range(H):
        for x in range(W):
            m = None
            for j in range(-ry, ry + 1):
                for i in range(-rx, rx + 1):
                    v = img[min(max(y + j, 0), H - 1), min(max(x + i, 0), W - 1)]
                    m = v if m is None else max(m, v)
            out[y, x] = m
    return out


def test_max_filter_brute_force_tiny():
    rng = np.random.default_rng(1)
    for (h, w, rx, ry) in [(1, 1, 2, 2), (2, 3, 1, 0), (5, 7, 2, 1), (7, 4, 0, 3), (9, 9, 4, 4)]:
        img = rng.standard_normal((h, w))
        assert np.array_equal(om.max_filter(img, rx, ry), _max_brute(img, rx, ry))


def test_max_filter_is_scipy_maximum_filter_nearest():
    rng = np.random.default_rng(2)
    for (h, w, rx, ry) in [(16, 16, 4, 4), (33, 17, 3, 1), (40, 64, 2, 4)]:
        img = rng.random((h, w)).astype(np.float32)
        ref = ndi.maximum_filter(img, size=(2 * ry + 1, 2 * rx + 1), mode="nearest")
        assert np.array_equal(om.max_filter(img, rx, ry), ref)


def test_max_filter_separable_equals_2d():
    rng = np.random.default_rng(3)
    img = rng.random((31, 45))
    assert np.array_equal(om.max_filter(om.max_filter(img, 4, 0), 0, 4), om.max_filter(img, 4, 4))


def test_max_filter_impulse_and_invariants():
    img = np.zeros((20, 30))
    img[5, 10] = 1.0
    out = om.max_filter(img, 3, 2)
    exp = np.zeros_like(img)
    exp[3:8, 7:14] = 1.0                      # rows 5 +- 2, columns 10 +- 3
    assert np.array_equal(out, exp)
    img[0, 0] = 2.0                           # at a corner the window is clamped
    assert om.max_filter(img, 3, 2)[:3, :4].min() == 2.0 and om.max_filter(img, 3, 2)[3, 0] < 2.0
    rng = np.random.default_rng(4)
    x = rng.random((12, 13))
    assert (om.max_filter(x, 2, 2) >= x).all()
    assert np.array_equal(om.max_filter(np.full((6, 5), 0.25), 4, 4), np.full((6, 5), 0.25))


# ------------------------------------------------------------ interpolate --
def test_interpolate_full_coverage_is_identity():
    rng = np.random.default_rng(5)
    rgba = np.concatenate([rng.random((3, 24, 40)), np.ones((1, 24, 40))])
    assert np.array_equal(oi.interpolate(rgba, 5), rgba[:3])


def test_interpolate_two_pixel_closed_form():
    # 2x2 image, colour c1 at (0,0) and c2 at (1,1), the other two uncovered.
    # Downsample weights per axis after clamping: index 0 gets (1+4+6)/16,
    # index 1 gets (4+1)/16, so D_1.a = (121 + 25)/256 and D_1.rgb =
    # (121 c1 + 25 c2)/256; the upsample of a 1x1 level is constant, so an
    # uncovered pixel gets (121 c1 + 25 c2) / 146.
    c1 = np.array([0.9, 0.2, 0.4])
    c2 = np.array([0.1, 0.7, 0.3])
    rgba = np.zeros((4, 2, 2))
    rgba[:3, 0, 0], rgba[3, 0, 0] = c1, 1.0
    rgba[:3, 1, 1], rgba[3, 1, 1] = c2, 1.0
    out = oi.interpolate(rgba, 2)
    exp = (121 * c1 + 25 * c2) / 146
    np.testing.assert_allclose(out[:, 0, 1], exp, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[:, 1, 0], exp, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[:, 0, 0], c1, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[:, 1, 1], c2, rtol=0, atol=1e-15)


def test_interpolate_constant_colour_and_linearity():
    rng = np.random.default_rng(6)
    alpha = (rng.random((37, 53)) < 0.1).astype(np.float64) * rng.random((37, 53))
    colour = np.array([0.3, 0.6, 0.9])
    rgba = np.concatenate([np.broadcast_to(colour[:, None, None], (3, 37, 53)), alpha[None]])
    out = oi.interpolate(rgba, 6)
    covered = oi.interpolate(np.concatenate([np.ones((3, 37, 53)), alpha[None]]), 6)[0] > 0
    np.testing.assert_allclose(out[:, covered], np.broadcast_to(colour[:, None], out[:, covered].shape), atol=1e-13)
    a, b = rng.random((3, 37, 53)), rng.random((3, 37, 53))
    fa = oi.interpolate(np.concatenate([a, alpha[None]]), 6)
    fb = oi.interpolate(np.concatenate([b, alpha[None]]), 6)
    fab = oi.interpolate(np.concatenate([0.25 * a + 0.5 * b, alpha[None]]), 6)
    np.testing.assert_allclose(fab, 0.25 * fa + 0.5 * fb, atol=1e-13)


def test_interpolate_one_level_divides_out_coverage():
    rng = np.random.default_rng(7)
    rgba = np.concatenate([rng.random((3, 9, 11)), (rng.random((1, 9, 11)) > 0.5) * rng.random((1, 9, 11))])
    out = oi.interpolate(rgba, 1)
    cov = rgba[3] > 0
    np.testing.assert_allclose(out[:, cov], rgba[:3][:, cov], rtol=1e-15)
    assert (out[:, ~cov] == 0).all()
