"""Pins of the FP64 Harris oracle (CPU only)."""

import numpy as np
import scipy.ndimage as ndi

from oracle import harris as hr
from paper_2012_07145_gb300 import synth


def test_gray_weights_from_the_workload_definition():
    assert abs(hr.gray(np.array([1.0, 0, 0]).reshape(3, 1, 1))[0, 0] - 0.299) < 1e-16
    assert abs(hr.gray(np.array([0, 1.0, 0]).reshape(3, 1, 1))[0, 0] - 0.587) < 1e-16
    assert abs(hr.gray(np.array([0, 0, 1.0]).reshape(3, 1, 1))[0, 0] - 0.114) < 1e-16


def test_stages_match_scipy_sobel_and_box():
    rgb = synth.rgb_f32(23, 31, seed=2).astype(np.float64)
    s = hr.harris_stages(rgb)
    np.testing.assert_allclose(s["ix"], ndi.sobel(s["gray"], axis=1, mode="nearest"), atol=1e-14, rtol=0)
    np.testing.assert_allclose(s["iy"], ndi.sobel(s["gray"], axis=0, mode="nearest"), atol=1e-14, rtol=0)
    ones = np.ones((3, 3))
    np.testing.assert_allclose(s["sxx"], ndi.correlate(s["ix"] ** 2, ones, mode="nearest"), atol=1e-13, rtol=0)
    np.testing.assert_allclose(s["sxy"], ndi.correlate(s["ix"] * s["iy"], ones, mode="nearest"), atol=1e-13,
                               rtol=0)


def test_constant_image_has_zero_response():
    rgb = np.full((3, 9, 12), 0.6)
    assert np.all(np.abs(hr.harris(rgb)) < 1e-30)   # FP64 summation-order residue only


def test_linear_ramp_closed_form():
    # g = a x + b y: interior Ix = 8a, Iy = 8b, det = 0, R = -k (9*64 (a^2 + b^2))^2.
    a, b = 0.013, -0.007
    H, W = 14, 17
    yy, xx = np.mgrid[0:H, 0:W]
    g = a * xx + b * yy
    rgb = np.stack([g, g, g])
    r = hr.harris(rgb)
    expect = -hr.HARRIS_K * (9 * 64 * (a * a + b * b)) ** 2
    np.testing.assert_allclose(r[2:-2, 2:-2], expect, rtol=1e-9, atol=0)


def test_transpose_symmetry():
    rgb = synth.rgb_f32(12, 19, seed=5).astype(np.float64)
    np.testing.assert_allclose(hr.harris(rgb.transpose(0, 2, 1)), hr.harris(rgb).T, atol=1e-13, rtol=0)


def test_corner_positive_edge_negative_flat_zero():
    img = np.zeros((40, 40))
    img[10:30, 10:30] = 1.0
    r = hr.harris(np.stack([img, img, img]))
    assert r[10, 10] > 0 and r[29, 29] > 0          # corners
    assert r[20, 10] < 0 and r[10, 20] < 0          # straight edges
    assert abs(r[20, 20]) < 1e-30 and r[2, 2] == 0    # flat inside and outside
