"""Pins of the FP64 unsharp-mask oracle and the exact histogram-equalize oracle (CPU only)."""

import json
import os

import numpy as np
import scipy.ndimage as ndi

from oracle import histeq as he
from oracle import unsharp as us
from paper_2012_07145_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
B5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0])


def test_unsharp_matches_scipy_blur():
    img = synth.rgb_f32(21, 17, seed=4).astype(np.float64)
    out = us.unsharp(img)
    for c in range(3):
        blur = ndi.correlate(img[c], np.outer(B5, B5) / 256.0, mode="nearest")
        np.testing.assert_allclose(out[c], img[c] + 1.5 * (img[c] - blur), rtol=0, atol=1e-14)


def test_unsharp_constant_ramp_and_zero_amount():
    c = np.full((3, 8, 9), 0.3)
    np.testing.assert_allclose(us.unsharp(c), c, atol=1e-15, rtol=0)
    H, W = 12, 15
    yy, xx = np.mgrid[0:H, 0:W]
    ramp = np.stack([0.01 * xx + 0.02 * yy] * 3).astype(np.float64)
    np.testing.assert_allclose(us.unsharp(ramp)[:, 2:-2, 2:-2], ramp[:, 2:-2, 2:-2], atol=1e-14, rtol=0)
    img = synth.rgb_f32(6, 7, seed=8).astype(np.float64)
    np.testing.assert_array_equal(us.unsharp(img, amount=0.0), img)


def test_histeq_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "histeq_worked_example.json")))
    img = np.array(g["image"], dtype=np.uint8)
    h, table, out = he.equalize(img)
    assert h[:4] == g["hist_head"] and sum(h) == img.size
    assert table[:4] == g["lut_head"]
    assert out.tolist() == g["output"]


def test_histogram_matches_bincount_and_properties():
    img = synth.gray_u8_lowcontrast(61, 47, seed=3)
    h, table, out = he.equalize(img)
    assert h == np.bincount(img.ravel(), minlength=256).tolist()
    assert sum(h) == img.size
    assert all(table[v] <= table[v + 1] for v in range(255))
    assert table[int(img.min())] == 0 and table[int(img.max())] == 255
    perm = np.random.default_rng(0).permutation(img.ravel()).reshape(img.shape)
    assert he.histogram(perm) == h


def test_histeq_constant_and_uniform_images():
    const = np.full((5, 7), 77, dtype=np.uint8)
    _, table, out = he.equalize(const)
    assert table == list(range(256)) and np.array_equal(out, const)
    uni = np.tile(np.arange(256, dtype=np.uint8), 3).reshape(3, 256)
    _, table, out = he.equalize(uni)
    assert table == list(range(256))
