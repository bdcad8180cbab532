"""Pins of the FP64 stencil oracle against things other than itself (CPU only)."""

import json
import os
from fractions import Fraction
from math import comb

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import stencil as st
from paper_2012_07145_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_single_stage_matches_scipy_nearest():
    # scipy.ndimage.correlate with mode='nearest' is an independent clamp-to-edge correlation.
    rng = np.random.default_rng(1)
    for shape in [(1, 1), (2, 3), (7, 5), (13, 29), (16, 16)]:
        img = rng.random(shape)
        for w in [st.binomial5_weights(), st.box5_weights(), rng.standard_normal((3, 5)),
                  rng.standard_normal((5, 1))]:
            ref = ndi.correlate(img, w, mode="nearest")
            np.testing.assert_allclose(st.stencil_clamp(img, w), ref, rtol=0, atol=1e-13)


def test_chain_per_stage_clamp_matches_scipy_chain():
    # Four successive nearest-mode correlations = a per-stage clamp on each producer.
    img = synth.stencil_input(37, 23)[0].astype(np.float64)
    ref = img
    for kind in st.chain_kinds(6, "alternate"):
        ref = ndi.correlate(ref, st.binomial5_weights() if kind == "binomial" else st.box5_weights(),
                            mode="nearest")
    np.testing.assert_allclose(st.stencil_chain(img, st.chain_kinds(6, "alternate")), ref,
                               rtol=0, atol=1e-13)


def test_chain_kinds_pattern():
    assert st.chain_kinds(4, "binomial") == ["binomial"] * 4
    kinds = st.chain_kinds(32, "alternate")
    assert kinds[0] == "binomial" and kinds[1] == "box" and kinds.count("box") == 16


def _impulse_profile(n_binomial: int, n_box: int):
    """Exact 1-D impulse response of n_binomial [1,4,6,4,1]/16 and n_box [1]*5/5 passes."""
    binom = [Fraction(comb(4 * n_binomial, k), 2 ** (4 * n_binomial)) for k in range(4 * n_binomial + 1)]
    boxp = [Fraction(1)]
    for _ in range(n_box):
        nxt = [Fraction(0)] * (len(boxp) + 4)
        for a, c in enumerate(boxp):
            for t in range(5):
                nxt[a + t] += c / 5
        boxp = nxt
    out = [Fraction(0)] * (len(binom) + len(boxp) - 1)
    for a, ca in enumerate(binom):
        for b, cb in enumerate(boxp):
            out[a + b] += ca * cb
    return np.array([float(v) for v in out])


@pytest.mark.parametrize("n_stages,pattern", [(4, "binomial"), (32, "alternate")])
def test_chain_impulse_response_closed_form(n_stages, pattern):
    kinds = st.chain_kinds(n_stages, pattern)
    nb = kinds.count("binomial")
    nx = kinds.count("box")
    p = _impulse_profile(nb, nx)
    radius = (len(p) - 1) // 2
    assert radius == 2 * n_stages
    size = 2 * radius + 1 + 2 * (radius + 4)
    img = np.zeros((size, size))
    c = size // 2
    img[c, c] = 1.0
    out = st.stencil_chain(img, kinds)
    expect = np.zeros_like(img)
    expect[c - radius:c + radius + 1, c - radius:c + radius + 1] = np.outer(p, p)
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-15 * p.max() ** 2 * 10)
    assert abs(out.sum() - 1.0) < 1e-12


def test_constant_and_linearity_and_transpose():
    kinds = st.chain_kinds(5, "alternate")
    a = synth.stencil_input(19, 11, seed=3)[0].astype(np.float64)
    b = synth.stencil_input(19, 11, seed=4)[0].astype(np.float64)
    np.testing.assert_allclose(st.stencil_chain(np.full((9, 6), 0.37), kinds), 0.37, rtol=0, atol=1e-15)
    lhs = st.stencil_chain(2.5 * a - 0.75 * b, kinds)
    rhs = 2.5 * st.stencil_chain(a, kinds) - 0.75 * st.stencil_chain(b, kinds)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13)
    np.testing.assert_allclose(st.stencil_chain(a.T, kinds), st.stencil_chain(a, kinds).T, rtol=0, atol=1e-14)


def test_one_d_example_of_sec4():
    g = json.load(open(os.path.join(GOLDEN, "stencil_1d_example.json")))
    row = np.array([g["input"]], dtype=np.float64)
    w = np.ones((1, 3))
    inter = st.stencil_clamp(row, w)
    out = st.stencil_clamp(inter, w)
    assert inter[0].tolist() == g["intermed"]
    assert out[0].tolist() == g["output"]


def test_point_evaluation_matches_full_chain():
    kinds = st.chain_kinds(7, "alternate")
    img = synth.stencil_input(41, 53, seed=9)[0].astype(np.float64)
    full = st.stencil_chain(img, kinds)
    for (x, y) in [(0, 0), (52, 40), (1, 39), (26, 20), (50, 2), (13, 0)]:
        assert abs(st.stencil_chain_point(img, kinds, x, y) - full[y, x]) < 1e-14
