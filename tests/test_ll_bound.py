"""CPU pins of the local Laplacian conditioning bound (tests/ll_bound.py).

The bound must hold for every perturbation of d = gray - g_k within the stated
FP32 uncertainty, including the adversarial ones (all +delta, all -delta,
each pixel pushed toward zero), on a gray image that puts pixels exactly on,
and within a few ulps of, every level g_k.  A first-order (Lipschitz) bound
must fail there, which shows the Hoelder term is the one that matters.
"""

import numpy as np

from oracle.local_laplacian import remap
from oracle.pyramid import collapse, gaussian_pyramid, laplacian_pyramid

import ll_bound

J, K, SIG, ALPHA, BETA = 4, 8, 0.1, 0.25, 1.0


def _out_gray(gray, eps_per_k):
    """out_gray of the filter with the remap of level k evaluated at d + eps_k."""
    g_pyr = gaussian_pyramid(gray, J)
    laps = [laplacian_pyramid(gaussian_pyramid(remap(gray + eps_per_k[k], k / (K - 1), SIG, ALPHA, BETA), J))
            for k in range(K)]
    out = []
    for l in range(J - 1):
        t = g_pyr[l] * (K - 1)
        k0 = np.minimum(np.floor(t), K - 2).astype(np.int64)
        f = t - k0
        stack = np.stack([laps[k][l] for k in range(K)])
        out.append((1 - f) * np.take_along_axis(stack, k0[None], 0)[0] + f * np.take_along_axis(stack, (k0 + 1)[None], 0)[0])
    out.append(g_pyr[J - 1])
    return collapse(out)


def _gray_on_levels(seed=0, h=40, w=56):
    rng = np.random.default_rng(seed)
    g = rng.uniform(0, 1, (h, w))
    levels = np.arange(K) / (K - 1)
    idx = rng.integers(0, h * w, 400)
    offs = np.array([0.0, 1e-12, -1e-12, 3e-9, -3e-9, 5e-8, -5e-8, 4e-7, -4e-7, 1e-4])
    g.ravel()[idx] = np.clip(levels[rng.integers(0, K, 400)] + offs[rng.integers(0, len(offs), 400)], 0, 1)
    return g


def test_bound_holds_for_perturbations_within_the_fp32_uncertainty():
    gray = _gray_on_levels()
    base = _out_gray(gray, [0.0] * K)
    bound = ll_bound.gray_bound(gray, J, K, SIG, ALPHA, BETA)
    rng = np.random.default_rng(1)
    dl = [ll_bound.delta_d(gray, k / (K - 1)) for k in range(K)]
    cases = [[+d for d in dl], [-d for d in dl],
             [-np.sign(gray - k / (K - 1)) * dl[k] for k in range(K)],        # toward zero: the largest change
             [np.sign(gray - k / (K - 1)) * dl[k] for k in range(K)]]
    cases += [[rng.uniform(-1, 1, gray.shape) * d for d in dl] for _ in range(4)]
    worst = 0.0
    for eps in cases:
        diff = np.abs(_out_gray(gray, eps) - base)
        assert (diff <= bound * (1 + 1e-9) + 1e-15).all()
        worst = max(worst, float((diff / np.maximum(bound, 1e-300)).max()))
    assert worst > 0.05      # the bound is not vacuous: the toward-zero case reaches a fair part of it


def test_first_order_bound_fails_near_the_levels():
    """A Lipschitz bound (slope alpha sigma^(1-alpha) a^(alpha-1) at a = |d|,
    capped at the slope at delta) underestimates the change of pixels on a
    level: the Hoelder term is needed."""
    gray = _gray_on_levels()
    base = _out_gray(gray, [0.0] * K)
    dl = [ll_bound.delta_d(gray, k / (K - 1)) for k in range(K)]
    eps = [-np.sign(gray - k / (K - 1)) * dl[k] * 2 for k in range(K)]      # cross zero
    diff = np.abs(_out_gray(gray, eps) - base)

    def lipschitz(g, gk, s, al, be):
        a = np.maximum(np.maximum(np.abs(g - gk), ll_bound.delta_d(g, gk)), 1e-300)
        return (al * s ** (1 - al) * a ** (al - 1) + be) * ll_bound.delta_d(g, gk)

    saved = ll_bound.remap_error_bound
    try:
        ll_bound.remap_error_bound = lipschitz
        first_order = ll_bound.gray_bound(gray, J, K, SIG, ALPHA, BETA)
    finally:
        ll_bound.remap_error_bound = saved
    assert (diff > first_order * 2).any()


def test_bound_is_small_away_from_the_levels_and_scales_with_alpha():
    rng = np.random.default_rng(3)
    gray = rng.uniform(0, 1, (48, 64))
    levels = np.arange(K) / (K - 1)
    gray = np.where(np.min(np.abs(gray[..., None] - levels), axis=-1) < 1e-3, gray + 2e-3, gray)
    b = ll_bound.gray_bound(gray, J, K, SIG, ALPHA, BETA)
    # at least 1e-3 from every level: a few ulps amplified by at most ~16 per
    # remap and by the 2(J-1) of the propagation
    assert np.median(b) < 5e-6 and b.max() < 3e-5
    # identity remap (Lipschitz 1): three roundings of d per level, same propagation
    assert ll_bound.gray_bound(gray, J, K, SIG, 1.0, 1.0).max() < 1e-5
    # colour bound: in_c / gray times the gray bound, 1 where gray = 0
    rgb = np.zeros((3, 4, 4), dtype=np.uint16)
    rgb[0] = 65535
    ob = ll_bound.output_bound(rgb, 2, K, SIG, ALPHA, BETA)
    inp, g = ll_bound.gray_of(rgb)
    gb = ll_bound.gray_bound(g, 2, K, SIG, ALPHA, BETA)
    assert np.allclose(ob[0], gb / 0.299) and np.allclose(ob[1], 0.0)
