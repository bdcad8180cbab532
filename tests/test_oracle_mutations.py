"""The oracle's pins catch plausible mistakes: each case plants one mistake in
the oracle (on the CPU, through monkeypatch: a dropped or wrong term, a sign,
an index, a boundary, a rounding) and runs the pins of that part of the oracle;
at least one of them must fail with an assertion."""

import numpy as np
import pytest

from oracle import bilateral_grid as ob
from oracle import harris as oh
from oracle import histeq as oeq
from oracle import interpolate as oi
from oracle import local_laplacian as oll
from oracle import maxfilter as om
from oracle import pyramid as pm
from oracle import stencil as ost
from oracle import unsharp as ou

import test_oracle_bilateral_grid as t_bg
import test_oracle_harris as t_h
import test_oracle_ll as t_ll
import test_oracle_maxfilter_interpolate as t_mi
import test_oracle_pyramid as t_py
import test_oracle_stencil as t_st
import test_oracle_unsharp_histeq as t_uh

STENCIL_PINS = [t_st.test_single_stage_matches_scipy_nearest, t_st.test_chain_per_stage_clamp_matches_scipy_chain,
                t_st.test_chain_kinds_pattern, lambda: t_st.test_chain_impulse_response_closed_form(4, "binomial"),
                lambda: t_st.test_chain_impulse_response_closed_form(32, "alternate"),
                t_st.test_constant_and_linearity_and_transpose, t_st.test_one_d_example_of_sec4,
                t_st.test_point_evaluation_matches_full_chain]
PYRAMID_PINS = [t_py.test_downsample_equals_nearest_correlation_then_subsample,
                t_py.test_upsample_equals_zero_stuffing_construction, t_py.test_ramps_interior,
                t_py.test_constant_preserved_and_sizes, t_py.test_laplacian_collapse_reconstructs]
HARRIS_PINS = [t_h.test_gray_weights_from_the_workload_definition, t_h.test_stages_match_scipy_sobel_and_box,
               t_h.test_constant_image_has_zero_response, t_h.test_linear_ramp_closed_form,
               t_h.test_transpose_symmetry, t_h.test_corner_positive_edge_negative_flat_zero]
LL_PINS = [t_ll.test_remap_hand_values, t_ll.test_identity_parameters_return_the_input,
           t_ll.test_constant_image_is_unchanged_for_any_parameters, t_ll.test_tiny_sigma_is_the_linear_remap_closed_form,
           t_ll.test_two_level_filter_by_per_pixel_evaluation, t_ll.test_quantize_rounds_half_to_even_and_clamps]
UNSHARP_HISTEQ_PINS = [t_uh.test_unsharp_matches_scipy_blur, t_uh.test_unsharp_constant_ramp_and_zero_amount,
                       t_uh.test_histeq_worked_example, t_uh.test_histogram_matches_bincount_and_properties,
                       t_uh.test_histeq_constant_and_uniform_images]
MAX_PINS = [t_mi.test_max_filter_brute_force_tiny, t_mi.test_max_filter_is_scipy_maximum_filter_nearest,
            t_mi.test_max_filter_separable_equals_2d, t_mi.test_max_filter_impulse_and_invariants]
INTERP_PINS = [t_mi.test_interpolate_full_coverage_is_identity, t_mi.test_interpolate_two_pixel_closed_form,
               t_mi.test_interpolate_constant_colour_and_linearity, t_mi.test_interpolate_one_level_divides_out_coverage]
GRID_PINS = [t_bg.test_splat_brute_force_and_counts, t_bg.test_range_level_is_decided_in_f32,
             t_bg.test_constant_image_is_preserved, t_bg.test_edge_far_apart_in_range_is_kept,
             t_bg.test_blur_axis_is_clamped_binomial, t_bg.test_slice_of_a_linear_grid_is_the_linear_function,
             t_bg.test_blur_is_the_separable_binomial_in_three_axes]


# ---------------------------------------------------------------- mistakes --
def _stencil_wrap(img, w):
    """A stage whose reads wrap around the image instead of clamping."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    ry, rx = (w.shape[0] - 1) // 2, (w.shape[1] - 1) // 2
    out = np.zeros((H, W))
    for j in range(-ry, ry + 1):
        for i in range(-rx, rx + 1):
            out += w[j + ry, i + rx] * img[np.ix_((np.arange(H) + j) % H, (np.arange(W) + i) % W)]
    return out


def _chain_clamped_on_input_only(img, kinds):
    """The chain computed on the input padded once (clamp at the input only)."""
    n = len(kinds)
    pad = 2 * n
    s = np.pad(np.asarray(img, dtype=np.float64), pad, mode="edge")
    for kind in kinds:
        w = ost.binomial5_weights() if kind == "binomial" else ost.box5_weights()
        H, W = s.shape
        out = np.zeros_like(s)
        for j in range(-2, 3):
            for i in range(-2, 3):
                out += w[j + 2, i + 2] * s[np.ix_(np.clip(np.arange(H) + j, 0, H - 1), np.clip(np.arange(W) + i, 0, W - 1))]
        s = out
    return s[pad:-pad, pad:-pad]


def _downsample_odd(img):
    """Downsample centred on (2x+1, 2y+1) instead of (2x, 2y)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    h, w = pm.down_size(H), pm.down_size(W)
    out = np.zeros((h, w))
    for j in range(-2, 3):
        rows = np.clip(2 * np.arange(h) + 1 + j, 0, H - 1)
        for i in range(-2, 3):
            cols = np.clip(2 * np.arange(w) + 1 + i, 0, W - 1)
            out += (pm.BINOMIAL5[j + 2] * pm.BINOMIAL5[i + 2] / 256.0) * img[np.ix_(rows, cols)]
    return out


def _collapse_with_laplacians(lap):
    """Collapse that adds the upsampled next Laplacian instead of the next result."""
    r = lap[-1]
    for l in range(len(lap) - 2, -1, -1):
        r = lap[l] + pm.upsample(lap[l + 1], lap[l].shape)
    return r


_remap = oll.remap


def _remap_detail_sign(i, g, sigma_r, alpha, beta):
    """Remap whose large-difference branch moves towards g instead of away."""
    i = np.asarray(i, dtype=np.float64)
    r = _remap(i, g, sigma_r, alpha, beta)
    d = i - g
    return np.where(np.abs(d) > sigma_r, g - np.sign(d) * (beta * (np.abs(d) - sigma_r) + sigma_r), r)


def _lut_round_down(h):
    c = oeq.cdf(h)
    n = c[-1]
    vmin = next(v for v in range(256) if h[v] > 0) if n > 0 else 0
    cmin = c[vmin]
    if n == cmin:
        return list(range(256))
    return [0 if c[v] < cmin else (c[v] - cmin) * 255 // (n - cmin) for v in range(256)]


def _cdf_exclusive(h):
    out, acc = [], 0
    for c in h:
        out.append(acc)
        acc += c
    return out


_max_filter = om.max_filter


def _range_level_truncated(v, r, gz):
    inv_r = np.float64(np.float32(1.0 / ob._r32(r)))
    zf = (np.asarray(v, dtype=np.float32).astype(np.float64) * inv_r).astype(np.float32)
    return np.clip(np.floor(zf.astype(np.float64)).astype(np.int64), 0, gz - 1)


def _blur_without_range_axis(g):
    return ob.blur_axis(ob.blur_axis(g, 1), 0)


def _slice_swapped_weights(g, img, s, r):
    """Trilinear slice that weights the x neighbours by the y fraction and the
    y neighbours by the x fraction."""
    H, W = img.shape
    GY, GX, GZ, _ = g.shape
    v = np.clip(np.asarray(img, dtype=np.float64), 0.0, 1.0)
    xf = np.broadcast_to(np.arange(W)[None, :] / s, (H, W))
    yf = np.broadcast_to(np.arange(H)[:, None] / s, (H, W))
    zf = v / r
    x0, y0, z0 = np.floor(xf).astype(int), np.floor(yf).astype(int), np.floor(zf).astype(int)
    fx, fy, fz = xf - x0, yf - y0, zf - z0
    acc = np.zeros((H, W, 2))
    for dz, wz in ((0, 1 - fz), (1, fz)):
        for dy, wy in ((0, 1 - fx), (1, fx)):
            for dx, wx in ((0, 1 - fy), (1, fy)):
                acc += (wz * wy * wx)[..., None] * g[np.clip(y0 + dy, 0, GY - 1), np.clip(x0 + dx, 0, GX - 1),
                                                      np.clip(z0 + dz, 0, GZ - 1)]
    return np.where(acc[..., 1] > 0, acc[..., 0] / np.where(acc[..., 1] > 0, acc[..., 1], 1.0), v)


def _point_from_a_crop_too_small(img, kinds, x, y):
    """A point evaluated on a crop of radius n (the chain's reach is 2n), whose
    cut edges then act as clamp boundaries."""
    img = np.asarray(img, dtype=np.float64)
    n = len(kinds)
    y0, x0 = max(y - n, 0), max(x - n, 0)
    crop = img[y0:y + n + 1, x0:x + n + 1]
    return float(ost.stencil_chain(crop, kinds)[y - y0, x - x0])


def _upsample_wrapping(coarse, fine_shape):
    """Upsample whose coarse index wraps around instead of clamping."""
    coarse = np.asarray(coarse, dtype=np.float64)
    hc, wc = coarse.shape
    H, W = fine_shape
    Y, X = np.arange(H), np.arange(W)
    out = np.zeros((H, W))
    for s in range(-2, 3):
        row_ok = (Y - s) % 2 == 0
        n = ((Y - s) // 2) % hc
        for t in range(-2, 3):
            col_ok = (X - t) % 2 == 0
            m = ((X - t) // 2) % wc
            out += np.where(row_ok[:, None] & col_ok[None, :], (pm.UP_TAPS[s] * pm.UP_TAPS[t]) * coarse[np.ix_(n, m)], 0.0)
    return out


def _histogram_off_by_one(img_u8):
    h = [0] * 256
    for v in np.asarray(img_u8, dtype=np.uint8).ravel().tolist():
        h[min(v + 1, 255)] += 1
    return h


def _max_filter_wrapping(img, rx, ry):
    img = np.asarray(img)
    H, W = img.shape
    out = None
    for j in range(-ry, ry + 1):
        for i in range(-rx, rx + 1):
            v = img[np.ix_((np.arange(H) + j) % H, (np.arange(W) + i) % W)]
            out = v.copy() if out is None else np.maximum(out, v)
    return out


def _ll_interp_weights_swapped(rgb_u16, levels=8, k_levels=8, sigma_r=0.1, alpha=1.0, beta=1.0):
    """The local Laplacian with the two levels' weights exchanged (f on the
    lower level, 1 - f on the upper)."""
    inp = np.asarray(rgb_u16, dtype=np.float64) / 65535.0
    gray = oll.GRAY_WEIGHTS[0] * inp[0] + oll.GRAY_WEIGHTS[1] * inp[1] + oll.GRAY_WEIGHTS[2] * inp[2]
    g_pyr = pm.gaussian_pyramid(gray, levels)
    lap_k = [pm.laplacian_pyramid(pm.gaussian_pyramid(oll.remap(gray, k / (k_levels - 1), sigma_r, alpha, beta), levels))
             for k in range(k_levels)]
    out_lap = []
    for l in range(levels - 1):
        t = g_pyr[l] * (k_levels - 1)
        k0 = np.minimum(np.floor(t), k_levels - 2).astype(np.int64)
        f = t - k0
        stack = np.stack([lap_k[k][l] for k in range(k_levels)])
        lo = np.take_along_axis(stack, k0[None], axis=0)[0]
        hi = np.take_along_axis(stack, (k0 + 1)[None], axis=0)[0]
        out_lap.append(f * lo + (1.0 - f) * hi)
    out_lap.append(g_pyr[levels - 1])
    out_gray = pm.collapse(out_lap)
    safe = np.where(gray > 0, gray, 1.0)
    return np.where((gray > 0)[None], inp * (out_gray / safe)[None], out_gray[None])


MISTAKES = {
    # stencil chains
    "box weights 1/24": ([(ost, "box5_weights", lambda: np.full((5, 5), 1.0 / 24.0))], STENCIL_PINS),
    "binomial weights /255": ([(ost, "binomial5_weights", lambda: np.outer(ost.BINOMIAL5, ost.BINOMIAL5) / 255.0)],
                              STENCIL_PINS),
    "wrap-around boundary": ([(ost, "stencil_clamp", _stencil_wrap)], STENCIL_PINS),
    "alternation starts with box": ([(ost, "chain_kinds", lambda n, p: ["box" if k % 2 == 0 else "binomial"
                                                                          for k in range(n)] if p == "alternate"
                                      else ["binomial"] * n)], STENCIL_PINS),
    "clamp on the input only": ([(ost, "stencil_chain", _chain_clamped_on_input_only)], STENCIL_PINS),
    "point evaluated on too small a crop": ([(ost, "stencil_chain_point", _point_from_a_crop_too_small)], STENCIL_PINS),
    "upsample index wraps": ([(pm, "upsample", _upsample_wrapping)], PYRAMID_PINS),
    "histogram bin off by one": ([(oeq, "histogram", _histogram_off_by_one)], UNSHARP_HISTEQ_PINS),
    "max window wraps around": ([(om, "max_filter", _max_filter_wrapping)], MAX_PINS),
    "no division by coverage": ([(oi, "unpremultiply", lambda v: np.array(v[:3], dtype=np.float64))], INTERP_PINS),
    # pyramids
    "downsample at odd pixels": ([(pm, "downsample", _downsample_odd)], PYRAMID_PINS),
    "upsample taps over 16": ([(pm, "UP_TAPS", {k: v / 2.0 for k, v in pm.UP_TAPS.items()})], PYRAMID_PINS),
    "coarse size floor(n/2)": ([(pm, "down_size", lambda n: max(1, n // 2))], PYRAMID_PINS),
    "collapse adds Laplacians": ([(pm, "collapse", _collapse_with_laplacians)], PYRAMID_PINS),
    # Harris
    "y derivative = x derivative": ([(oh, "sobel_y_weights", oh.sobel_x_weights)], HARRIS_PINS),
    "Sobel smoothing [1,1,1]": ([(oh, "SOBEL_SMOOTH", np.array([1.0, 1.0, 1.0]))], HARRIS_PINS),
    "gray weights R and B swapped": ([(oh, "GRAY_WEIGHTS", (0.114, 0.587, 0.299))], HARRIS_PINS),
    "window mean instead of sum": ([(oh, "stencil_clamp", lambda img, w: ost.stencil_clamp(
        img, w / w.sum() if w.sum() != 0 else w))], HARRIS_PINS),
    # local Laplacian
    "remap detail branch sign": ([(oll, "remap", _remap_detail_sign)], LL_PINS),
    "collapse adds Laplacians (LL)": ([(oll, "collapse", _collapse_with_laplacians)], LL_PINS),
    "LL level weights exchanged": ([(oll, "local_laplacian_float", _ll_interp_weights_swapped)], LL_PINS),
    "u16 by truncation": ([(oll, "quantize_u16", lambda x: np.clip(np.floor(np.asarray(x) * 65535.0), 0, 65535)
                            .astype(np.uint16))], LL_PINS),
    "LL gray weights R and B swapped": ([(oll, "GRAY_WEIGHTS", (0.114, 0.587, 0.299))], LL_PINS),
    # unsharp, histogram equalize
    "unsharp blurs with the box": ([(ou, "binomial5_weights", ost.box5_weights)], UNSHARP_HISTEQ_PINS),
    "LUT rounds down": ([(oeq, "lut", _lut_round_down)], UNSHARP_HISTEQ_PINS),
    "exclusive CDF": ([(oeq, "cdf", _cdf_exclusive)], UNSHARP_HISTEQ_PINS),
    # max filter
    "window one smaller": ([(om, "max_filter", lambda img, rx, ry: _max_filter(img, max(rx - 1, 0), max(ry - 1, 0)))],
                           MAX_PINS),
    "horizontal window only": ([(om, "max_filter", lambda img, rx, ry: _max_filter(img, rx, 0))], MAX_PINS),
    # interpolate
    "over weighted by the back's alpha": ([(oi, "over", lambda f, b: f + (1.0 - b[3])[None] * b)], INTERP_PINS),
    "no premultiplication": ([(oi, "premultiply", lambda rgba: np.array(rgba, dtype=np.float64))], INTERP_PINS),
    # bilateral grid
    "range level truncated": ([(ob, "range_level", _range_level_truncated)], GRID_PINS),
    "no blur along the range": ([(ob, "blur", _blur_without_range_axis)], GRID_PINS),
    "slice x and y fractions swapped": ([(ob, "slice_grid", _slice_swapped_weights)], GRID_PINS),
    "blur taps over 15": ([(ob, "B5", np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 15.0)], GRID_PINS),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_a_planted_mistake_fails_a_pin(name, monkeypatch):
    patches, pins = MISTAKES[name]
    for module, attr, value in patches:
        monkeypatch.setattr(module, attr, value)
    failed = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed.append(getattr(pin, "__name__", "pin"))
        except Exception as e:   # the mistake also broke the pin's own arithmetic: noticed too
            failed.append(f"{getattr(pin, '__name__', 'pin')} ({type(e).__name__})")
    assert failed, f"no pin notices the planted mistake: {name}"
    assert any("(" not in f for f in failed), f"{name}: noticed only through exceptions {failed}"
