"""Per-pixel error bound of the local Laplacian filter from the conditioning of
its remap (test infrastructure: used by the parity tests, pinned on the CPU by
test_ll_bound.py).

For alpha < 1 the remap r(i) = g + sign(d) sigma (|d|/sigma)^alpha, d = i - g,
has an unbounded slope at d = 0 (Paris et al. 2011; the local Laplacian app of
Sec. 6).  An FP32 evaluation cannot know d better than to the rounding of its
operands, and x^alpha is only alpha-Hoelder at 0, so near a level g_k the remap
of any FP32 implementation may differ from the exact one by far more than the
rounding of its own output.  That error is the method's conditioning, not the
kernel's, and this module bounds it per output pixel:

1. Uncertainty of d in FP32, per pixel and level (u = 2^-24):
     |delta d| <= u (7 |i| + |g_k| + |d|)
   (plus the same with 2^-53 for the FP64 oracle's own rounding of d, which
   matters where d is within a few ulps of 0: the oracle's gray of a saturated
   pixel is 1 - 2^-53, not 1)
   gray i = 0.299 R s + 0.587 G s + 0.114 B s with s = 1/65535: every term has
   at most six relative roundings (s, the product with s, the weight, up to
   three accumulations), all terms are positive, so |delta i| <= 6u|i| (7 with
   margin for second-order terms); g_k = k/(K-1) is rounded once (u|g_k|); the
   subtraction once (u|d|).
2. Remap error for a = |d|, delta = |delta d| (x^alpha is monotone and
   concave; its largest change over [a - delta, a + delta] is at the left):
     a > delta:  sigma^(1-alpha) ((a + delta)^alpha - (a - delta)^alpha)
     a <= delta: 2 sigma^(1-alpha) (a + delta)^alpha     (d may change sign)
   plus beta delta for the linear branch outside the band (|d| > sigma).
3. Propagation: every later step is linear in the remapped images with
   non-negative weights (Gaussian pyramid, upsample), differences of them
   (Laplacian) or convex combinations (the interpolation in k), so the error of
   L_l[r_k] is at most G_l[E_k] + U(G_{l+1}[E_k]), the interpolated level at
   most (1-f) B_{l,k0} + f B_{l,k0+1}, and the collapse adds the levels'
   bounds as it adds the levels.  The residual G_{J-1}[gray] holds no remap.
4. Colour: out_c = in_c out_gray / gray multiplies the gray bound by
   in_c / gray (by 1 where gray = 0).

The ordinary FP32 rounding of every other operation is not in this bound; the
parity test allows it separately (1e-5 of the output range, the tolerance of
every FP32 stage).
"""

import numpy as np

from oracle.local_laplacian import GRAY_WEIGHTS
from oracle.pyramid import gaussian_pyramid, upsample

U = 2.0 ** -24
U64 = 2.0 ** -53
C_GRAY = 7.0


def delta_d(gray, gk):
    """Bound of |d_fp32 - d_oracle| for d = gray - g_k (item 1): the FP32
    uncertainty plus the oracle's own FP64 one (the same count of roundings at
    2^-53), which the comparison with the oracle also sees."""
    return (U + U64) * (C_GRAY * np.abs(gray) + abs(gk) + np.abs(gray - gk))


def remap_error_bound(gray, gk, sigma, alpha, beta):
    """Bound of |r_fp32 - r| per pixel for level g_k (item 2)."""
    a = np.abs(gray - gk)
    dl = delta_d(gray, gk)
    lo = np.maximum(a - dl, 0.0)
    hoelder = np.where(a > dl, (a + dl) ** alpha - lo ** alpha, 2.0 * (a + dl) ** alpha)
    return sigma ** (1.0 - alpha) * hoelder + beta * dl


def gray_of(rgb_u16):
    inp = np.asarray(rgb_u16, dtype=np.float64) / 65535.0
    return inp, GRAY_WEIGHTS[0] * inp[0] + GRAY_WEIGHTS[1] * inp[1] + GRAY_WEIGHTS[2] * inp[2]


def gray_bound(gray, levels, k_levels, sigma, alpha, beta):
    """Bound of the error of out_gray caused by the remap's conditioning (items 1-3)."""
    J, K = levels, k_levels
    g_pyr = gaussian_pyramid(gray, J)
    per_k = []
    for k in range(K):
        e = gaussian_pyramid(remap_error_bound(gray, k / (K - 1), sigma, alpha, beta), J)
        per_k.append([e[l] + upsample(e[l + 1], e[l].shape) for l in range(J - 1)])
    r = np.zeros_like(g_pyr[J - 1])
    for l in range(J - 2, -1, -1):
        t = g_pyr[l] * (K - 1)
        k0 = np.clip(np.minimum(np.floor(t), K - 2), 0, K - 2).astype(np.int64)
        f = np.clip(t - k0, 0.0, 1.0)
        stack = np.stack([per_k[k][l] for k in range(K)])
        lo = np.take_along_axis(stack, k0[None], axis=0)[0]
        hi = np.take_along_axis(stack, (k0 + 1)[None], axis=0)[0]
        r = (1.0 - f) * lo + f * hi + upsample(r, g_pyr[l].shape)
    return r


def output_bound(rgb_u16, levels, k_levels, sigma, alpha, beta):
    """Per-pixel, per-channel bound [3][H][W] in [0, 1] units (items 1-4)."""
    inp, gray = gray_of(rgb_u16)
    b = gray_bound(gray, levels, k_levels, sigma, alpha, beta)
    ratio = np.where(gray > 0, inp / np.where(gray > 0, gray, 1.0), 1.0)
    return b[None] * ratio
