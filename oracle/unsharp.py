"""Unsharp mask, FP64 (oracle; test infrastructure only).

Unsharp mask is one of the imaging apps of Sec. 6; the paper does not give its
arithmetic.  Reading used: per channel c,
    blur_c = 5x5 binomial stencil of in_c (b (x) b / 256, b = [1,4,6,4,1], clamp-to-edge)
    out_c  = in_c + amount * (in_c - blur_c),  amount = 1.5, no output clamp.
"""

import numpy as np

from .stencil import stencil_clamp, binomial5_weights

AMOUNT = 1.5


def unsharp(img: np.ndarray, amount: float = AMOUNT) -> np.ndarray:
    """Planar [C][H][W] in, planar [C][H][W] out."""
    img = np.asarray(img, dtype=np.float64)
    out = np.empty_like(img)
    for c in range(img.shape[0]):
        blur = stencil_clamp(img[c], binomial5_weights())
        out[c] = img[c] + amount * (img[c] - blur)
    return out
