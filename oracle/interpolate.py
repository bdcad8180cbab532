"""Pyramid interpolation of a partially covered RGBA image, FP64 (oracle; test
infrastructure only).

The interpolate app of Sec. 6 (named among the Halide-repository apps; the
paper gives no definition).  Reading used here: the multi-scale fill of the
uncovered pixels of an RGBA image (alpha = coverage) by premultiplied
pyramids, with the binomial downsample and upsample of ``pyramid``:

    P      = (R a, G a, B a, a)                      premultiplied input
    D_0    = P,  D_l = downsample(D_{l-1})           l = 1 .. J-1
    I_{J-1} = D_{J-1}
    I_l    = D_l + (1 - D_l.a) * U(I_{l+1})          every channel, alpha too
    out    = I_0.a > 0 ? I_0.rgb / I_0.a : 0         3 channels

Covered pixels (a = 1) keep their colour exactly; uncovered ones take the
coverage-weighted colour of the coarser levels.
"""

import numpy as np

from . import pyramid as pm


def premultiply(rgba: np.ndarray) -> np.ndarray:
    a = rgba[3]
    return np.stack([rgba[0] * a, rgba[1] * a, rgba[2] * a, a])


def over(front: np.ndarray, back: np.ndarray) -> np.ndarray:
    """Premultiplied compositing of front over back, every channel."""
    return front + (1.0 - front[3])[None] * back


def unpremultiply(v: np.ndarray) -> np.ndarray:
    a = v[3]
    safe = np.where(a > 0, a, 1.0)
    return np.stack([np.where(a > 0, v[c] / safe, 0.0) for c in range(3)])


def interpolate(rgba: np.ndarray, levels: int) -> np.ndarray:
    """[4][H][W] RGBA (float) -> [3][H][W] RGB, FP64, J = levels pyramid levels."""
    x = np.asarray(rgba, dtype=np.float64)
    D = [premultiply(x)]
    for _ in range(1, levels):
        D.append(np.stack([pm.downsample(D[-1][c]) for c in range(4)]))
    I = D[-1]
    for l in range(levels - 2, -1, -1):
        fine = D[l].shape[1:]
        up = np.stack([pm.upsample(I[c], fine) for c in range(4)])
        I = over(D[l], up)
    return unpremultiply(I)
