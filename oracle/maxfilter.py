"""Max filter, exact (oracle; test infrastructure only).

The max filter app of Sec. 6 (named among the Halide-repository apps; the
paper gives no definition).  Reading used here, per channel, with the
clamp-to-edge boundary of every stage:

    out(x, y) = max_{|i| <= rx, |j| <= ry} in(clamp(x + i, 0, W-1), clamp(y + j, 0, H-1))

The pipeline computes it as two stages, a horizontal maximum (rx, 0) and a
vertical one (0, ry); because the clamp acts on each coordinate separately the
two stages give exactly the 2-D window maximum.  Maxima are exact, so there is
no rounding anywhere: the GPU result must equal this one bit for bit.
"""

import numpy as np


def max_filter(img: np.ndarray, rx: int, ry: int) -> np.ndarray:
    """2-D window maximum of one channel (H x W), clamp-to-edge: the maximum
    over the (2rx+1)(2ry+1) shifted copies of the image."""
    img = np.asarray(img)
    H, W = img.shape
    ys = np.arange(H)
    xs = np.arange(W)
    out = None
    for j in range(-ry, ry + 1):
        rows = np.clip(ys + j, 0, H - 1)
        for i in range(-rx, rx + 1):
            cols = np.clip(xs + i, 0, W - 1)
            v = img[np.ix_(rows, cols)]
            out = v.copy() if out is None else np.maximum(out, v)
    return out


def max_filter_planes(img: np.ndarray, rx: int, ry: int) -> np.ndarray:
    """Per channel of a [C][H][W] image."""
    return np.stack([max_filter(img[c], rx, ry) for c in range(img.shape[0])])
