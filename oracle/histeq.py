"""Histogram equalization of a uint8 image, exact integers (oracle; test infrastructure only).

Histogram equalize is one of the imaging apps of Sec. 6 (and Sec. 6.5 / Sec. 8
discuss its parallel reduction); the paper gives no formula.  Reading used:

    h[v]   = #{p : in(p) = v},  v = 0..255
    cdf[v] = sum_{u <= v} h[u]
    cmin   = cdf[min pixel value],  N = W * H
    N == cmin (a constant image):  LUT[v] = v
    otherwise: LUT[v] = 0 if cdf[v] < cmin, else
               ((cdf[v] - cmin) * 255 * 2 + (N - cmin)) // (2 * (N - cmin))
               (round half up of (cdf[v] - cmin) / (N - cmin) * 255)
    out(p) = LUT[in(p)]

All arithmetic is on Python integers, so there is no rounding anywhere.
"""

import numpy as np


def histogram(img_u8: np.ndarray) -> list:
    """256 counts, by visiting every pixel once."""
    h = [0] * 256
    for v in np.asarray(img_u8, dtype=np.uint8).ravel().tolist():
        h[v] += 1
    return h


def cdf(h: list) -> list:
    """Inclusive prefix sum of the counts."""
    out, acc = [], 0
    for c in h:
        acc += c
        out.append(acc)
    return out


def lut(h: list) -> list:
    """Equalization lookup table (256 uint8 values) from the histogram."""
    c = cdf(h)
    n = c[-1]
    vmin = next(v for v in range(256) if h[v] > 0) if n > 0 else 0
    cmin = c[vmin]
    if n == cmin:
        return list(range(256))
    den = n - cmin
    return [0 if c[v] < cmin else ((c[v] - cmin) * 255 * 2 + den) // (2 * den) for v in range(256)]


def equalize(img_u8: np.ndarray):
    """(histogram, lut, output image) of a uint8 image."""
    img = np.asarray(img_u8, dtype=np.uint8)
    h = histogram(img)
    table = lut(h)
    out = np.asarray(table, dtype=np.uint8)[img]
    return h, table, out
