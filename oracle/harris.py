"""Harris corner response, FP64 (oracle; test infrastructure only).

Harris corner detection is one of the imaging apps of Sec. 6; the paper does
not give its arithmetic.  This is the reading used throughout:

    g   = 0.299 R + 0.587 G + 0.114 B
    Ix  = sum_j s_j [g(x+1, y+j) - g(x-1, y+j)]      Sobel, unnormalized, s = [1,2,1]
    Iy  = sum_i s_i [g(x+i, y+1) - g(x+i, y-1)]
    Sxx = box3(Ix*Ix), Syy = box3(Iy*Iy), Sxy = box3(Ix*Iy)   3x3 sums (not means)
    R   = Sxx*Syy - Sxy^2 - k*(Sxx+Syy)^2                       k = 0.04

Every stencil clamps reads of its own producer to the image (clamp-to-edge on
g for the Sobel stage and on the product images for the box sums).  The
response is neither thresholded nor non-maximum suppressed.
"""

import numpy as np

from .stencil import stencil_clamp

GRAY_WEIGHTS = (0.299, 0.587, 0.114)
SOBEL_SMOOTH = np.array([1.0, 2.0, 1.0])
SOBEL_DIFF = np.array([-1.0, 0.0, 1.0])
HARRIS_K = 0.04


def gray(rgb: np.ndarray) -> np.ndarray:
    """Luma of a planar [3][H][W] image: 0.299 R + 0.587 G + 0.114 B."""
    rgb = np.asarray(rgb, dtype=np.float64)
    return GRAY_WEIGHTS[0] * rgb[0] + GRAY_WEIGHTS[1] * rgb[1] + GRAY_WEIGHTS[2] * rgb[2]


def sobel_x_weights() -> np.ndarray:
    """w[j][i] = s_j * d_i: derivative along x, smoothing along y."""
    return np.outer(SOBEL_SMOOTH, SOBEL_DIFF)


def sobel_y_weights() -> np.ndarray:
    """w[j][i] = d_j * s_i: derivative along y, smoothing along x."""
    return np.outer(SOBEL_DIFF, SOBEL_SMOOTH)


def harris_stages(rgb: np.ndarray, k: float = HARRIS_K) -> dict:
    """All intermediate stages, in definition order."""
    g = gray(rgb)
    ix = stencil_clamp(g, sobel_x_weights())
    iy = stencil_clamp(g, sobel_y_weights())
    box = np.ones((3, 3))
    sxx = stencil_clamp(ix * ix, box)
    syy = stencil_clamp(iy * iy, box)
    sxy = stencil_clamp(ix * iy, box)
    r = sxx * syy - sxy * sxy - k * (sxx + syy) ** 2
    return dict(gray=g, ix=ix, iy=iy, sxx=sxx, syy=syy, sxy=sxy, response=r)


def harris(rgb: np.ndarray, k: float = HARRIS_K) -> np.ndarray:
    """Harris response R [H][W] of a planar RGB image [3][H][W]."""
    return harris_stages(rgb, k)["response"]
