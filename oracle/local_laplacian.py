"""Local Laplacian filter, FP64 (oracle; test infrastructure only).

The local Laplacian app of Sec. 6 is named but not defined in the paper.  This
follows the published method of Paris, Hasinoff and Kautz (2011) with the
discretised intensity levels of Aubry et al. (2014):

  input uint16 RGB -> v / 65535; gray = 0.299 R + 0.587 G + 0.114 B.
  K intensity levels g_k = k / (K-1), k = 0..K-1.
  Remap with d = i - g:
      |d| <= sigma_r:  r(i) = g + sign(d) * sigma_r * (|d| / sigma_r)^alpha
      otherwise:       r(i) = g + sign(d) * (beta * (|d| - sigma_r) + sigma_r)
  For each k: Gaussian pyramid (J levels) of r_k(gray) and its Laplacian pyramid.
  Gaussian pyramid of gray itself.
  Output Laplacian, level l < J-1, pixel p:
      t = G_l[gray](p) * (K-1), k0 = min(floor(t), K-2), f = t - k0,
      L'_l(p) = (1-f) L_l[r_k0](p) + f L_l[r_k0+1](p)
  Residual L'_{J-1} = G_{J-1}[gray]; collapse gives out_gray.
  Colour: out_c = in_c * out_gray / gray where gray > 0, else out_gray.
  uint16 output: clamp(rint(out_c * 65535), 0, 65535)   (rint rounds half to even).

With alpha = beta = 1 the remap is the identity, every level's interpolated
Laplacian equals L_l[gray] and the collapse telescopes back to gray, so the
filter returns its input; the tests use that as a pin.
"""

import numpy as np

from .pyramid import gaussian_pyramid, laplacian_pyramid, collapse

GRAY_WEIGHTS = (0.299, 0.587, 0.114)


def remap(i: np.ndarray, g: float, sigma_r: float, alpha: float, beta: float) -> np.ndarray:
    """Paris et al. point-wise remapping of intensities i around the level g."""
    i = np.asarray(i, dtype=np.float64)
    d = i - g
    ad = np.abs(d)
    sgn = np.sign(d)
    with np.errstate(divide="ignore", invalid="ignore"):
        inside = g + sgn * sigma_r * np.power(ad / sigma_r, alpha)
    outside = g + sgn * (beta * (ad - sigma_r) + sigma_r)
    return np.where(ad <= sigma_r, np.where(ad == 0.0, g, inside), outside)


def local_laplacian_float(rgb_u16: np.ndarray, levels: int = 8, k_levels: int = 8,
                          sigma_r: float = 0.1, alpha: float = 1.0, beta: float = 1.0) -> np.ndarray:
    """Float result out_c (before quantisation), planar [3][H][W], in [0,1] units."""
    inp = np.asarray(rgb_u16, dtype=np.float64) / 65535.0
    gray = GRAY_WEIGHTS[0] * inp[0] + GRAY_WEIGHTS[1] * inp[1] + GRAY_WEIGHTS[2] * inp[2]
    g_pyr = gaussian_pyramid(gray, levels)
    lap_k = []
    for k in range(k_levels):
        gk = k / (k_levels - 1)
        lap_k.append(laplacian_pyramid(gaussian_pyramid(remap(gray, gk, sigma_r, alpha, beta), levels)))
    out_lap = []
    for l in range(levels - 1):
        t = g_pyr[l] * (k_levels - 1)
        k0 = np.minimum(np.floor(t), k_levels - 2).astype(np.int64)
        f = t - k0
        stack = np.stack([lap_k[k][l] for k in range(k_levels)])
        lo = np.take_along_axis(stack, k0[None], axis=0)[0]
        hi = np.take_along_axis(stack, (k0 + 1)[None], axis=0)[0]
        out_lap.append((1.0 - f) * lo + f * hi)
    out_lap.append(g_pyr[levels - 1])
    out_gray = collapse(out_lap)
    ratio_ok = gray > 0
    safe = np.where(ratio_ok, gray, 1.0)
    out = np.where(ratio_ok[None], inp * (out_gray / safe)[None], out_gray[None])
    return out


def quantize_u16(x: np.ndarray) -> np.ndarray:
    """clamp(rint(x * 65535), 0, 65535) as uint16."""
    return np.clip(np.rint(np.asarray(x, dtype=np.float64) * 65535.0), 0, 65535).astype(np.uint16)


def local_laplacian(rgb_u16: np.ndarray, levels: int = 8, k_levels: int = 8,
                    sigma_r: float = 0.1, alpha: float = 1.0, beta: float = 1.0) -> np.ndarray:
    """uint16 planar [3][H][W] output of the local Laplacian filter."""
    return quantize_u16(local_laplacian_float(rgb_u16, levels, k_levels, sigma_r, alpha, beta))
