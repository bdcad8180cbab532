"""Bilateral grid, FP64 (oracle; test infrastructure only).

The bilateral grid app of Sec. 6 (named among the Halide-repository apps; the
paper gives no definition).  Reading used here: the bilateral filter of a gray
image through the bilateral grid of Chen, Paris and Durand (2007), with spatial
cell size s (pixels) and range cell size r (intensity):

  v(x, y) = clamp(I(x, y), 0, 1);  GZ = floor(1/r + 1/2) + 1 range levels.
  Splat: grid cell (gx, gy), gx in [0, ceil(W/s)], gy in [0, ceil(H/s)], takes
    the s x s pixels (clamp(gx s + i - s/2), clamp(gy s + j - s/2)), i, j in
    [0, s); each adds (v, 1) to range level z = floor(f32(v * f32(1/r)) + 1/2)
    clamped to [0, GZ-1].  The level is an integer decided by a float, so it is
    decided in f32, as the kernel does (v * (1/r) + 1/2 with one rounding).
  Blur: [1,4,6,4,1]/16 along z, then x, then y, clamped at the grid's ends,
    for the value and the weight separately.
  Slice: at (x, y) the grid position (x/s, y/s, v/r); trilinear interpolation
    (indices clamped to the grid) of the blurred value and weight; out =
    value / weight (v where the weight is 0).
"""

import numpy as np

B5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def _r32(r: float) -> float:
    """The range cell size as the f32 parameter the pipeline is given."""
    return float(np.float32(r))


def levels(r: float) -> int:
    return int(np.floor(1.0 / _r32(r) + 0.5)) + 1


def grid_size(w: int, h: int, s: int):
    return (w + s - 1) // s + 1, (h + s - 1) // s + 1


def range_level(v: np.ndarray, r: float, gz: int) -> np.ndarray:
    """floor(v * (1/r) + 1/2) with the product and the sum rounded once to f32
    (the exact product of two f32 values fits in f64)."""
    inv_r = np.float64(np.float32(1.0 / _r32(r)))
    zf = (np.asarray(v, dtype=np.float32).astype(np.float64) * inv_r + 0.5).astype(np.float32)
    return np.clip(np.floor(zf.astype(np.float64)).astype(np.int64), 0, gz - 1)


def splat(img: np.ndarray, s: int, r: float) -> np.ndarray:
    """[GY][GX][GZ][2] grid of (sum of v, count)."""
    H, W = img.shape
    v = np.clip(np.asarray(img, dtype=np.float32), 0.0, 1.0)
    gz = levels(r)
    GX, GY = grid_size(W, H, s)
    z = range_level(v, r, gz)
    g = np.zeros((GY, GX, gz, 2))
    for gy in range(GY):
        rows = np.clip(gy * s + np.arange(s) - s // 2, 0, H - 1)
        for gx in range(GX):
            cols = np.clip(gx * s + np.arange(s) - s // 2, 0, W - 1)
            vv = v[np.ix_(rows, cols)].astype(np.float64).ravel()
            zz = z[np.ix_(rows, cols)].ravel()
            np.add.at(g[gy, gx, :, 0], zz, vv)
            np.add.at(g[gy, gx, :, 1], zz, 1.0)
    return g


def blur_axis(g: np.ndarray, axis: int) -> np.ndarray:
    n = g.shape[axis]
    out = np.zeros_like(g)
    for k in range(5):
        idx = np.clip(np.arange(n) + k - 2, 0, n - 1)
        out += B5[k] * np.take(g, idx, axis=axis)
    return out


def blur(g: np.ndarray) -> np.ndarray:
    return blur_axis(blur_axis(blur_axis(g, 2), 1), 0)   # z, then x, then y


def slice_grid(g: np.ndarray, img: np.ndarray, s: int, r: float) -> np.ndarray:
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
        zi = np.clip(z0 + dz, 0, GZ - 1)
        for dy, wy in ((0, 1 - fy), (1, fy)):
            yi = np.clip(y0 + dy, 0, GY - 1)
            for dx, wx in ((0, 1 - fx), (1, fx)):
                xi = np.clip(x0 + dx, 0, GX - 1)
                acc += (wz * wy * wx)[..., None] * g[yi, xi, zi]
    return np.where(acc[..., 1] > 0, acc[..., 0] / np.where(acc[..., 1] > 0, acc[..., 1], 1.0), v)


def bilateral_grid(img: np.ndarray, s: int = 8, r: float = 0.1) -> np.ndarray:
    """1-channel H x W image -> its bilateral-grid filtered image, FP64."""
    return slice_grid(blur(splat(img, s, r)), img, s, r)
