"""Binomial image pyramids, FP64 (oracle; test infrastructure only).

The local Laplacian app of Sec. 6 builds Gaussian and Laplacian pyramids with a
5-tap binomial filter; the paper gives no formula, so this module states the
reading (the Burt-Adelson construction):

Downsample (level l -> l+1), output size (ceil(H/2), ceil(W/2)):
    G_{l+1}(x, y) = sum_{i,j in [-2,2]} b_i b_j / 256 * G_l(clamp(2x+i), clamp(2y+j)),
    b = [1, 4, 6, 4, 1].

Upsample (coarse u -> a fine grid of a given size), per dimension the coarse
samples are zero-stuffed and filtered with 2*b/16 = [1,4,6,4,1]/8, with the
coarse index clamped to the coarse image:
    U(X) = sum_{m : |X - 2m| <= 2} a(X - 2m) * u[clamp(m)],  a(0)=6/8, a(+-1)=4/8, a(+-2)=1/8,
which gives (u[m-1] + 6u[m] + u[m+1]) / 8 at X = 2m and (u[m] + u[m+1]) / 2 at
X = 2m+1.  In 2-D the weight of coarse sample (m, n) is a(X-2m) * a(Y-2n).

Laplacian level l < J-1:  L_l = G_l - U(G_{l+1}) on G_l's grid; L_{J-1} = G_{J-1}.
Collapse: R_{J-1} = L_{J-1}, R_l = L_l + U(R_{l+1}); R_0 reconstructs G_0.
"""

import numpy as np

BINOMIAL5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0])
UP_TAPS = {-2: 1.0 / 8.0, -1: 4.0 / 8.0, 0: 6.0 / 8.0, 1: 4.0 / 8.0, 2: 1.0 / 8.0}


def down_size(n: int) -> int:
    """Size of the next coarser level: ceil(n / 2)."""
    return (n + 1) // 2


def downsample(img: np.ndarray) -> np.ndarray:
    """G_{l+1} from G_l by the 2-D sum over the 5x5 binomial window at (2x, 2y)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    h, w = down_size(H), down_size(W)
    out = np.zeros((h, w))
    ys = 2 * np.arange(h)
    xs = 2 * np.arange(w)
    for j in range(-2, 3):
        rows = np.clip(ys + j, 0, H - 1)
        for i in range(-2, 3):
            cols = np.clip(xs + i, 0, W - 1)
            out += (BINOMIAL5[j + 2] * BINOMIAL5[i + 2] / 256.0) * img[np.ix_(rows, cols)]
    return out


def upsample(coarse: np.ndarray, fine_shape: tuple) -> np.ndarray:
    """U(coarse) on a fine grid of shape (H, W), by the sum over coarse samples.

    For every pair of offsets (s, t) in [-2, 2]^2, the fine point (X, Y) takes
    coarse sample n = (Y - s)/2, m = (X - t)/2 (clamped) when both are integers,
    weighted a(s) * a(t).
    """
    coarse = np.asarray(coarse, dtype=np.float64)
    hc, wc = coarse.shape
    H, W = fine_shape
    Y = np.arange(H)
    X = np.arange(W)
    out = np.zeros((H, W))
    for s in range(-2, 3):
        row_ok = (Y - s) % 2 == 0
        n = np.clip((Y - s) // 2, 0, hc - 1)
        for t in range(-2, 3):
            col_ok = (X - t) % 2 == 0
            m = np.clip((X - t) // 2, 0, wc - 1)
            contrib = (UP_TAPS[s] * UP_TAPS[t]) * coarse[np.ix_(n, m)]
            out += np.where(row_ok[:, None] & col_ok[None, :], contrib, 0.0)
    return out


def gaussian_pyramid(img: np.ndarray, levels: int) -> list:
    """[G_0 = img, G_1, ..., G_{levels-1}]."""
    g = [np.asarray(img, dtype=np.float64)]
    for _ in range(levels - 1):
        g.append(downsample(g[-1]))
    return g


def laplacian_pyramid(gauss: list) -> list:
    """[L_0, ..., L_{J-1}] with L_l = G_l - U(G_{l+1}) and L_{J-1} = G_{J-1}."""
    lap = [gauss[l] - upsample(gauss[l + 1], gauss[l].shape) for l in range(len(gauss) - 1)]
    lap.append(gauss[-1])
    return lap


def collapse(lap: list) -> np.ndarray:
    """R_{J-1} = L_{J-1}; R_l = L_l + U(R_{l+1}); returns R_0."""
    r = lap[-1]
    for l in range(len(lap) - 2, -1, -1):
        r = lap[l] + upsample(r, lap[l].shape)
    return r
