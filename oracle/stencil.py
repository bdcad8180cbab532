"""Clamp-to-edge 2-D stencils and stencil chains, FP64 (oracle; test infrastructure only).

Definition followed (Sec. 2, Fig. 1 and the stencil-chain app of Sec. 6): each
point of a stage reads a window of the previous stage.  A stage with weights
w of shape (2ry+1, 2rx+1) computes

    out(x, y) = sum_{j=-ry..ry} sum_{i=-rx..rx} w[j+ry][i+rx] * in(clamp(x+i), clamp(y+j))

with clamp(x) = min(max(x, 0), W-1) in x and the same with H-1 in y.  In a chain
every stage clamps reads of its own producer on that producer's domain (the
boundary condition belongs to each stage, not only to the pipeline input).

The 32-stage chain alternates kernels: stage k (0-based) uses the binomial
kernel outer([1,4,6,4,1],[1,4,6,4,1])/256 when k is even and the normalized
5x5 box (all weights 1/25) when k is odd.
"""

import numpy as np

BINOMIAL5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0])


def binomial5_weights() -> np.ndarray:
    """5x5 binomial kernel b (x) b / 256 with b = [1, 4, 6, 4, 1]; exact in FP64."""
    return np.outer(BINOMIAL5, BINOMIAL5) / 256.0


def box5_weights() -> np.ndarray:
    """Normalized 5x5 box: every weight 1/25 (the FP64 quotient)."""
    return np.full((5, 5), 1.0 / 25.0)


def stencil_clamp(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """One clamp-to-edge stencil stage on a single-channel image [H][W].

    Direct 2-D weighted sum over the window, one tap at a time; each tap reads
    the input at clamped coordinates (the definition above, written out).
    """
    img = np.asarray(img, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    H, W = img.shape
    ry = (w.shape[0] - 1) // 2
    rx = (w.shape[1] - 1) // 2
    assert w.shape == (2 * ry + 1, 2 * rx + 1)
    out = np.zeros((H, W), dtype=np.float64)
    ys = np.arange(H)
    xs = np.arange(W)
    for j in range(-ry, ry + 1):
        rows = np.clip(ys + j, 0, H - 1)
        for i in range(-rx, rx + 1):
            cols = np.clip(xs + i, 0, W - 1)
            out += w[j + ry, i + rx] * img[np.ix_(rows, cols)]
    return out


def chain_kinds(n_stages: int, pattern: str) -> list:
    """Kernel kind of each stage: 'binomial' for all stages, or 'alternate'
    (binomial when the 0-based stage index is even, box when it is odd)."""
    if pattern == "binomial":
        return ["binomial"] * n_stages
    if pattern == "alternate":
        return ["binomial" if k % 2 == 0 else "box" for k in range(n_stages)]
    raise ValueError(pattern)


def stencil_chain(img: np.ndarray, kinds: list) -> np.ndarray:
    """S_0 = img; S_k = stencil_k(S_{k-1}) with a per-stage clamp; returns S_n."""
    s = np.asarray(img, dtype=np.float64)
    for kind in kinds:
        w = binomial5_weights() if kind == "binomial" else box5_weights()
        s = stencil_clamp(s, w)
    return s


def stencil_chain_point(img: np.ndarray, kinds: list, x: int, y: int) -> float:
    """S_n(x, y) alone, computed from the smallest clamped window that feeds it.

    Used to check single outputs of full-size images without evaluating every
    stage everywhere.  It applies the same definition: the stage-k value at a
    point is the weighted sum of stage-(k-1) values at clamped coordinates, so
    only the stage-k values on a window of radius 2*(n-k) around (x, y),
    clamped to the image, are needed.
    """
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    n = len(kinds)
    # coordinates (already clamped) each stage is needed on
    need_x = [None] * (n + 1)
    need_y = [None] * (n + 1)
    need_x[n] = np.array([x])
    need_y[n] = np.array([y])
    for k in range(n, 0, -1):
        offs = np.arange(-2, 3)
        need_x[k - 1] = np.unique(np.clip((need_x[k][:, None] + offs[None, :]).ravel(), 0, W - 1))
        need_y[k - 1] = np.unique(np.clip((need_y[k][:, None] + offs[None, :]).ravel(), 0, H - 1))
    vals = img[np.ix_(need_y[0], need_x[0])]
    for k in range(1, n + 1):
        w = binomial5_weights() if kinds[k - 1] == "binomial" else box5_weights()
        px, py = need_x[k - 1], need_y[k - 1]
        out = np.zeros((len(need_y[k]), len(need_x[k])))
        for j in range(-2, 3):
            ry = np.searchsorted(py, np.clip(need_y[k] + j, 0, H - 1))
            for i in range(-2, 3):
                rx = np.searchsorted(px, np.clip(need_x[k] + i, 0, W - 1))
                out += w[j + 2, i + 2] * vals[np.ix_(ry, rx)]
        vals = out
    return float(vals[0, 0])
