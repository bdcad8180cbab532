"""CPU mirror of the tiled stencil-chain kernel's schedule
(paper_2012_07145_gb300/csrc/k_chain.cu): the shared-memory geometry of a
tile, the split of a stage into work items (4-column block, row segment) by a
float reciprocal product, the sweeps of every stage over its rectangle with
the overlapped-tile recompute of Sec. 2 (Fig. 1), the replication of the image
edge into the out-of-image part of a border tile's rectangles, and the last
stage's direct stores.

It checks, without a GPU, what the kernel relies on:
  - the float product (it + 0.5) * rcp(nb), truncated, is the exact quotient
    it / nb for every item index and block count a tile can have;
  - every read and write of a sweep, including the rows of a last segment that
    runs past its rectangle, lies inside its buffer, and both buffers fit the
    block's shared memory;
  - every output pixel is written exactly once, by the tile that owns it, and
    reads nothing that was never written (buffers start as NaN);
  - the values equal the clamp-to-edge chain computed directly (FP64).
The geometry helpers restate the kernel's host code (chain_geom)."""

import itertools

import numpy as np
import pytest

HEADER, SMEM_LIMIT = 128, 227 * 1024 - 1024
BIN = [1 / 16, 4 / 16, 6 / 16, 4 / 16, 1 / 16]
BOX = [0.2] * 5


def geom(d, tw, th):
    W0, H0 = tw + 4 * d, th + 4 * d
    P = (W0 + 3) & ~3
    BH = min(H0, 256)
    nby = -(-H0 // BH)
    r_seg = ((H0 + 15) & ~15) + 4
    R = max(nby * BH, r_seg)
    buf = (P * R + 31) & ~31
    return dict(W0=W0, H0=H0, P=P, BH=BH, nby=nby, R=R, buf=buf, smem=HEADER + 128 + 2 * buf * 4)


def item_split(it, nb):
    """The kernel's (segment, block) of item it: float32 arithmetic, one
    correctly rounded reciprocal, one rounded sum and one rounded product."""
    rnb = np.float32(1) / np.float32(nb)
    sg = ((np.asarray(it).astype(np.float32) + np.float32(0.5)) * rnb).astype(np.int64)
    return sg, np.asarray(it) - sg * nb


def test_item_split_is_the_exact_quotient():
    # every block count of a 4-column block split up to 64 blocks (256
    # columns), every item index below 2^21
    it = np.arange(1 << 21, dtype=np.int64)
    for nb in range(1, 65):
        sg, b = item_split(it, nb)
        assert (sg == it // nb).all() and (b == it % nb).all(), nb
    # wider rectangles: shared memory bounds a tile to fewer than 2^13 items
    it = np.arange(1 << 14, dtype=np.int64)
    for nb in range(65, 1500):
        sg, b = item_split(it, nb)
        assert (sg == it // nb).all(), nb


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 8, 16, 32])
def test_sweeps_stay_inside_their_buffers(d):
    hs = [1, 2, 3, 5, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 256, 257, 300, 600]
    checked = 0
    for tw, th, seg in itertools.product(range(8, 1025, 8), hs, (4, 8, 16)):
        g = geom(d, tw, th)
        if g["smem"] > SMEM_LIMIT:
            continue
        checked += 1
        assert g["nby"] * g["BH"] <= g["R"] and g["BH"] <= 256       # the stacked TMA boxes
        assert g["buf"] % 32 == 0                                    # buffer B 128-byte aligned
        for s in range(1, d + 1):
            Ws, Hs = tw + 4 * (d - s), th + 4 * (d - s)
            nb, nseg = Ws // 4, -(-Hs // seg)
            assert Ws % 4 == 0 and nb * nseg < (1 << 21)
            assert nseg * seg + 3 <= g["R"] - 1, (d, tw, th, seg, s)  # last producer row read
            assert 4 * (nb - 1) + 7 <= g["P"] - 1                      # last producer column read
            assert nseg * seg - 1 <= g["R"] - 1                       # last row written
    assert checked > 0


def chain_reference(img, ws):
    """The chain by its definition: each stage clamps its reads to its producer."""
    s = img.astype(np.float64)
    H, W = s.shape
    xs = np.clip(np.arange(W)[:, None] + np.arange(-2, 3)[None, :], 0, W - 1)
    ys = np.clip(np.arange(H)[:, None] + np.arange(-2, 3)[None, :], 0, H - 1)
    for wx, wy in ws:
        hx = (s[:, xs] * np.array(wx)).sum(-1)
        s = (hx[ys, :] * np.array(wy)[None, :, None]).sum(1)
    return s


def fixup(buf, x0, y0, Ws, Hs, W, H):
    """The out-of-image part of a rectangle takes the value of the nearest
    in-image pixel of the same rectangle."""
    cx0, cx1 = max(0, -x0), min(Ws, W - x0)
    cy0, cy1 = max(0, -y0), min(Hs, H - y0)
    assert cx0 < cx1 and cy0 < cy1
    ys = np.clip(np.arange(Hs), cy0, cy1 - 1)
    xs = np.clip(np.arange(Ws), cx0, cx1 - 1)
    src = buf[ys[:, None], xs[None, :]].copy()          # reads only the in-image part
    inside = np.zeros((Hs, Ws), bool)
    inside[cy0:cy1, cx0:cx1] = True
    region = buf[:Hs, :Ws]
    region[~inside] = src[~inside]


def replay(img, ws, d, tw, th, seg, tma=True):
    H, W = img.shape
    g = geom(d, tw, th)
    R, P = g["R"], g["P"]
    out = np.full((H, W), np.nan)
    written = np.zeros((H, W), int)
    for by, bx in itertools.product(range(-(-H // th)), range(-(-W // tw))):
        ox, oy = bx * tw, by * th
        bufs = [np.full((R, P), np.nan), np.full((R, P), np.nan)]
        xin, yin = ox - 2 * d, oy - 2 * d
        A = bufs[0]
        if tma:     # boxes of P columns, zero outside the image, then the edge fixup
            for r, c in itertools.product(range(g["nby"] * g["BH"]), range(P)):
                y, x = yin + r, xin + c
                A[r, c] = img[y, x] if 0 <= y < H and 0 <= x < W else 0.0
            if xin < 0 or yin < 0 or xin + g["W0"] > W or yin + g["H0"] > H:
                fixup(A, xin, yin, g["W0"], g["H0"], W, H)
        else:       # clamped per-thread loads of the W0 x H0 rectangle
            for r, c in itertools.product(range(g["H0"]), range(g["W0"])):
                A[r, c] = img[min(max(yin + r, 0), H - 1), min(max(xin + c, 0), W - 1)]
        border = xin < 0 or yin < 0 or xin + g["W0"] > W or yin + g["H0"] > H
        for s in range(1, d + 1):
            src, dst = bufs[(s - 1) % 2], bufs[s % 2]
            Ws, Hs = tw + 4 * (d - s), th + 4 * (d - s)
            nb, nseg = Ws // 4, -(-Hs // seg)
            wx, wy = ws[s - 1]
            its = np.arange(nb * nseg)
            sgs, bs = item_split(its, nb)
            assert sorted(zip(sgs.tolist(), bs.tolist())) == sorted(itertools.product(range(nseg), range(nb)))
            for sg, b in zip(sgs.tolist(), bs.tolist()):
                r0 = sg * seg
                assert r0 + seg + 3 < R and 4 * b + 7 < P
                rows = src[r0:r0 + seg + 4, 4 * b:4 * b + 8]
                h = sum(wx[m] * rows[:, m:m + 4] for m in range(5))          # x pass, 4 columns
                v = sum(wy[m] * h[m:m + seg] for m in range(5))              # y pass, seg rows
                if s < d:
                    dst[r0:r0 + seg, 4 * b:4 * b + 4] = v
                    continue
                for k, c in itertools.product(range(seg), range(4)):
                    y, x = r0 + k, 4 * b + c
                    if y < th and oy + y < H and x < tw and ox + x < W:
                        out[oy + y, ox + x] = v[k, c]
                        written[oy + y, ox + x] += 1
            if s < d and border:
                fixup(dst, ox - 2 * (d - s), oy - 2 * (d - s), Ws, Hs, W, H)
    return out, written


@pytest.mark.parametrize("h,w,d,tw,th,seg,tma", [
    (23, 41, 1, 8, 6, 4, True), (37, 53, 4, 16, 10, 8, True), (29, 75, 3, 24, 7, 16, True),
    (40, 130, 2, 40, 14, 4, False), (65, 129, 4, 64, 64, 8, True), (1, 1, 4, 8, 1, 4, True),
    (2, 9, 2, 8, 6, 16, False), (70, 17, 8, 16, 33, 8, True)])
def test_tiled_schedule_writes_each_pixel_once_and_computes_the_chain(h, w, d, tw, th, seg, tma):
    img = np.random.default_rng(h * 1000 + w).random((h, w))
    ws = [(BIN, BIN) if k % 2 == 0 else (BOX, BOX) for k in range(d)]
    out, written = replay(img, ws, d, tw, th, seg, tma)
    assert (written == 1).all()
    assert np.abs(out - chain_reference(img, ws)).max() < 1e-12
