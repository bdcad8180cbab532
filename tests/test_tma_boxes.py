"""CPU mirror of every tensor copy (cp.async.bulk.tensor) the kernels issue.

A tensor copy faults the GPU when its innermost start coordinate times the
element size is not a multiple of 16 bytes (nothing checks it before the copy
runs), when its shared-memory destination does not start on a 128-byte
boundary, or when the box's row is not a multiple of 16 bytes (the encode
call refuses it).  A box dimension is at most 256 elements.  This file
restates, kernel by kernel, the host geometry that sets each box (its
dimensions, its start coordinates and its destination slot) and checks those
rules for every box a launch can issue, together with the accounting the
kernels rely on: the bytes each mbarrier expects equal the box's, every slot
and barrier lies inside the block's shared memory, and every lane's read of a
slot lies inside the box.  Nothing here touches a GPU."""

import itertools

import pytest

SMEM_LIMIT = 227 * 1024 - 1024
ESIZE = {"f32": 4, "f16": 2, "bf16": 2}


def ru(v, m):
    return (v + m - 1) // m * m


def check_box(dims, esize, x, dst, expect_tx=None):
    """The rules of one tensor copy: dims (inner first), start column x, the
    destination's offset from a 128-byte aligned base."""
    assert all(1 <= d <= 256 for d in dims), dims
    assert dims[0] * esize % 16 == 0, ("box row not a multiple of 16 bytes", dims, esize)
    assert x * esize % 16 == 0, ("start column not 16-byte aligned", x, esize)
    assert dst % 128 == 0, ("destination not 128-byte aligned", dst)
    nbytes = esize
    for d in dims:
        nbytes *= d
    if expect_tx is not None:
        assert expect_tx == nbytes, (expect_tx, nbytes)
    return nbytes


# ---------------------------------------------------------------------------
# k_chain (tiled): stage 0 as stacked boxes, straight into buffer A (f32 whose
# halo origin is 16-byte aligned) or staged in buffer B and converted
# ---------------------------------------------------------------------------

def chain_geom(d, tw, th):
    W0, H0 = tw + 4 * d, th + 4 * d
    P = (W0 + 3) & ~3
    BH = min(H0, 256)
    nby = -(-H0 // BH)
    R = max(nby * BH, ((H0 + 15) & ~15) + 4)
    buf = (P * R + 31) & ~31
    return dict(W0=W0, H0=H0, P=P, BH=BH, nby=nby, buf=buf)


def chain_boxes(d, tw, th, dt, tiles_x):
    """(dims, start column, destination, expected bytes) of every box of every
    tile column, or None where stage 0 takes the clamped per-thread loads."""
    g = chain_geom(d, tw, th)
    esize = ESIZE[dt]
    align = 16 // esize
    xin0 = -2 * d
    off = xin0 % align            # equals ((xin % align) + align) % align in C
    header = 128
    boxes = []
    direct = dt == "f32" and off == 0 and g["P"] <= 256
    if direct:
        bw, base, sub = g["P"], header, 0
    else:
        sbw = ru(g["W0"] + off, align)
        if not (sbw <= 256 and g["nby"] * g["BH"] * sbw * esize <= g["buf"] * 4):
            return None, g
        bw, base, sub = sbw, header + g["buf"] * 4, off
    tx = g["nby"] * g["BH"] * bw * esize
    for bx, k in itertools.product(range(tiles_x), range(g["nby"])):
        boxes.append(((bw, g["BH"], 1), bx * tw + xin0 - sub, base + k * g["BH"] * bw * esize, None))
    # the region the boxes fill lies inside the header and the two buffers
    end = header + (1 if direct else 2) * g["buf"] * 4
    assert max(b[2] for b in boxes) + g["BH"] * bw * esize <= end
    return (boxes, tx), g


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_tiled_chain_boxes(dt):
    esize = ESIZE[dt]
    checked = 0
    for d, tw, th in itertools.product(list(range(1, 9)) + [16, 32], range(8, 257, 8),
                                       (1, 6, 16, 31, 64, 100, 200, 252, 300)):
        res, g = chain_boxes(d, tw, th, dt, tiles_x=6)
        if 128 + 128 + 2 * g["buf"] * 4 > SMEM_LIMIT or res is None:
            continue
        boxes, tx = res
        total = sum(check_box(dims, esize, x, dst) for dims, x, dst, _ in boxes) // 6
        assert total == tx          # one mbarrier expects every box of the tile
        assert tx < 1 << 20         # within an mbarrier's transaction count
        checked += 1
    assert checked > 100


# ---------------------------------------------------------------------------
# k_chain_lines: the 16-row input ring, four boxes of kStep rows
# ---------------------------------------------------------------------------

L_STEP, L_RING, L_GROUPS, L_HEADER = 4, 12, 4, 128


def lines_geom(D, tw, esize):
    tbase, widest = [0], 0
    for p in range(D // 2):
        nb = (tw + 4 * (D - (2 * p + 1)) + 7) // 8
        widest = max(widest, nb)
        tbase.append(tbase[-1] + 2 * nb)
    P0 = ru(tw + 4 * D, 128 // esize)
    P = ru(8 * widest, 32)
    off = L_HEADER + L_GROUPS * L_STEP * P0 * esize
    for r in range(1, D):
        off = ru(off, 128) + 16 * (r & 1) + L_RING * P * 4
    return dict(threads=ru(tbase[-1], 32), P0=P0, smem=ru(off, 128) + 256)


def lines_ok(D, tw, th, esize):
    if D < 2 or D > 8 or D % 2 or (2 * D * esize) % 16 or tw < 8 or tw % 8 or th < 2 * D + 2:
        return False
    g = lines_geom(D, tw, esize)
    return g["P0"] <= 256 and g["threads"] <= 256 and g["smem"] <= SMEM_LIMIT


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_line_buffer_chain_boxes(dt):
    esize = ESIZE[dt]
    checked = 0
    for D, tw, th in itertools.product((2, 4, 6, 8), range(8, 257, 8), (16, 18, 32, 64, 256)):
        if not lines_ok(D, tw, th, esize):
            continue
        g = lines_geom(D, tw, esize)
        assert L_GROUPS * 8 <= 64                        # the mbarriers, then the abort flag at byte 64
        for bx, gi in itertools.product(range(6), range(9)):
            dst = L_HEADER + (gi % L_GROUPS) * L_STEP * g["P0"] * esize
            check_box((g["P0"], L_STEP, 1), esize, bx * tw - 2 * D, dst, expect_tx=L_STEP * g["P0"] * esize)
            assert dst + L_STEP * g["P0"] * esize <= L_HEADER + L_GROUPS * L_STEP * g["P0"] * esize
        checked += 1
    assert checked > 20


# ---------------------------------------------------------------------------
# The streaming kernels: per-warp rings of kRing slots behind kBarBytes of
# mbarriers; warp w's slot s starts at kBarBytes + (w kRing + s) slot_bytes
# from the 128-byte aligned base; box q of a warp goes to slot q % kRing.
# Every kernel takes at most 256 threads (8 warps).
# ---------------------------------------------------------------------------

def check_ring(esize, box, xs, slot_bytes, kring, bar_bytes, reads, warps=8):
    """reads: (first element, elements, vector bytes) of each lane's loads
    from a slot, counted from the slot's start."""
    assert warps * kring * 8 <= bar_bytes                      # the ring's mbarriers
    assert 128 + bar_bytes + warps * kring * slot_bytes <= SMEM_LIMIT
    nbytes = None
    for w, s, x in itertools.product(range(warps), range(kring), xs):
        dst = bar_bytes + (w * kring + s) * slot_bytes
        nbytes = check_box(box, esize, x, dst)
    assert nbytes <= slot_bytes
    elems = nbytes // esize
    for first, n, vec in reads:
        assert 0 <= first and first + n <= elems, (first, n, elems)
        assert (first * esize) % vec == 0, (first, vec)
    return nbytes


def strip_geom_rows(esize):
    """k_stencil_rows / k_harris_rows: lanes of 4 columns, halo lanes so that
    a box starts on a 16-byte boundary."""
    hl = 1 if esize == 4 else 2
    return hl, 4 * (32 - 2 * hl)


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_streaming_stencil_boxes(dt):
    esize = ESIZE[dt]
    hl, sw = strip_geom_rows(esize)
    xs = [s * sw - 4 * hl for s in range(60)]
    reads = [(rr * 128 + 4 * lane, 4, 4 * esize) for rr, lane in itertools.product(range(4), range(32))]
    check_ring(esize, (128, 4, 1), xs, 128 * 4 * esize, 3, 512, reads)


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_streaming_harris_boxes(dt):
    esize = ESIZE[dt]
    hl, sw = strip_geom_rows(esize)
    xs = [s * sw - 4 * hl for s in range(60)]
    reads = [(pl * 128 * 2 + u * 128 + 4 * lane, 4, 4 * esize)
             for pl, u, lane in itertools.product(range(3), range(2), range(32))]
    check_ring(esize, (128, 2, 3), xs, 128 * 2 * 3 * esize, 4, 512, reads)


@pytest.mark.parametrize("dt,depth,cols", [(dt, d, c) for dt in ESIZE for d in (1, 2, 3, 4) for c in (4, 8)])
def test_streaming_chain_boxes(dt, depth, cols):
    esize = ESIZE[dt]
    hl = (2 * depth + cols - 1) // cols
    if esize == 2 and (cols * hl) % 8:
        hl += 1
    sw = cols * (32 - 2 * hl)
    assert sw > 0
    xs = [s * sw - cols * hl for s in range(60)]
    reads = [(rr * 32 * cols + cols * lane, cols, 4 * esize) for rr, lane in itertools.product(range(4), range(32))]
    check_ring(esize, (32 * cols, 4, 1), xs, 32 * cols * 4 * esize, 3, 256, reads)


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_max_filter_boxes(dt):
    esize = ESIZE[dt]
    pad = 4 if esize == 2 else 0
    box_w = 136 if esize == 2 else 128
    slot = ru(box_w * 4 * esize, 128)
    xs = [120 * s - 4 - pad for s in range(60)]
    reads = [(rr * box_w + 4 * lane + pad, 4, 4 * esize) for rr, lane in itertools.product(range(4), range(32))]
    # (a bf16 box is 1088 bytes: slots a box apart would not start on 128-byte
    # boundaries, so they are spaced at the next multiple of 128)
    check_ring(esize, (box_w, 4, 1), xs, slot, 3, 512, reads)


def test_interpolate_level_boxes():
    # fine level f32 RGBA: box of 68 columns x 2 rows x 4 planes from 4
    # columns left of the strip's first fine column (30 coarse columns a strip)
    xs = [2 * (30 * s) - 4 for s in range(60)]
    reads = []
    for W, s, lane in itertools.product((1, 2, 61, 64, 121, 640), range(3), range(32)):
        m = 30 * s + lane - 1
        if 2 * (30 * s) > W - 1:
            continue
        X0, X1 = min(max(2 * m, 0), W - 1), min(max(2 * m + 1, 0), W - 1)
        c0, c1 = X0 - (60 * s - 4), X1 - (60 * s - 4)
        pair = 2 * m >= 0 and 2 * m + 1 <= W - 1
        for ch, odd in itertools.product(range(4), range(2)):
            q = (2 * ch + odd) * 68
            if pair:
                reads.append((q + c0, 2, 8))
            else:
                reads += [(q + c0, 1, 4), (q + c1, 1, 4)]
    check_ring(4, (68, 2, 4), xs, 2304, 3, 512, reads)


def test_tiled_harris_boxes():
    # three planes of the gray's rectangle plus its halo, staged after the
    # gray buffer, from A = 16 / esize columns left of the tile
    for esize, tw, th in itertools.product((4, 2), range(8, 233, 8), (1, 8, 16, 64, 128, 252)):
        GW, GH, Pg, Pp, PH = tw + 4, th + 4, tw + 12, tw + 8, th + 2
        A = 16 // esize
        off = A - 2
        bw = ru(GW + off, A)
        gray_floats = (Pg * GH + 31) & ~31
        staging = bw * GH * 3 * esize
        region = ru(max(staging, 3 * Pp * PH * 4), 128)
        if bw > 256 or GH > 256 or 128 + 128 + gray_floats * 4 + region > SMEM_LIMIT:
            continue
        for bx in range(6):
            check_box((bw, GH, 3), esize, bx * tw - A, 128 + gray_floats * 4, expect_tx=staging)
        assert staging <= region
        # every gray column x (0 .. GW-1) is box column x + off
        assert off >= 0 and GW - 1 + off < bw
