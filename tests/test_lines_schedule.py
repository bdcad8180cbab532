"""CPU mirror of the line-buffer stencil-chain kernel's schedule
(paper_2012_07145_gb300/csrc/k_chain_lines.cu): every thread's stage and
column block, the lockstep steps, the TMA boxes of the input ring, the
12-row rings of the intermediate stages, the feeds of each stage (clamped
rows, the top row entering three taps, the bottom row fed again) and the
running partial sums of the y pass.

It replays the kernel step by step on small images and checks, without a
GPU, what the kernel relies on:
  - a ring row is read only after the step that wrote it; no slot is written
    in the step that reads another row from it (the threads of one step run
    concurrently); every row read from a slot is the row the reader expects;
  - an input box is issued before the step that reads it, into a slot none
    of whose rows is read again;
  - every shared-memory access lies inside the block's allocation;
  - every output pixel is written exactly once, by the tile that owns it;
  - the values equal the clamp-to-edge chain computed directly (FP64).
The geometry helpers restate the kernel's host code (lines_geom)."""

import itertools

import numpy as np
import pytest

STEP, RING, GROUPS, HEADER = 4, 12, 4, 128
BIN = [1 / 16, 4 / 16, 6 / 16, 4 / 16, 1 / 16]
BOX = [0.2] * 5


def ru(v, m):
    return (v + m - 1) // m * m


def geom(D, tw, esize=4):
    tbase, widest = [0], 0
    for p in range(D // 2):
        nb = (tw + 4 * (D - (2 * p + 1)) + 7) // 8
        widest = max(widest, nb)
        tbase.append(tbase[-1] + 2 * nb)
    P0 = ru(tw + 4 * D, 128 // esize)
    P = ru(8 * widest, 32)
    off = HEADER
    ring_off = [off]
    off += GROUPS * STEP * P0 * esize
    for r in range(1, D):
        off = ru(off, 128) + 16 * (r & 1)
        ring_off.append(off)
        off += RING * P * 4
    return dict(tbase=tbase, threads=ru(tbase[-1], 32), P0=P0, P=P, ring_off=ring_off, smem=ru(off, 128) + 256)


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


def replay(img, ws, D, tw, th):
    H, W = img.shape
    g = geom(D, tw)
    P0, P = g["P0"], g["P"]
    usable = g["smem"] - 128          # after the kernel aligns its base to 128 bytes
    out = np.full((H, W), np.nan)
    written = np.zeros((H, W), int)
    for by, bx in itertools.product(range(-(-H // th)), range(-(-W // tw))):
        ox, oy = bx * tw, by * th
        a0, b0 = max(oy - 2 * D, 0), min(oy + th + 2 * D, H)
        ngroups = (b0 - a0 + STEP - 1) // STEP
        K = 2 * D - 1 + (min(oy + th, H) + 2 - max(oy - 2, 0) + STEP - 1) // STEP
        rings = [dict() for _ in range(D)]      # slot -> (row, values, step written)
        issued, last_read0 = {}, {}

        def issue(gi, k):
            assert gi - GROUPS not in issued or last_read0.get(gi - GROUPS, -1) < k, "box overwrites a slot in use"
            for j in range(STEP):
                r = a0 + STEP * gi + j
                vals = np.array([img[r, ox - 2 * D + c] if 0 <= r < H and 0 <= ox - 2 * D + c < W else 0.0
                                 for c in range(P0)])
                rings[0][(gi % GROUPS) * STEP + j] = (r, vals, k)
            issued[gi] = k

        threads = []
        for t in range(g["threads"]):
            for q in range(D // 2):
                if g["tbase"][q] <= t < g["tbase"][q + 1]:
                    j = t - g["tbase"][q]
                    s, b = 2 * q + 1 + (j & 1), j >> 1
                    Xp = ox - 2 * (D - s + 1)
                    ap = max(oy - 2 * (D - s + 1), 0)
                    bp = min(oy + th + 2 * (D - s + 1), H)
                    nfeed = min(oy + th + 2 * (D - s), H) + 2 - ap
                    c0 = Xp + 8 * b
                    threads.append(dict(s=s, b=b, Xp=Xp, ap=ap, bp=bp, top=ap == 0, nfeed=nfeed, Ls=2 * s - 1,
                                        nsteps=(nfeed + STEP - 1) // STEP, c0=c0,
                                        xedge=c0 < 0 or c0 + 11 > W - 1, acc=np.zeros((4, 8))))
        if ngroups > 0:
            issue(0, -1)
        for k in range(K):
            if k + 1 < ngroups:
                issue(k + 1, k)
            writes, reads = [], {}
            for T in threads:
                s, b = T["s"], T["b"]
                if not T["Ls"] <= k < T["Ls"] + T["nsteps"]:
                    continue
                if s == 1 and k - 1 < ngroups:
                    assert issued.get(k - 1, k) < k, "input box waited for before it was issued"
                wx, wy = ws[s - 1]
                acc = T["acc"]
                for u in range(STEP):
                    i = (k - T["Ls"]) * STEP + u
                    if i >= T["nfeed"]:
                        continue
                    r = min(T["ap"] + i, T["bp"] - 1)
                    if s == 1:
                        slot, pitch, elems = (r - a0) & (GROUPS * STEP - 1), P0 * 4, P0
                        last_read0[(r - a0) // STEP] = k
                    else:
                        slot, pitch, elems = r % RING, P * 4, P
                    assert slot in rings[s - 1], ("ring slot read before anything was written to it", s, r, k)
                    rr, vals, wk = rings[s - 1][slot]
                    assert rr == r and wk < k, ("ring row", s, r, rr, wk, k)
                    reads[(s - 1, slot)] = r
                    if T["xedge"]:
                        cols = [min(min(max(T["c0"] + q, 0), W - 1) - T["Xp"], elems - 1) for q in range(12)]
                    else:
                        cols = [8 * b + q for q in range(12)]
                    lo = g["ring_off"][s - 1] + slot * pitch + min(cols) * 4
                    hi = g["ring_off"][s - 1] + slot * pitch + (max(cols) + 1) * 4
                    assert 0 <= lo and hi <= usable, "shared-memory read outside the allocation"
                    x = np.array([vals[c] if c < len(vals) else np.nan for c in cols])
                    h = np.array([sum(wx[m] * x[c + m] for m in range(5)) for c in range(8)])
                    if u == 0 and T["top"] and i == 0:
                        acc[2] = wy[0] * h + wy[1] * h + wy[2] * h
                        acc[3] = wy[0] * h + wy[1] * h
                        acc[0] = wy[0] * h
                        continue
                    if i >= 4 - 2 * T["top"]:
                        o = T["ap"] + i - 2
                        v = acc[u] + wy[4] * h
                        if s < D:
                            off = g["ring_off"][s] + (o % RING) * P * 4 + 32 * b
                            assert off % 16 == 0 and off + 32 <= usable, "shared-memory write outside the allocation"
                            writes.append((s, o % RING, o, b, v))
                        else:
                            for c in range(8):
                                if 8 * b + c < tw and ox + 8 * b + c < W:
                                    assert oy <= o < min(oy + th, H), "output row outside the tile"
                                    out[o, ox + 8 * b + c] = v[c]
                                    written[o, ox + 8 * b + c] += 1
                    acc[(u + 1) & 3] += wy[3] * h
                    acc[(u + 2) & 3] += wy[2] * h
                    acc[(u + 3) & 3] += wy[1] * h
                    acc[u] = wy[0] * h
            for s, slot, o, b, v in writes:      # the step's writes, checked against its reads, then applied
                assert reads.get((s, slot), o) == o, ("slot written while read for another row", s, slot, o, k)
                if slot not in rings[s] or rings[s][slot][0] != o:
                    rings[s][slot] = (o, np.full(P, np.nan), k)
                rings[s][slot][1][8 * b:8 * b + 8] = v
                rings[s][slot] = (o, rings[s][slot][1], k)
    return out, written


@pytest.mark.parametrize("h,w,depth,tw,th", [(23, 41, 2, 8, 6), (37, 53, 4, 16, 10), (29, 75, 8, 32, 18),
                                             (40, 130, 6, 40, 14), (65, 129, 8, 64, 64), (1, 1, 4, 64, 10),
                                             (2, 9, 2, 8, 6)])
def test_line_buffer_schedule_reads_only_finished_rows_and_computes_the_chain(h, w, depth, tw, th):
    img = np.random.default_rng(h * 100 + w).random((h, w))
    ws = [(BIN, BIN) if k % 2 == 0 else (BOX, BOX) for k in range(depth)]
    out, written = replay(img, ws, depth, tw, th)
    assert (written == 1).all()
    assert np.abs(out - chain_reference(img, ws)).max() < 1e-12
