"""Benchmark-driven autotuner for fusion depth, tile shape and thread mapping.

The paper's autotuning mode compiles and benchmarks candidate schedules and
keeps the fastest (Sec. 6, "Autotuning").  Here every candidate is a runtime
schedule of the same compiled kernels, so a candidate costs one launch
sequence, not a compile.  The candidate space follows Sec. 4.1-4.3:

  - fusion depth d (how many consecutive stages share a kernel),
  - tile width (innermost thread dimension 16/32/64 x 4 columns per thread),
    tile height (powers of two),
  - threads per block and serial rows per thread (1, 2, 4, 8 plus odd 3, 5, 7
    and longer segments),

pruned by the rules of Sec. 4.6: hardware limits (shared memory per block,
threads), too few blocks to keep every SM busy (fewer than 2 x SMs, Sec. 4.3),
and thread counts that leave most threads idle.  Every timed candidate's
output is compared bit for bit with the stage-per-kernel result, so tuning
also checks schedule invariance.  Results go to schedules.json, keyed by
workload.

For the application pipelines (Harris, unsharp mask, histogram equalize) the
space is the grouping -- every stage its own kernel, or the whole pipeline in
one group -- crossed with the kernels that can run the one group: the tiled
kernel over its tile shapes, threads and serial rows, the streaming kernel
over run lengths and threads, and the generic interpreter.  Those results
are keyed by application and image size ("harris_2560x1536"), since the best
run length and tile depend on how many tiles or runs the image has per SM.
"""

import argparse
import itertools
import json
import os
import statistics
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
DB_PATH = os.path.join(PKG, "schedules.json")
SMS = 152
SMEM_LIMIT = 227 * 1024 - 1024


def chain_smem_bytes(depth, tile_w, tile_h):
    """Mirror of the kernel's shared-memory plan (two ping-pong buffers)."""
    W0, H0 = tile_w + 4 * depth, tile_h + 4 * depth
    P = (W0 + 3) & ~3
    BH = min(H0, 256)
    R = max((H0 + BH - 1) // BH * BH, ((H0 + 15) & ~15) + 4)
    buf = (P * R + 31) & ~31
    return 256 + 2 * buf * 4


def chain_candidates(n_stages, W, H, quick=False):
    depths = [d for d in (1, 2, 4, 8, 16, 32) if n_stages % d == 0]
    tws = (32, 64, 128) if not quick else (64, 128)
    ths = (16, 32, 64, 128) if not quick else (32, 64)
    # thread counts that are not powers of two too: a stage's work items
    # (4-column blocks x row segments) rarely divide 256, and the threads left
    # over wait at the stage barrier
    threads = (96, 128, 160, 192, 224, 256, 320, 384, 512) if not quick else (192, 256)
    serials = (4, 8, 16) if not quick else (8, 16)
    out = []
    for d, tw, th, t, s in itertools.product(depths, tws, ths, threads, serials):
        if chain_smem_bytes(d, tw, th) > SMEM_LIMIT:
            continue                                   # hardware limit
        blocks = -(-W // tw) * -(-H // th)
        if blocks < 2 * SMS and (tw > 32 or th > 16):
            continue                                   # leaves SMs idle
        items = (tw // 4) * -(-th // s)
        if items < t // 2:
            continue                                   # most threads idle in the last stage
        out.append(dict(depth=d, tile_w=tw, tile_h=th, threads=t, serial_y=s))
    return out


def time_candidate(p, bi, bo, stream, flush, reps=15):
    import torch
    s = stream.cuda_stream
    p.realize(bi, bo, s)   # uncaptured first run
    p.realize(bi, bo, s)   # graph capture
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.realize(bi, bo, s)
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(x.elapsed_time(y) for x, y in ts)


def tune_chain(name, n_stages=32, pattern="alternate", W=2560, H=1536, quick=False, log=print):
    import torch
    from . import hp, pipelines, synth
    img = synth.stencil_input(H, W, seed=0)
    x = hp.padded_copy(torch.from_numpy(img), "cuda")
    ref = hp.padded_empty(1, H, W, torch.float32, "cuda")
    y = hp.padded_empty(1, H, W, torch.float32, "cuda")
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    bi = [hp.buffer_from_tensor(x, hp.HP_F32)]
    p = pipelines.stencil_chain(n_stages, pattern)
    p.use_cuda_graph(True)
    p.realize(bi, hp.buffer_from_tensor(ref, hp.HP_F32), stream.cuda_stream)
    plain_ms = time_candidate(p, bi, hp.buffer_from_tensor(y, hp.HP_F32), stream, flush)
    log(f"plain stage-per-kernel: {plain_ms:.4f} ms")
    best = None
    results = []
    for c in chain_candidates(n_stages, W, H, quick):
        try:
            pipelines.chain_schedule(p, **c)
            ms = time_candidate(p, bi, hp.buffer_from_tensor(y, hp.HP_F32), stream, flush)
        except hp.HPError as e:
            log(f"skip {c}: {e}")
            continue
        same = torch.equal(y.view(torch.int32), ref.view(torch.int32))
        if not same:
            raise RuntimeError(f"schedule {c} changed the result: schedules must be bit-identical")
        results.append((ms, c))
        if best is None or ms < best[0]:
            best = (ms, c)
            log(f"best so far {ms:.4f} ms {c}")
    results.sort(key=lambda r: r[0])
    return dict(params=best[1], ms=best[0], plain_ms=plain_ms, candidates=len(results),
                top5=[dict(ms=m, **c) for m, c in results[:5]], device=torch.cuda.get_device_name())


# ------------------------------------------------------------ applications --
def apply_schedule(p, entry):
    """Applies a schedule entry of schedules.json (an application's) to p."""
    from . import pipelines
    kind = entry["schedule"]
    if kind == "root":
        pipelines.root_schedule(p)
    elif kind == "fused":
        pipelines.fused_schedule(p, tile_w=entry.get("tile_w", 32), tile_h=entry.get("tile_h", 32),
                                 threads=entry.get("threads", 256), impl=entry.get("impl"))
        if entry.get("serial_y"):
            n = len(p.stages)
            p.schedule([0] * n, tile_w=[entry["tile_w"]], tile_h=[entry["tile_h"]], threads=[entry["threads"]],
                       serial_y=[entry["serial_y"]], impl=[entry["impl"]] if entry.get("impl") is not None else None)
    else:
        raise ValueError(f"unknown schedule kind {kind}")


def app_candidates(app):
    from . import hp
    out = [dict(schedule="root")]
    if app == "histeq":
        return out + [dict(schedule="fused")]
    out.append(dict(schedule="fused", impl=hp.HP_IMPL_GENERIC, tile_w=32, tile_h=32, threads=256))
    tiled_w = (32, 64, 96) if app.startswith("harris") else (64, 128)
    for tw, th, t, sy in itertools.product(tiled_w, (16, 32, 64), (128, 256), (4, 8)):
        out.append(dict(schedule="fused", impl=hp.HP_IMPL_AUTO, tile_w=tw, tile_h=th, threads=t, serial_y=sy))
    runs = (8, 11, 14, 17, 20, 26, 32) if app.startswith("harris") else (12, 16, 20, 24, 32, 48, 64, 96)
    strip = 112 if app.endswith("bf16") else 120      # 2-byte inputs take 112-column strips
    for th, t in itertools.product(runs, (128, 256)):
        out.append(dict(schedule="fused", impl=hp.HP_IMPL_WAVE, tile_w=strip, tile_h=th, threads=t))
    return out


def app_io(app, H, W):
    """Seeded input and output buffers of an application at H x W."""
    import torch
    from . import hp, pipelines, synth
    if app == "harris":
        p, img, idt, oc, odt, tdt = pipelines.harris(), synth.rgb_f32(H, W, seed=0), hp.HP_F32, 1, hp.HP_F32, torch.float32
    elif app == "harris_bf16":   # bf16 input, intermediates and output; f32 arithmetic
        p = pipelines.harris(io_storage=hp.HP_BF16, inner_storage=hp.HP_BF16)
        img, idt, oc, odt, tdt = synth.rgb_f32(H, W, seed=0), hp.HP_BF16, 1, hp.HP_BF16, torch.bfloat16
    elif app == "unsharp":
        p, img, idt, oc, odt, tdt = pipelines.unsharp(), synth.rgb_f32(H, W, seed=0), hp.HP_F32, 3, hp.HP_F32, torch.float32
    elif app == "histeq":
        p, img, idt, oc, odt, tdt = (pipelines.histeq(), synth.gray_u8_lowcontrast(H, W, seed=0), hp.HP_U8, 1, hp.HP_U8,
                                     torch.uint8)
    else:
        raise ValueError(app)
    t = torch.from_numpy(img)
    x = hp.padded_copy(t.to(tdt) if tdt in (torch.bfloat16, torch.float16) else t, "cuda")
    ref = hp.padded_empty(oc, H, W, tdt, "cuda")
    y = hp.padded_empty(oc, H, W, tdt, "cuda")
    return p, [hp.buffer_from_tensor(x, idt)], ref, y, odt   # the buffer keeps x alive


def tune_app(app, W, H, log=print):
    import torch
    from . import hp
    p, bi, ref, y, odt = app_io(app, H, W)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    p.use_cuda_graph(True)
    p.realize(bi, hp.buffer_from_tensor(ref, odt), stream.cuda_stream)   # the default (stage-per-kernel) result
    torch.cuda.synchronize()
    as_bits = ((lambda t: t.view(torch.int32)) if ref.dtype == torch.float32 else
               (lambda t: t.view(torch.int16)) if ref.dtype in (torch.bfloat16, torch.float16) else (lambda t: t))
    results = []
    plain_ms = None
    for c in app_candidates(app):
        try:
            apply_schedule(p, c)
            ms = time_candidate(p, bi, hp.buffer_from_tensor(y, odt), stream, flush)
        except hp.HPError as e:
            log(f"skip {c}: {e}")
            continue
        if not torch.equal(as_bits(y), as_bits(ref)):
            raise RuntimeError(f"schedule {c} changed the result: schedules must be bit-identical")
        if p.device_error():
            raise RuntimeError(f"schedule {c} reported a device error")
        if c["schedule"] == "root":
            plain_ms = ms
        results.append((ms, c))
        log(f"{ms:.4f} ms {c}")
    results.sort(key=lambda r: r[0])
    best = results[0]
    return dict(params=best[1], ms=best[0], plain_ms=plain_ms, candidates=len(results),
                top5=[dict(ms=m, **c) for m, c in results[:5]], device=torch.cuda.get_device_name())


def save(name, entry):
    db = json.load(open(DB_PATH)) if os.path.exists(DB_PATH) else {}
    db[name] = entry
    with open(DB_PATH, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="chain32")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out", default=None, help="also write the entry to this JSON file")
    ap.add_argument("--sizes", default="2560x1536", help="applications: comma-separated WxH image sizes")
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(PKG))
    import __graft_entry__
    __graft_entry__.build()
    entries = {}
    if args.config == "chain32":
        entries["chain32"] = tune_chain("chain32", 32, "alternate", 2560, 1536, args.quick)
    elif args.config == "chain4":
        entries["chain4"] = tune_chain("chain4", 4, "binomial", 512, 512, args.quick)
    elif args.config in ("harris", "harris_bf16", "unsharp", "histeq"):
        sizes = [(int(a), int(b)) for a, b in (s.split("x") for s in args.sizes.split(","))]
        for W, H in sizes:
            entries[f"{args.config}_{W}x{H}"] = tune_app(args.config, W, H)
    else:
        raise SystemExit(f"unknown config {args.config}")
    for k, e in entries.items():
        save(k, e)
    if args.out:
        json.dump(entries, open(args.out, "w"), indent=1)
    print(json.dumps(entries))


if __name__ == "__main__":
    main()
