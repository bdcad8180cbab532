"""Benchmark-driven autotuner for fusion grouping, kernel choice, tile shape and
thread mapping.

The paper's autotuning mode compiles and benchmarks candidate schedules and
keeps the fastest (Sec. 6, "Autotuning").  Here every candidate is a runtime
schedule of the same compiled kernels, so a candidate costs one launch
sequence, not a compile.  The candidate spaces follow Sec. 4.1-4.3:

  - fusion depth d (how many consecutive stages share a kernel),
  - the kernel of a fused group: tiled (tile width 32/64/128, tile height a
    power of two, threads per block, serial rows per thread -- 4, 8, 16), or
    streaming (one warp per column strip, 4 or 8 columns per lane, rows per
    run, threads per block), or the generic interpreter,
  - for the local Laplacian, per pyramid level: streaming or tiled kernels,
    rows per run and threads,

pruned by the rules of Sec. 4.6: hardware limits (shared memory per block,
threads), too few blocks to keep the SMs busy (fewer than half the SMs, Sec.
4.3; small images that live in L2 still gain from larger tiles than 2 x SMs
blocks would allow),
thread counts that leave most threads idle, and kernels that spill registers
to local memory (measured: the library reports the register and local-memory
figures of the kernels a realize launched).  Every timed candidate's output is
compared bit for bit with the stage-per-kernel result, so tuning also checks
schedule invariance.

Results go to schedules.json, keyed by (pipeline, width x height, storage
type): "stencil_chain_32_alternate/2560x1536/f32", "harris/2560x1536/bf16",
since the best tile, depth and run length depend on how many tiles or runs the
image has per SM and on the bytes per value.
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
DTYPES = ("f32", "f16", "bf16", "u8", "u16")


def key(pipeline, w, h, dtype):
    return f"{pipeline}/{w}x{h}/{dtype}"


def parse_key(k):
    pipeline, size, dtype = k.split("/")
    w, h = (int(v) for v in size.split("x"))
    return pipeline, w, h, dtype


def load_db():
    return json.load(open(DB_PATH)) if os.path.exists(DB_PATH) else {}


def lookup(pipeline, w, h, dtype):
    """The stored entry of a workload, or None."""
    return load_db().get(key(pipeline, w, h, dtype))


def save(k, entry):
    db = load_db()
    db[k] = entry
    with open(DB_PATH, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)


# ------------------------------------------------------------- stencil chain --
def chain_smem_bytes(depth, tile_w, tile_h):
    """Mirror of the tiled chain kernel's shared-memory plan (two ping-pong buffers)."""
    W0, H0 = tile_w + 4 * depth, tile_h + 4 * depth
    P = (W0 + 3) & ~3
    BH = min(H0, 256)
    R = max((H0 + BH - 1) // BH * BH, ((H0 + 15) & ~15) + 4)
    buf = (P * R + 31) & ~31
    return 256 + 2 * buf * 4


def chain_strip_w(depth, cols, esize):
    """Mirror of the streaming chain kernel's strip width: whole lanes of halo
    covering 2 depth columns on each side (a 16-byte aligned box start)."""
    hl = -(-2 * depth // cols)
    if esize == 2 and (cols * hl) % 8:
        hl += 1
    return cols * (32 - 2 * hl)


def chain_candidates(n_stages, W, H, quick=False, esize=4):
    from . import hp
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
        if blocks < SMS // 2 and (tw > 32 or th > 16):
            continue                                   # leaves most SMs idle
        items = (tw // 4) * -(-th // s)
        if items < t // 2:
            continue                                   # most threads idle in the last stage
        out.append(dict(depth=d, tile_w=tw, tile_h=th, threads=t, serial_y=s))
    # the line-buffer kernel: an even depth, tile widths with tile_w + 4 depth
    # at most 256 columns (one TMA box), tile heights of at least 2 depth + 2
    for d, tw, th in itertools.product((2, 4, 6, 8), (32, 64, 96, 112, 128, 144, 160, 176, 192, 224, 240),
                                       (16, 32, 48, 64, 96, 128, 192, 256) if not quick else (32, 64, 128)):
        if d > n_stages or tw + 4 * d > 256 or th < 2 * d + 2 or (esize == 2 and d % 4):
            continue
        if any(min(d, n_stages - k) % 2 for k in range(0, n_stages, d)):
            continue                                   # every group an even number of stages
        if -(-W // tw) * -(-H // th) < SMS // 2:
            continue                                   # leaves most SMs idle
        out.append(dict(depth=d, tile_w=tw, tile_h=th, threads=256, serial_y=8, impl=hp.HP_IMPL_LINES))
    # the streaming kernel: depth 2 (4 or 8 columns per lane) or 4 (4 columns),
    # rows per run (0: one run per resident warp), threads per block
    for d, cols in ((2, 4), (2, 8), (4, 4)):
        if n_stages % d:
            continue
        for th, t in itertools.product((0, 12, 16, 20, 24, 32) if not quick else (0, 16), (64, 128, 256)):
            out.append(dict(depth=d, tile_w=chain_strip_w(d, cols, esize), tile_h=th, threads=t, serial_y=8,
                            impl=hp.HP_IMPL_WAVE))
    return out


# ----------------------------------------------------------- applications --
def apply_schedule(p, entry):
    """Applies an application schedule (the params of a Harris, unsharp or
    histogram-equalization entry) to p."""
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


def app_candidates(app, dtype="f32"):
    from . import hp
    out = [dict(schedule="root")]
    if app == "histeq":
        return out + [dict(schedule="fused")]
    out.append(dict(schedule="fused", impl=hp.HP_IMPL_GENERIC, tile_w=32, tile_h=32, threads=256))
    tiled_w = (32, 64, 96) if app == "harris" else (64, 128)
    for tw, th, t, sy in itertools.product(tiled_w, (16, 32, 64), (128, 256), (4, 8)):
        out.append(dict(schedule="fused", impl=hp.HP_IMPL_AUTO, tile_w=tw, tile_h=th, threads=t, serial_y=sy))
    runs = (8, 11, 14, 17, 20, 26, 32) if app == "harris" else (12, 16, 20, 24, 32, 48, 64, 96)
    strip = 112 if dtype in ("f16", "bf16") else 120      # 2-byte inputs take 112-column strips
    for th, t in itertools.product(runs, (64, 128, 192, 256)):
        out.append(dict(schedule="fused", impl=hp.HP_IMPL_WAVE, tile_w=strip, tile_h=th, threads=t))
    return out


# --------------------------------------------------------- local Laplacian --
def ll_candidates():
    """The per-level fusion of the local Laplacian (every level's groups as
    local_laplacian_fused_schedule forms them) over: the streaming kernels'
    rows per run and threads; and the tiled downsample / per-pixel level
    kernels in their place."""
    out = []
    for t, rows in itertools.product((128, 256), (0, 1, 2, 4, 8, 16)):
        out.append(dict(threads=t, rows=rows))
    for dt, lt in ((16, 0), (0, 32), (16, 32)):
        out.append(dict(threads=256, rows=0, down_tile=dt, level_tile=lt))
    return out


# ---------------------------------------------------------------- workloads --
# Each workload: how to build its pipeline (with the stage ids a schedule
# needs), its seeded input and output, its candidate space and how a
# candidate is applied.
def workload(pipeline, w, h, dtype):
    """(build, inputs, out_shape, candidates, apply, kind) of a workload."""
    from . import hp, pipelines, synth
    st = {"f32": hp.HP_F32, "f16": hp.HP_F16, "bf16": hp.HP_BF16, "u8": hp.HP_U8, "u16": hp.HP_U16}[dtype]
    if pipeline.startswith("stencil_chain_"):
        _, _, n, pattern = pipeline.split("_")
        n = int(n)
        return dict(kind="chain", build=lambda: (pipelines.stencil_chain(n, pattern, storage=st), None),
                    inputs=lambda: [(synth.stencil_input(h, w, seed=0), st)], out=(1, h, w, st),
                    candidates=lambda quick: chain_candidates(n, w, h, quick, 4 if st == hp.HP_F32 else 2),
                    apply=lambda p, ids, c: pipelines.chain_schedule(p, **c))
    if pipeline in ("harris", "unsharp", "histeq"):
        if pipeline == "harris":
            build = lambda: (pipelines.harris(io_storage=st, inner_storage=st), None)
            img, oc = synth.rgb_f32(h, w, seed=0), 1
        elif pipeline == "unsharp":
            build = lambda: (pipelines.unsharp(storage=st), None)
            img, oc = synth.rgb_f32(h, w, seed=0), 3
        else:
            build = lambda: (pipelines.histeq(), None)
            img, oc = synth.gray_u8_lowcontrast(h, w, seed=0), 1
        return dict(kind="app", build=build, inputs=lambda: [(img, st)], out=(oc, h, w, st),
                    candidates=lambda quick: app_candidates(pipeline, dtype),
                    apply=lambda p, ids, c: apply_schedule(p, c))
    if pipeline.startswith("local_laplacian_"):
        J, K = (int(v[1:]) for v in pipeline.split("_")[2:4])
        return dict(kind="ll", build=lambda: pipelines.local_laplacian(levels=J, k_levels=K),
                    inputs=lambda: [(synth.rgb_u16_gradient_noise(h, w, seed=0), hp.HP_U16)], out=(3, h, w, hp.HP_U16),
                    candidates=lambda quick: ll_candidates(),
                    apply=lambda p, ids, c: pipelines.local_laplacian_fused_schedule(p, ids, **c))
    raise ValueError(pipeline)


def apply_entry(p, ids, pipeline, entry):
    """Applies a stored entry of `pipeline` (as lookup returns it) to p; ids:
    the stage ids of pipelines that need them (the local Laplacian's)."""
    from . import pipelines
    c = entry["params"]
    if pipeline.startswith("stencil_chain_"):
        pipelines.chain_schedule(p, **c)
    elif pipeline.startswith("local_laplacian_"):
        pipelines.local_laplacian_fused_schedule(p, ids, **c)
    else:
        apply_schedule(p, c)


# ------------------------------------------------------------------ timing --
def time_candidate(p, bi, bo, stream, flush, reps=15, probe=False):
    """Median ms of `reps` graph replays (L2 flushed before each: written and
    read back); with probe, also the (kernels, max registers, max local bytes)
    of the launched kernels."""
    import torch
    s = stream.cuda_stream
    if probe:
        p.probe_kernel_attrs(True)
    p.realize(bi, bo, s)   # uncaptured first run
    attrs = p.kernel_attrs() if probe else None
    if probe:
        p.probe_kernel_attrs(False)
    p.realize(bi, bo, s)   # graph capture
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()   # evict the candidate's data from L2, then leave clean lines there
        torch.sum(flush)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.realize(bi, bo, s)
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    ms = statistics.median(x.elapsed_time(y) for x, y in ts)
    return (ms, attrs) if probe else ms


def tune(pipeline, w, h, dtype, quick=False, log=print):
    """Times every candidate of the workload (pruning on hardware limits and
    spills), checks each bit for bit against the stage-per-kernel result, and
    returns the schedules.json entry."""
    import torch
    from . import hp
    wl = workload(pipeline, w, h, dtype)
    to_dev = {hp.HP_F32: torch.float32, hp.HP_F16: torch.float16, hp.HP_BF16: torch.bfloat16, hp.HP_U8: torch.uint8,
              hp.HP_U16: torch.int16}
    bi, keep = [], []
    for arr, dt in wl["inputs"]():
        import numpy as np
        t = torch.from_numpy(np.ascontiguousarray(arr))
        if dt in (hp.HP_F16, hp.HP_BF16):
            t = t.to(to_dev[dt])
        elif dt == hp.HP_U16:
            t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint16).view(np.int16))
        x = hp.padded_copy(t, "cuda")
        keep.append(x)
        bi.append(hp.buffer_from_tensor(x, dt))
    oc, oh, ow, odt = wl["out"]
    ref = hp.padded_empty(oc, oh, ow, to_dev[odt], "cuda")
    y = hp.padded_empty(oc, oh, ow, to_dev[odt], "cuda")
    as_bits = ((lambda t: t.view(torch.int32)) if ref.dtype == torch.float32 else
               (lambda t: t.view(torch.int16)) if ref.element_size() == 2 else (lambda t: t))
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    p, ids = wl["build"]()
    p.use_cuda_graph(True)
    p.realize(bi, hp.buffer_from_tensor(ref, odt), stream.cuda_stream)   # stage-per-kernel (the default)
    torch.cuda.synchronize()
    plain_ms = time_candidate(p, bi, hp.buffer_from_tensor(y, odt), stream, flush)
    log(f"{key(pipeline, w, h, dtype)}: stage-per-kernel {plain_ms:.4f} ms")
    results, pruned = [], []
    for c in wl["candidates"](quick):
        try:
            wl["apply"](p, ids, c)
            ms, attrs = time_candidate(p, bi, hp.buffer_from_tensor(y, odt), stream, flush, probe=True)
        except hp.HPError as e:
            log(f"skip {c}: {e}")
            continue
        if not torch.equal(as_bits(y), as_bits(ref)):
            raise RuntimeError(f"schedule {c} changed the result: schedules must be bit-identical")
        if p.device_error():
            raise RuntimeError(f"schedule {c} reported a device error")
        if attrs[2] > 0:
            pruned.append(dict(params=c, local_bytes=attrs[2], registers=attrs[1]))
            log(f"pruned (spills {attrs[2]} B/thread) {c}")
            continue
        results.append((ms, c, attrs[1]))
        log(f"{ms:.4f} ms {c}")
    results.sort(key=lambda r: r[0])
    best = results[0]
    return dict(workload=dict(pipeline=pipeline, w=w, h=h, dtype=dtype), kind=wl["kind"], params=best[1],
                ms=best[0], plain_ms=plain_ms, registers=best[2], candidates=len(results),
                pruned_spills=len(pruned), top5=[dict(ms=m, registers=r, **c) for m, c, r in results[:5]],
                device=torch.cuda.get_device_name())


# The workloads of the benchmark: the stencil chains (32 stages at 2560x1536 in
# f32, f16 and bf16 storage; 4 binomial stages at 512x512), the applications
# at the five serving sizes (Harris also with bf16 storage), and the local
# Laplacian at 2560x1536.
SERVING_SIZES = [(256, 256), (640, 480), (1920, 1080), (2560, 1536), (4096, 3072)]
BENCH_WORKLOADS = (
    [("stencil_chain_32_alternate", 2560, 1536, d) for d in ("f32", "f16", "bf16")]
    + [("stencil_chain_4_binomial", 512, 512, "f32")]
    + [(a, w, h, "f32") for a in ("harris", "unsharp") for w, h in SERVING_SIZES]
    + [("histeq", w, h, "u8") for w, h in SERVING_SIZES]
    + [("harris", 2560, 1536, "bf16"), ("local_laplacian_J8_K8", 2560, 1536, "u16")])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="all",
                    help="'all' (the benchmark's workloads) or pipeline/WxH/dtype, comma-separated")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out", default=None, help="also write the entries to this JSON file")
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(PKG))
    import __graft_entry__
    __graft_entry__.build()
    todo = BENCH_WORKLOADS if args.workload == "all" else [parse_key(k) for k in args.workload.split(",")]
    entries = {}
    for pipeline, w, h, dtype in todo:
        k = key(pipeline, w, h, dtype)
        entries[k] = tune(pipeline, w, h, dtype, args.quick)
        save(k, entries[k])
    if args.out:
        json.dump(entries, open(args.out, "w"), indent=1)
    print(json.dumps({k: dict(ms=e["ms"], plain_ms=e["plain_ms"], params=e["params"]) for k, e in entries.items()}))


if __name__ == "__main__":
    main()
