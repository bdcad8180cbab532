"""Benchmark: MPix/s of the fused 32-stage stencil chain (2560x1536, f32) on GB300.

One step = one realization of the whole pipeline (every stage of the chain) on
one image already resident in HBM.  The L2 cache (129 MB) is flushed between
timed steps by writing a 256 MiB buffer; each step is timed with CUDA events
on the launching stream.  Also reported on the same line: the stage-per-kernel
schedule of the same pipeline, the end-to-end rate through the C ABI with host
buffers (copies included), the roofline of the dominant kernel, the oracle on
the host cores, and the SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config NAME]

Under torchrun each rank runs an independent replica on its own GPU (the
pipeline has no exchange step); `value` is the whole-job rate.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPix/s fused vs stage-per-kernel on 1 GB300 at stated tol; %HBM roofline; p50/p99"
L2_FLUSH_BYTES = 256 << 20
SMS = 152
FP32_LANES_PER_SM = 128


# ------------------------------------------------------------------ configs --
def config_table():
    from paper_2012_07145_gb300 import hp, pipelines
    return {
        # the headline: 32-stage chain, binomial/box alternating, fused + tuned
        "chain32": dict(workload="stencil_chain_32_alternate_2560x1536_f32", h=1536, w=2560, c=1,
                        build=lambda: pipelines.stencil_chain(32, "alternate"), dtype=hp.HP_F32,
                        fused=lambda p: pipelines.chain_schedule(p, **tuned("chain32")),
                        flops_px=32 * 18, bytes_px=8),
        "chain4": dict(workload="stencil_chain_4_binomial_512x512_f32", h=512, w=512, c=1,
                       build=lambda: pipelines.stencil_chain(4, "binomial"), dtype=hp.HP_F32,
                       fused=lambda p: pipelines.chain_schedule(p, depth=4, tile_w=64, tile_h=32),
                       flops_px=4 * 18, bytes_px=8),
    }


def tuned(name):
    """Schedule parameters chosen by the autotuner (schedules.json), else defaults."""
    path = os.path.join(ROOT, "paper_2012_07145_gb300", "schedules.json")
    if os.path.exists(path):
        db = json.load(open(path))
        if name in db:
            return db[name]["params"]
    return dict(depth=8, tile_w=64, tile_h=32, threads=256, serial_y=8)


# ------------------------------------------------------------------ helpers --
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_chain.cu", "stage_math.cuh", "tma.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2012_07145_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{kernel}:{workload}")
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec["dram_bytes_per_launch"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []      # (wall time, csv line)
        self.t0 = self.t1 = None

    def _reader(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line))

    def start(self):
        """Starts sampling and returns once the first sample has arrived."""
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._reader, daemon=True).start()
        deadline = time.time() + 10
        while not self.lines and time.time() < deadline:
            time.sleep(0.01)

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [l for t, l in self.lines if self.t0 is None or (self.t0 <= t <= self.t1 + 0.1)]
        if not inside:   # region shorter than the sampling period: take the nearest sample after it
            inside = [l for t, l in self.lines if self.t0 is not None and t >= self.t0][:1]
        for line in inside:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm --
def time_steps(p, xin, yout, steps, warmup, flush, stream, dtype, sampler=None):
    import torch
    from paper_2012_07145_gb300 import hp
    bi = [hp.buffer_from_tensor(xin, dtype)]
    bo = hp.buffer_from_tensor(yout, dtype)
    s = stream.cuda_stream
    for _ in range(warmup):
        p.realize(bi, bo, s)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    n0 = hp.launch_count()
    if sampler:
        sampler.mark_begin()
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        p.realize(bi, bo, s)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_end()
    launches = hp.launch_count() - n0
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    return statistics.mean(ms), launches, ms


def run_ours(args, cfg_name):
    import torch
    import torch.distributed as dist
    from paper_2012_07145_gb300 import hp, synth, pipelines
    import __graft_entry__

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()
    cfg = config_table()[cfg_name]
    H, W, C = cfg["h"], cfg["w"], cfg["c"]
    img = synth.stencil_input(H, W, seed=rank)
    stream = torch.cuda.current_stream()
    xin = hp.padded_copy(torch.from_numpy(img), "cuda")
    yout = hp.padded_empty(C, H, W, torch.float32, "cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    if args.only_fused:   # profiling runs: the fused pipeline alone, nothing else on the GPU
        p = cfg["build"]()
        cfg["fused"](p)
        ms, launches, _ = time_steps(p, xin, yout, args.steps, args.warmup, flush, stream, cfg["dtype"])
        if rank == 0:
            print(json.dumps({"only_fused": cfg["workload"], "ms_per_step": ms, "launches": launches}))
        return None
    # stage-per-kernel comparator
    p_plain = cfg["build"]()
    p_plain.use_cuda_graph(True)
    plain_ms, plain_launches, _ = time_steps(p_plain, xin, yout, max(args.steps // 4, 3), args.warmup, flush,
                                             stream, cfg["dtype"])
    # fused, tuned schedule (the headline)
    p = cfg["build"]()
    cfg["fused"](p)
    p.use_cuda_graph(True)
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms, launches, ms_all = time_steps(p, xin, yout, args.steps, args.warmup, flush, stream, cfg["dtype"],
                                      sampler)
    clocks = sampler.stop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the C ABI with pinned host buffers
    hin = torch.from_numpy(img).pin_memory()
    hout = torch.empty((C, H, W), dtype=torch.float32).pin_memory()
    bi = [hp.buffer_from_tensor(hin, cfg["dtype"])]
    bo = hp.buffer_from_tensor(hout, cfg["dtype"])
    for _ in range(3):
        p.realize_host(bi, bo, stream.cuda_stream)
    e2e_steps = max(10, min(args.steps, 200))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        p.realize_host(bi, bo, stream.cuda_stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    out_check = hout.numpy()[0]

    # parity spot check of this run's output against the oracle (a few points)
    from oracle import stencil as ost
    kinds = ost.chain_kinds(len(p.stages), "alternate" if cfg_name == "chain32" else "binomial")
    pts = [(0, 0), (W - 1, H - 1), (W // 3, H // 2)]
    err = max(abs(float(out_check[y, x]) - ost.stencil_chain_point(img[0].astype(np.float64), kinds, x, y))
              for x, y in pts)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    npx = H * W
    peaks, peak_kind = measured_peaks()
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    launches_per_step = launches / args.steps
    kernel_ms = ms / launches_per_step
    flops_launch = cfg["flops_px"] * npx / launches_per_step
    achieved = flops_launch / (kernel_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": round(world * npx / (ms * 1e-3) / 1e6, 2),
        "unit": "MPix/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded uniform [0,1) image; no dataset)",
        "config": {"workload": cfg["workload"], "schedule": tuned(cfg_name) if cfg_name == "chain32" else "fused",
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}",
                   "launch": "CUDA graph replay of the fused launches"},
        "plain": {"value": round(npx / (plain_ms * 1e-3) / 1e6, 2), "unit": "MPix/s", "ms_per_step": round(plain_ms, 5),
                  "launches_per_step": plain_launches / max(args.steps // 4, 3),
                  "schedule": "stage-per-kernel (one launch per stage), CUDA graph replay"},
        "speedup_vs_plain": round(plain_ms / ms, 3),
        "e2e": {"value": round(npx / e2e_s / 1e6, 2), "unit": "MPix/s",
                "h2d_bytes_per_step": int(img.nbytes), "d2h_bytes_per_step": int(img.nbytes)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4),
                     "traffic": recorded_traffic("k_chain", cfg["workload"]),
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz ({peak_kind} clock)",
                     "kernel": "k_chain", "kernel_ms": round(kernel_ms, 5),
                     "hbm_achieved_gbs": round(cfg["bytes_px"] * npx / launches_per_step / (kernel_ms * 1e-3) / 1e9, 1),
                     "hbm_peak_gbs": peaks.get("hbm_gbs")},
        "clocks": clocks,
        "parity_spot_max_abs_err": err,
        "step_ms_p50": round(statistics.median(ms_all), 5),
        "step_ms_p99": round(float(np.percentile(ms_all, 99)), 5),
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg_name, seconds=args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    return line


# ------------------------------------------------------------- oracle (CPU) --
def cpu_baseline(cfg_name, seconds=15.0, rows=None):
    """The FP64 oracle, as it stands, on a bounded band of the same workload."""
    from oracle import stencil as ost
    from paper_2012_07145_gb300 import synth
    cfg = config_table()[cfg_name]
    W = cfg["w"]
    rows = rows or min(cfg["h"], 256)
    img = synth.stencil_input(rows, W, seed=0)[0].astype(np.float64)
    kinds = ost.chain_kinds(32 if cfg_name == "chain32" else 4, "alternate" if cfg_name == "chain32" else "binomial")
    t0 = time.perf_counter()
    n = 0
    while True:
        ost.stencil_chain(img, kinds)
        n += 1
        if time.perf_counter() - t0 >= seconds * 0.5:
            break
    dt = (time.perf_counter() - t0) / n
    return {"value": round(rows * W / dt / 1e6, 4), "unit": "MPix/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} run(s) of the FP64 oracle on a {W}x{rows} band (same per-pixel work), numpy, 1 thread"}


def run_reference(args, cfg_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cfg = config_table()[cfg_name]
    from oracle import stencil as ost
    from paper_2012_07145_gb300 import synth
    W = cfg["w"]
    kinds = ost.chain_kinds(32 if cfg_name == "chain32" else 4, "alternate" if cfg_name == "chain32" else "binomial")
    # size each step's band so that all steps together take about two minutes
    probe = synth.stencil_input(8, W, seed=0)[0].astype(np.float64)
    t0 = time.perf_counter()
    ost.stencil_chain(probe, kinds)
    per_row = (time.perf_counter() - t0) / 8
    rows = int(max(1, min(cfg["h"], 120.0 / max(args.steps, 1) / per_row)))
    img = synth.stencil_input(rows, W, seed=0)[0].astype(np.float64)
    for _ in range(min(args.warmup, 1)):
        ost.stencil_chain(img, kinds)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ost.stencil_chain(img, kinds)
    dt = (time.perf_counter() - t0) / args.steps
    v = round(rows * W / dt / 1e6, 4)
    return {"metric": METRIC, "value": v, "unit": "MPix/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": cfg["workload"], "sample": f"{W}x{rows} band per step"},
            "cpu_baseline": {"value": v, "unit": "MPix/s", "cores": 1, "kind": "oracle",
                             "sample": f"FP64 oracle on a {W}x{rows} band per step, numpy, 1 thread"},
            "e2e": {"value": v, "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="chain32")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--only-fused", action="store_true",
                    help="time the fused pipeline only (for profiler runs); prints no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    line = run_reference(args, args.config) if args.impl == "reference" else run_ours(args, args.config)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
