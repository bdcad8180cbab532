"""Benchmark: MPix/s of the fused 32-stage stencil chain (2560x1536, f32) on GB300.

One step = one realization of the whole pipeline (every stage of the chain) on
one image already resident in HBM.  The L2 cache (129 MB) is flushed between
timed steps by writing a 256 MiB buffer and reading it back, so a timed step
finds none of its data in L2 and no dirty lines of the flush to write back;
each step is timed with CUDA events on the launching stream.  Also reported on the same line: the stage-per-kernel
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
FP32_LANES_PER_SM = 128
# the workloads the default line also reports, compactly, beside the headline
DEFAULT_CONFIGS = "chain4,chain32_f16,chain32_bf16,harris,harris_bf16,unsharp,histeq,ll,serving"


# ------------------------------------------------------------------ configs --
def _chain_cfg(name, n, pattern, H, W, storage_name="f32"):
    from paper_2012_07145_gb300 import hp, pipelines, synth
    st = {"f32": hp.HP_F32, "f16": hp.HP_F16, "bf16": hp.HP_BF16}[storage_name]
    esize = 4 if storage_name == "f32" else 2
    tkey = (f"stencil_chain_{n}_{pattern}", W, H, storage_name)

    def fused(p):
        apply_tuned(p, None, tkey, lambda q: pipelines.chain_schedule(q, depth=8, tile_w=64, tile_h=32))

    def oracle_sample(rows):
        from oracle import stencil as ost
        img = synth.stencil_input(rows, W, seed=0)[0].astype(np.float64)
        return lambda: ost.stencil_chain(img, ost.chain_kinds(n, pattern))

    def parity(out, inputs):
        from oracle import stencil as ost
        img = inputs[0][0][0].astype(np.float64)
        pts = [(0, 0), (W - 1, H - 1), (W // 3, H // 2)]
        ref = [ost.stencil_chain_point(img, ost.chain_kinds(n, pattern), x, y) for x, y in pts]
        return max(abs(float(out[0][y, x]) - r) for (x, y), r in zip(pts, ref))

    def lowp_error(out, inputs):
        """The 16-bit storage error against the FP64 oracle on the top band of
        the image (rows whose whole dependency cone lies in the band): the
        oracle fed the rounded input, and the original input."""
        import torch
        from oracle import stencil as ost
        band, keep = 4 * n + 64, 64
        img = inputs[0][0][0][:band].astype(np.float64)
        rounded = torch.from_numpy(inputs[0][0][0][:band].astype(np.float32)).to(
            torch.float16 if storage_name == "f16" else torch.bfloat16).double().numpy()
        kinds = ost.chain_kinds(n, pattern)
        got = out[0][:keep].astype(np.float64)
        errs = []
        for src in (rounded, img):
            ref = ost.stencil_chain(src, kinds)[:keep]
            errs.append(float(np.abs(got - ref).max() / (ref.max() - ref.min())))
        return {"rounded_input": errs[0], "original_input": errs[1],
                "measure": f"max |gpu - oracle| / range over rows 0..{keep - 1} (oracle on rows 0..{band - 1})"}

    # the method's work per output pixel (a separable 5x5 stage, per pass):
    # binomial ((a+e) + 4(b+d)) + 6c, then x 1/16: 7 flops (an fma counts 2);
    # box (((a+b) + (c+d)) + e) x 1/5: 5 flops
    n_binomial = sum(1 for k in range(n) if pattern == "binomial" or k % 2 == 0)
    flops_px = 14 * n_binomial + 10 * (n - n_binomial)
    algorithmic = (f"{flops_px} FP32 flops per output pixel: {n_binomial} binomial stages x 14 + "
                   f"{n - n_binomial} box stages x 10 (2 separable passes each, fma = 2 flops)")
    return dict(workload=f"stencil_chain_{n}_{pattern}_{W}x{H}_{storage_name}", h=H, w=W,
                inputs=lambda seed: [(synth.stencil_input(H, W, seed=seed), st)], out=(1, H, W, st),
                build=lambda: pipelines.stencil_chain(n, pattern, storage=st), fused=fused,
                tuned_key=tkey, flops_px=flops_px, algorithmic=algorithmic, fp32_instr_px=10 * n,
                bytes_px=2 * esize, bound="alu", kernel="k_chain", dtype=storage_name,
                oracle_sample=oracle_sample, parity=parity, sample_rows=64,
                lowp_error=lowp_error if storage_name != "f32" else None)


def config_table():
    from paper_2012_07145_gb300 import hp, pipelines, synth
    cfgs = {
        # the headline: 32-stage chain, binomial/box alternating, fused + tuned
        "chain32": _chain_cfg("chain32", 32, "alternate", 1536, 2560),
        "chain32_f16": _chain_cfg("chain32", 32, "alternate", 1536, 2560, "f16"),
        "chain32_bf16": _chain_cfg("chain32", 32, "alternate", 1536, 2560, "bf16"),
        "chain4": _chain_cfg("chain4", 4, "binomial", 512, 512),
    }
    # the same 32-stage chain on the streaming kernel (4 stages in registers per warp strip)
    wave = _chain_cfg("chain32", 32, "alternate", 1536, 2560)
    wave["workload"] += "_streaming"
    wave["kernel"] = "k_chain_rows"
    wave["fused"] = lambda p: pipelines.chain_schedule(p, depth=2, tile_w=120, tile_h=0, threads=256,
                                                       impl=hp.HP_IMPL_WAVE)
    wave["tuned_key"] = None
    cfgs["chain32_wave"] = wave
    H, W = 1536, 2560

    def harris_parity(out, inputs):
        from oracle import harris as ohr
        rgb = inputs[0][0][:, :64, :64].astype(np.float64)
        ref = ohr.harris(rgb)[:62, :62]          # rows/cols away from the band's cut edge
        return float(np.abs(out[0][:62, :62] - ref).max() / (ref.max() - ref.min()))

    def harris_sample(rows):
        from oracle import harris as ohr
        rgb = synth.rgb_f32(rows, W, seed=0).astype(np.float64)
        return lambda: ohr.harris(rgb)

    cfgs["harris"] = dict(workload=f"harris_rgb_{W}x{H}_f32", h=H, w=W,
                          inputs=lambda seed: [(synth.rgb_f32(H, W, seed=seed), hp.HP_F32)], out=(1, H, W, hp.HP_F32),
                          build=lambda: pipelines.harris(),
                          fused=app_schedule("harris", W, H, "f32", dict(schedule="fused", impl=hp.HP_IMPL_WAVE,
                                                                         tile_w=120, tile_h=14, threads=256)),
                          tuned_key=("harris", W, H, "f32"),
                          flops_px=68, bytes_px=16, bound="hbm", kernel="k_harris_rows", dtype="f32",
                          oracle_sample=harris_sample, parity=harris_parity, sample_rows=128)
    def harris_bf16_parity(out, inputs):
        import torch
        from oracle import harris as ohr
        # the oracle on the bf16-rounded input (the storage error of the stages is what is stated)
        rgb = torch.from_numpy(inputs[0][0][:, :64, :64]).to(torch.bfloat16).double().numpy()
        ref = ohr.harris(rgb)[:62, :62]
        return float(np.abs(out[0][:62, :62] - ref).max() / (ref.max() - ref.min()))

    def harris_bf16_error(out, inputs):
        import torch
        from oracle import harris as ohr
        band = inputs[0][0][:, :96, :]
        rounded = torch.from_numpy(band).to(torch.bfloat16).double().numpy()
        got = out[0][:92].astype(np.float64)
        errs = []
        for src in (rounded, band.astype(np.float64)):
            ref = ohr.harris(src)[:92]
            errs.append(float(np.abs(got - ref).max() / (ref.max() - ref.min())))
        return {"rounded_input": errs[0], "original_input": errs[1],
                "measure": "max |gpu - oracle| / range over rows 0..91 (oracle on rows 0..95)"}

    cfgs["harris_bf16"] = dict(workload=f"harris_rgb_{W}x{H}_bf16", h=H, w=W,
                               inputs=lambda seed: [(synth.rgb_f32(H, W, seed=seed), hp.HP_BF16)],
                               out=(1, H, W, hp.HP_BF16),
                               build=lambda: pipelines.harris(io_storage=hp.HP_BF16, inner_storage=hp.HP_BF16),
                               fused=app_schedule("harris", W, H, "bf16", dict(schedule="fused", impl=hp.HP_IMPL_WAVE,
                                                                               tile_w=112, tile_h=14, threads=128)),
                               tuned_key=("harris", W, H, "bf16"),
                               flops_px=68, bytes_px=8, bound="hbm", kernel="k_harris_rows", dtype="bf16",
                               oracle_sample=harris_sample, parity=harris_bf16_parity, sample_rows=128,
                               lowp_error=harris_bf16_error)
    UH, UW = 3072, 4096

    def unsharp_sample(rows):
        from oracle import unsharp as ous
        img = synth.rgb_f32(rows, UW, seed=0).astype(np.float64)
        return lambda: ous.unsharp(img)

    def unsharp_parity(out, inputs):
        from oracle import unsharp as ous
        img = inputs[0][0][:, :64, :64].astype(np.float64)
        ref = ous.unsharp(img)[:, :60, :60]
        return float(np.abs(out[:, :60, :60] - ref).max() / (ref.max() - ref.min()))

    cfgs["unsharp"] = dict(workload=f"unsharp_rgb_{UW}x{UH}_f32", h=UH, w=UW,
                           inputs=lambda seed: [(synth.rgb_f32(UH, UW, seed=seed), hp.HP_F32)],
                           out=(3, UH, UW, hp.HP_F32), build=lambda: pipelines.unsharp(),
                           fused=app_schedule("unsharp", UW, UH, "f32", dict(schedule="fused", impl=hp.HP_IMPL_WAVE,
                                                                             tile_w=120, tile_h=16, threads=128)),
                           tuned_key=("unsharp", UW, UH, "f32"),
                           flops_px=63, bytes_px=24, bound="hbm", kernel="k_stencil_rows", dtype="f32",
                           oracle_sample=unsharp_sample, parity=unsharp_parity, sample_rows=96)

    def histeq_sample(rows):
        from oracle import histeq as ohe
        img = synth.gray_u8_lowcontrast(rows, UW, seed=0)[0]
        return lambda: ohe.equalize(img)

    def histeq_parity(out, inputs):
        from oracle import histeq as ohe
        ref = ohe.equalize(inputs[0][0][0])[2]
        return int((out[0] != ref).sum())

    cfgs["histeq"] = dict(workload=f"histeq_u8_{UW}x{UH}", h=UH, w=UW,
                          inputs=lambda seed: [(synth.gray_u8_lowcontrast(UH, UW, seed=seed), hp.HP_U8)],
                          out=(1, UH, UW, hp.HP_U8), build=lambda: pipelines.histeq(),
                          fused=app_schedule("histeq", UW, UH, "u8", dict(schedule="fused")),
                          tuned_key=("histeq", UW, UH, "u8"),
                          flops_px=0, bytes_px=2, bound="hbm", kernel="k_histeq", dtype="u8",
                          oracle_sample=histeq_sample, parity=histeq_parity, sample_rows=256)

    def ll_build():
        return pipelines.local_laplacian(levels=8, k_levels=8)[0]

    def ll_fused(p):
        pl, ids = pipelines.local_laplacian(levels=8, k_levels=8)      # the stage ids of p's identical build
        apply_tuned(p, ids, ("local_laplacian_J8_K8", W, H, "u16"),
                    lambda q: pipelines.local_laplacian_fused_schedule(q, ids))

    def ll_sample(rows):
        from oracle import local_laplacian as oll
        img = synth.rgb_u16_gradient_noise(rows, W, seed=0)
        return lambda: oll.local_laplacian(img, levels=8, k_levels=8)

    def ll_parity(out, inputs):
        return int(np.abs(out.astype(np.int64) - inputs[0][0].astype(np.int64)).max())   # identity parameters

    # The dominant kernel (largest share of the ncu launch list): level 1 of the
    # remap pyramid straight from the input, timed alone on the same input.
    # Algorithmic FP32 flops per fine pixel (FMA = 2): gray 8; the remap outside
    # the band for 8 levels 8 x 5 = 40; the full remap for the two levels of the
    # band 2 x 8 = 16; downsample x pass 9 channels x 9 flops at every second
    # column 40.5; y pass 9 x 9 at every fourth pixel 20.25.  Total 124.75.
    ll_dominant = dict(kernel="k_ll_remap_rows", flops_per_launch=124.75 * W * H,
                       algorithmic="124.75 FP32 flops per fine pixel (gray 8, remap 8 levels outside the band 40, "
                                   "2 levels in the band 16, 9-channel downsample x pass 40.5 and y pass 20.25)",
                       build=lambda: pipelines.remap_pyramid_level1(), out=(9, (H + 1) // 2, (W + 1) // 2, hp.HP_F32))
    cfgs["ll"] = dict(workload=f"local_laplacian_rgb_u16_{W}x{H}_J8_K8", h=H, w=W,
                      inputs=lambda seed: [(synth.rgb_u16_gradient_noise(H, W, seed=seed), hp.HP_U16)],
                      out=(3, H, W, hp.HP_U16), build=ll_build, fused=ll_fused,
                      tuned_key=("local_laplacian_J8_K8", W, H, "u16"),
                      flops_px=0, bytes_px=12, bound="alu", kernel="k_ll_remap_rows", dtype="u16",
                      dominant=ll_dominant, oracle_sample=ll_sample, parity=ll_parity, sample_rows=128)
    def maxfilter_sample(rows):
        from oracle import maxfilter as om
        img = synth.rgb_f32(rows, W, seed=0)
        return lambda: om.max_filter_planes(img, 4, 4)

    def maxfilter_parity(out, inputs):
        from oracle import maxfilter as om
        ref = om.max_filter_planes(inputs[0][0][:, :64, :64], 4, 4)[:, :60, :60]
        return int((out[:, :60, :60] != ref).sum())      # exact: mismatching values in the sampled corner

    cfgs["maxfilter"] = dict(workload=f"max_filter_rgb_{W}x{H}_9x9_f32", h=H, w=W,
                             inputs=lambda seed: [(synth.rgb_f32(H, W, seed=seed), hp.HP_F32)],
                             out=(3, H, W, hp.HP_F32), build=lambda: pipelines.max_filter(4),
                             fused=lambda p: p.schedule([0, 0]),
                             flops_px=0, bytes_px=24, bound="hbm", kernel="k_max_rows", dtype="f32",
                             oracle_sample=maxfilter_sample, parity=maxfilter_parity, sample_rows=64)

    def interp_build():
        return pipelines.interpolate(10)[0]

    def interp_fused(p):
        _, ids = pipelines.interpolate(10)
        pipelines.interpolate_fused_schedule(p, ids)

    def interp_sample(rows):
        from oracle import interpolate as oi
        img = synth.rgba_sparse_f32(rows, W, seed=0).astype(np.float64)
        return lambda: oi.interpolate(img, 10)

    def interp_parity(out, inputs):
        img = inputs[0][0]
        cov = img[3] > 0                                   # covered pixels keep their colour exactly
        return int((out[:, cov] != img[:3][:, cov]).sum())

    # dominant kernel: the finest group (premultiply, upsample of I_1, composite,
    # division by coverage) timed alone; algorithmic bytes per fine pixel: the
    # RGBA input 16, I_1 at a quarter of the pixels 4, the RGB output 12
    def premultiplied(seed):
        x = synth.rgba_sparse_f32(H, W, seed=seed)
        return np.concatenate([x[:3] * x[3:4], x[3:4]]).astype(np.float32)

    interp_dominant = dict(kernel="k_interp_rows", bound="hbm", bytes_per_launch=32 * W * H,
                           algorithmic="32 bytes per fine pixel (premultiplied RGBA level 0 16, the 4-channel level 1 "
                                       "at a quarter of the pixels 4, RGB output 12)",
                           build=lambda: pipelines.interpolate_finest(),
                           inputs=lambda seed: [(premultiplied(seed), hp.HP_F32),
                                                (synth.uniform_f32((4, (H + 1) // 2, (W + 1) // 2), seed, stream=8),
                                                 hp.HP_F32)],
                           out=(3, H, W, hp.HP_F32))
    def bg_sample(rows):
        from oracle import bilateral_grid as ob
        img = synth.gray_f32_gradient_noise(rows, W, seed=0)[0]
        return lambda: ob.bilateral_grid(img, 8, 0.1)

    def bg_parity(out, inputs):
        from oracle import bilateral_grid as ob
        ref = ob.bilateral_grid(inputs[0][0][0][:96], 8, 0.1)[:64]   # rows whose grid cells lie inside the band
        return float(np.abs(out[0][:64].astype(np.float64) - ref).max())

    def bg_grid(seed):
        # a blurred-grid-like input for the slice alone: values in [0, w], weights in [1, 64]
        gx, gy = (W + 7) // 8 + 1, (H + 7) // 8 + 1
        wts = 1.0 + 63.0 * synth.uniform_f32((11, gy, gx), seed, stream=10)
        vals = wts * synth.uniform_f32((11, gy, gx), seed, stream=11)
        return np.stack([vals, wts], axis=1).reshape(22, gy, gx).astype(np.float32)

    bg_dominant = dict(kernel="k_grid_slice", bound="hbm", bytes_per_launch=8 * W * H + 22 * 4 * ((W + 7) // 8 + 1) * ((H + 7) // 8 + 1),
                       algorithmic="8 bytes per pixel (the image read, the output written) plus the grid "
                                   "(22 channels x 321 x 193 cells x 4 bytes) read once",
                       build=lambda: pipelines.bilateral_grid_slice_only(8, 0.1),
                       inputs=lambda seed: [(bg_grid(seed), hp.HP_F32),
                                            (synth.gray_f32_gradient_noise(H, W, seed=seed), hp.HP_F32)],
                       out=(1, H, W, hp.HP_F32))
    cfgs["bilateral"] = dict(workload=f"bilateral_grid_gray_{W}x{H}_s8_r0.1_f32", h=H, w=W,
                             inputs=lambda seed: [(synth.gray_f32_gradient_noise(H, W, seed=seed), hp.HP_F32)],
                             out=(1, H, W, hp.HP_F32), build=lambda: pipelines.bilateral_grid(8, 0.1),
                             fused=lambda p: pipelines.bilateral_grid_fused_schedule(p),
                             flops_px=0, bytes_px=8, bound="hbm", kernel="k_grid_slice", dtype="f32",
                             dominant=bg_dominant, oracle_sample=bg_sample, parity=bg_parity, sample_rows=64)

    cfgs["interpolate"] = dict(workload=f"interpolate_rgba_{W}x{H}_J10_f32", h=H, w=W,
                               inputs=lambda seed: [(synth.rgba_sparse_f32(H, W, seed=seed), hp.HP_F32)],
                               out=(3, H, W, hp.HP_F32), build=interp_build, fused=interp_fused,
                               flops_px=0, bytes_px=28, bound="hbm", kernel="k_interp_rows", dtype="f32",
                               dominant=interp_dominant, oracle_sample=interp_sample, parity=interp_parity,
                               sample_rows=64)
    return cfgs


def apply_tuned(p, ids, tkey, default):
    """Applies the autotuner's stored schedule of a workload (schedules.json,
    keyed by pipeline, size and storage type), else the default schedule."""
    from paper_2012_07145_gb300 import tuner
    entry = tuner.lookup(*tkey)
    if entry is None:
        default(p)
    else:
        tuner.apply_entry(p, ids, tkey[0], entry)


def app_schedule(app, w, h, dtype, default):
    """A function applying the tuned schedule of an application at w x h and
    this storage type, else the given default schedule."""
    from paper_2012_07145_gb300 import tuner
    return lambda p: apply_tuned(p, None, (app, w, h, dtype), lambda q: tuner.apply_schedule(q, default))


def schedule_of(cfg_name, cfg):
    """The schedule a bench line ran, for its config record."""
    from paper_2012_07145_gb300 import tuner
    tkey = cfg.get("tuned_key")
    entry = tuner.lookup(*tkey) if tkey else None
    if entry is None:
        return "default (see pipelines.py)"
    return dict(entry["params"], source=f"schedules.json {tuner.key(*tkey)} (tuner.py)")


# ------------------------------------------------------------------ helpers --
def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2012_07145_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel (the files the record lists); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{kernel}:{workload}")
    if not rec or rec.get("source_hash") != kernel_source_hash(rec.get("sources", [])):
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
def flush_l2(flush):
    """Evicts the previous step's data from L2: writes the 256 MiB buffer, then
    reads it back so that the lines left in L2 are clean (the timed kernels do
    not pay the write-back of the flush itself)."""
    import torch
    flush.zero_()
    torch.sum(flush)


def time_steps(p, bi, bo, steps, warmup, flush, stream, sampler=None):
    import torch
    from paper_2012_07145_gb300 import hp
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
        flush_l2(flush)
        starts[i].record(stream)
        p.realize(bi, bo, s)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_end()
    launches = hp.launch_count() - n0
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    return statistics.mean(ms), launches, ms


def _torch_dtype(dt):
    import torch
    from paper_2012_07145_gb300 import hp
    return {hp.HP_F32: torch.float32, hp.HP_F16: torch.float16, hp.HP_BF16: torch.bfloat16,
            hp.HP_U8: torch.uint8, hp.HP_U16: torch.int16}[dt]


def _host_tensor(arr, dt):
    """Pinned host tensor of a numpy image in the hp dtype's element type."""
    import torch
    from paper_2012_07145_gb300 import hp
    if dt in (hp.HP_F16, hp.HP_BF16):
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).to(_torch_dtype(dt))
    elif dt == hp.HP_U16:
        t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint16).view(np.int16))
    else:
        t = torch.from_numpy(np.ascontiguousarray(arr))
    return t.pin_memory()


def _to_numpy(t, dt):
    from paper_2012_07145_gb300 import hp
    if dt in (hp.HP_F16, hp.HP_BF16):
        return t.float().cpu().numpy()
    if dt == hp.HP_U16:
        return t.cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def measure_fp32_peak(device_index):
    """FP32 peak of this GPU, measured (hp_measure_fp32_peak): scalar fma and
    paired fma.rn.f32x2 kernels on every SM, each timed with CUDA events over
    about 0.3 s while nvidia-smi samples the SM clock.  The peak is the faster
    form; flops per MHz normalise it to the clock it ran at."""
    import torch
    from paper_2012_07145_gb300 import hp
    s = torch.cuda.current_stream().cuda_stream
    out = {}
    for paired in (False, True):
        f, ms, sms = hp.measure_fp32_peak(paired, iters=512, launches=4, stream=s)      # size the run
        launches = max(10, int(300.0 / max(ms, 1e-3)))
        sampler = ClockSampler(device_index)
        sampler.start()
        sampler.mark_begin()
        f, ms, sms = hp.measure_fp32_peak(paired, iters=512, launches=launches, stream=s)
        sampler.mark_end()
        clk = sampler.stop()
        out["paired" if paired else "scalar"] = {"tflops": round(f / 1e12, 3), "ms_per_launch": round(ms, 4),
                                                 "launches": launches, "sm_mhz": clk["sm_mhz"],
                                                 "reasons": clk["reasons"]}
        out["sms"] = sms
    best = max(("scalar", "paired"), key=lambda k: out[k]["tflops"])
    out["peak_tflops"] = out[best]["tflops"]
    out["peak_form"] = best
    mhz = out[best]["sm_mhz"]
    out["tflops_per_ghz"] = round(out[best]["tflops"] / (mhz / 1e3), 3) if mhz else None
    out["nominal_tflops_at_2070_mhz"] = round(out["sms"] * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12, 2)
    return out


def measure_config(cfg_name, cfg, steps, warmup, flush, stream, peaks, peak_kind, fp32, local=0, world=1,
                   headline=False):
    """Times one workload: the stage-per-kernel comparator, the fused tuned
    schedule (with clocks sampled during its timed region), the roofline of
    its dominant kernel and a parity spot check.  Returns the measurements
    and the objects the end-to-end timing needs."""
    import torch
    from paper_2012_07145_gb300 import hp
    H, W = cfg["h"], cfg["w"]
    C, OH, OW, odt = cfg["out"]
    rank = int(os.environ.get("RANK", "0"))
    inputs = cfg["inputs"](rank)
    dev_in = [hp.padded_copy(_host_tensor(a, dt), "cuda") for a, dt in inputs]
    yout = hp.padded_empty(C, OH, OW, _torch_dtype(odt), "cuda")
    bi = [hp.buffer_from_tensor(t, dt) for t, (_, dt) in zip(dev_in, inputs)]
    bo = hp.buffer_from_tensor(yout, odt)
    # stage-per-kernel comparator
    p_plain = cfg["build"]()
    p_plain.use_cuda_graph(True)
    plain_steps = max(steps // 4, 3)
    plain_ms, plain_launches, _ = time_steps(p_plain, bi, bo, plain_steps, warmup, flush, stream)
    # fused, tuned schedule
    p = cfg["build"]()
    cfg["fused"](p)
    p.use_cuda_graph(True)
    sampler = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms, launches, ms_all = time_steps(p, bi, bo, steps, warmup, flush, stream, sampler)
    clocks = sampler.stop()
    torch.cuda.synchronize()
    assert p.device_error() == 0, "a kernel reported a device-side error"
    out_np = _to_numpy(yout, odt)
    err = cfg["parity"](out_np, inputs)
    lowp = cfg["lowp_error"](out_np, inputs) if cfg.get("lowp_error") else None

    npx = OH * OW
    fp32_peak = fp32["peak_tflops"]
    fp32_src = (f"measured: hp_measure_fp32_peak, {fp32['peak_form']} fma on {fp32['sms']} SMs at "
                f"{fp32[fp32['peak_form']]['sm_mhz']} MHz median")
    launches_per_step = launches / steps
    kernel_ms = ms / launches_per_step
    if "dominant" in cfg:
        # a multi-kernel step: its dominant kernel timed alone, on the same
        # input, with the same L2 flush between launches
        dom = cfg["dominant"]
        dp = dom["build"]()
        dc, dh, dw, ddt = dom["out"]
        dout = hp.padded_empty(dc, dh, dw, _torch_dtype(ddt), "cuda")
        dbi = bi
        if "inputs" in dom:
            dins = dom["inputs"](0)
            dtens = [hp.padded_copy(_host_tensor(a, dt), "cuda") for a, dt in dins]
            dbi = [hp.buffer_from_tensor(t, dt) for t, (_, dt) in zip(dtens, dins)]
        dms, dlaunches, _ = time_steps(dp, dbi, hp.buffer_from_tensor(dout, ddt), steps, warmup, flush, stream)
        if dom.get("bound", "alu") == "hbm":
            achieved = dom["bytes_per_launch"] / (dms * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                    "frac": round(achieved / peaks.get("hbm_gbs", 6800.0), 4),
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
        else:
            achieved = dom["flops_per_launch"] / (dms * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": round(achieved / fp32_peak, 4), "peak_source": fp32_src}
        roof.update({"algorithmic": dom["algorithmic"], "timed": "the dominant group alone, one launch per step",
                     "launches_per_timed_step": dlaunches / steps})
        kernel_ms = dms
    elif cfg["bound"] == "alu":
        achieved = cfg["flops_px"] * npx / launches_per_step / (kernel_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4), "peak_source": fp32_src,
                "algorithmic": cfg["algorithmic"]}
        if cfg.get("fp32_instr_px"):
            # FP32 instructions the fixed per-stage expression issues (tap5: 1 mul
            # + 4 fma per pass, 2 passes), against one FP32 instruction per lane
            # and clock on every SM at the clock sampled during the timed region
            mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
            issue = cfg["fp32_instr_px"] * npx / launches_per_step / (kernel_ms * 1e-3)
            roof["fp32_issue_frac"] = round(issue / (fp32["sms"] * FP32_LANES_PER_SM * mhz * 1e6), 4)
            roof["fp32_issue_basis"] = (f"{cfg['fp32_instr_px']} FP32 instructions per output pixel "
                                        f"(10 per stage: 2 passes x (1 mul + 4 fma)) vs {fp32['sms']} SMs x "
                                        f"{FP32_LANES_PER_SM} lanes x {mhz} MHz")
    else:
        achieved = cfg["bytes_px"] * npx / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": round(achieved / peaks.get("hbm_gbs", 6800.0), 4),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "algorithmic": f"{cfg['bytes_px']} bytes per output pixel (input + output once), over the whole step"}
    roof.update({"traffic": recorded_traffic(cfg["kernel"], cfg["workload"]), "kernel": cfg["kernel"],
                 "kernel_ms": round(kernel_ms, 5), "launches_per_step": launches_per_step})
    if roof["bound"] == "hbm":   # also against the nominal HBM3e bandwidth, for context
        roof["frac_of_nominal_7900_gbs"] = round(roof["achieved"] / 7900.0, 4)
    res = dict(npx=npx, ms=ms, ms_all=ms_all, launches=launches, plain_ms=plain_ms, plain_launches=plain_launches,
               plain_steps=plain_steps, roof=roof, clocks=clocks, err=err, p=p, inputs=inputs, lowp=lowp)
    return res


def compact_entry(cfg_name, cfg, r):
    return {"workload": cfg["workload"], "value": round(r["npx"] / (r["ms"] * 1e-3) / 1e6, 2), "unit": "MPix/s",
            "ms_per_step": round(r["ms"], 5), "plain": round(r["npx"] / (r["plain_ms"] * 1e-3) / 1e6, 2),
            "speedup_vs_plain": round(r["plain_ms"] / r["ms"], 3), "bound": r["roof"]["bound"],
            "frac": r["roof"]["frac"], "kernel": r["roof"]["kernel"], "kernel_ms": r["roof"]["kernel_ms"],
            "launches_per_step": r["launches"] / max(1, len(r["ms_all"])),
            "clocks": {k: r["clocks"].get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "parity": r["err"], "parity_kind": cfg.get("parity_kind", "max |gpu - oracle| at sampled points"),
            "schedule": schedule_of(cfg_name, cfg),
            **({"error_vs_fp64": r["lowp"]} if r.get("lowp") else {})}


def run_ours(args, cfg_name):
    import torch
    import torch.distributed as dist
    from paper_2012_07145_gb300 import hp
    import __graft_entry__

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()
    table = config_table()
    cfg = table[cfg_name]
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    if args.only_fused:   # profiling runs: the fused pipeline alone, nothing else on the GPU
        inputs = cfg["inputs"](rank)
        C, OH, OW, odt = cfg["out"]
        dev_in = [hp.padded_copy(_host_tensor(a, dt), "cuda") for a, dt in inputs]
        yout = hp.padded_empty(C, OH, OW, _torch_dtype(odt), "cuda")
        bi = [hp.buffer_from_tensor(t, dt) for t, (_, dt) in zip(dev_in, inputs)]
        p = cfg["build"]()
        cfg["fused"](p)
        ms, launches, _ = time_steps(p, bi, hp.buffer_from_tensor(yout, odt), args.steps, args.warmup, flush, stream)
        if rank == 0:
            print(json.dumps({"only_fused": cfg["workload"], "ms_per_step": ms, "launches": launches}))
        return None
    peaks, peak_kind = measured_peaks()
    fp32 = measure_fp32_peak(local)
    r = measure_config(cfg_name, cfg, args.steps, args.warmup, flush, stream, peaks, peak_kind, fp32, local, world,
                       headline=True)
    ms = r["ms"]
    if world > 1:
        from paper_2012_07145_gb300 import replicas
        dist.barrier()
        ms = replicas.max_over_ranks(ms, device="cuda")   # the slowest replica bounds the job

    # end to end through the C ABI with pinned host buffers: every step copies
    # its image in and its result out.  A stream of images through
    # hp_realize_host_async (the copies of one image overlap the realize of
    # the next; one wait at the end), and one image per synchronous
    # hp_realize_host call
    p, inputs = r["p"], r["inputs"]
    C, OH, OW, odt = cfg["out"]
    hin = [_host_tensor(a, dt) for a, dt in inputs]
    hout = torch.empty((C, OH, OW), dtype=_torch_dtype(odt)).pin_memory()
    hbi = [hp.buffer_from_tensor(t, dt) for t, (_, dt) in zip(hin, inputs)]
    hbo = hp.buffer_from_tensor(hout, odt)
    e2e_steps = max(10, min(args.steps, 200))
    for _ in range(3):
        p.realize_host_async(hbi, hbo, stream.cuda_stream)
    p.realize_host_wait()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        p.realize_host_async(hbi, hbo, stream.cuda_stream)
    p.realize_host_wait()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    err_e2e = cfg["parity"](_to_numpy(hout, odt), inputs)
    for _ in range(3):
        p.realize_host(hbi, hbo, stream.cuda_stream)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        p.realize_host(hbi, hbo, stream.cuda_stream)
    e2e_sync_s = (time.perf_counter() - t0) / e2e_steps

    # the other workloads, compactly, on the same GPU (rank 0's replica only)
    others = {}
    if args.configs and rank == 0 and world == 1:
        for name in [n for n in args.configs.split(",") if n and n != cfg_name]:
            if name == "serving":
                others[name] = serving_compact(rate=1000.0, requests=200)
                continue
            oc = table[name]
            torch.cuda.synchronize()
            others[name] = compact_entry(name, oc, measure_config(name, oc, args.steps, args.warmup, flush, stream,
                                                                  peaks, peak_kind, fp32, local))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    npx = r["npx"]
    in_bytes = int(sum(a.nbytes for a, _ in inputs))
    out_bytes = int(C * OH * OW * hp.DTYPE_BYTES[odt])
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
        "dtype": cfg["dtype"],
        "data": "synthetic (seeded images with the workload's shape and value distribution; no dataset)",
        "config": {"workload": cfg["workload"],
                   "schedule": schedule_of(cfg_name, cfg),
                   "l2": "flushed between timed steps (256 MiB written, then read back: clean lines)", "parallelism": f"replicas x{world}",
                   "launch": "CUDA graph replay"},
        "plain": {"value": round(npx / (r["plain_ms"] * 1e-3) / 1e6, 2), "unit": "MPix/s",
                  "ms_per_step": round(r["plain_ms"], 5),
                  "launches_per_step": r["plain_launches"] / r["plain_steps"],
                  "schedule": "stage-per-kernel (one launch per stage), CUDA graph replay"},
        "speedup_vs_plain": round(r["plain_ms"] / ms, 3),
        "e2e": {"value": round(npx / e2e_s / 1e6, 2), "unit": "MPix/s",
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes, "parity_spot": err_e2e,
                "api": "hp_realize_host_async per image (copy in, realize, copy out; consecutive images "
                       "overlap), hp_realize_host_wait after the last",
                "one_image_per_call": {"value": round(npx / e2e_sync_s / 1e6, 2), "unit": "MPix/s",
                                       "api": "hp_realize_host (synchronises every call)"}},
        "gpu_launches": int(r["launches"]),
        "roofline": r["roof"],
        "fp32_peak_probe": fp32,
        "clocks": r["clocks"],
        "parity_spot": r["err"],
        "step_ms_p50": round(statistics.median(r["ms_all"]), 5),
        "step_ms_p99": round(float(np.percentile(r["ms_all"], 99)), 5),
    }
    if others:
        line["configs"] = others
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, seconds=args.cpu_seconds)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(cfg_name, seconds=args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    return line


# ------------------------------------------------------------- oracle (CPU) --
def cpu_baseline(cfg, seconds=15.0):
    """The oracle, as it stands, on a bounded band of the same workload."""
    rows = cfg["sample_rows"]
    fn = cfg["oracle_sample"](rows)
    t0 = time.perf_counter()
    n = 0
    while True:
        fn()
        n += 1
        if time.perf_counter() - t0 >= seconds * 0.5:
            break
    dt = (time.perf_counter() - t0) / n
    return {"value": round(rows * cfg["w"] / dt / 1e6, 4), "unit": "MPix/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} run(s) of the oracle on a {cfg['w']}x{rows} band of the workload (same per-pixel "
                      f"work), numpy, 1 thread"}


def _oracle_worker(cfg_name, seconds):
    """One host process of the all-cores oracle timing: its own band, as many
    runs as fit in `seconds` (at least one).  Returns (pixels, elapsed)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    cfg = config_table()[cfg_name]
    rows = cfg["sample_rows"]
    fn = cfg["oracle_sample"](rows)
    t0 = time.perf_counter()
    n = 0
    while True:
        fn()
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return rows * cfg["w"] * n, time.perf_counter() - t0


def cpu_baseline_all_cores(cfg_name, seconds=15.0):
    """The oracle on every host core at once: one process per core (spawned, so
    no CUDA state is inherited), each on its own band of the workload; rate =
    all pixels / the slowest process's wall time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(cfg_name, seconds * 0.5)] * cores)
    px = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    cfg = config_table()[cfg_name]
    return {"value": round(px / wall / 1e6, 4), "unit": "MPix/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each running the oracle on a {cfg['w']}x{cfg['sample_rows']} band of the "
                      f"workload for about {seconds * 0.5:.0f} s (numpy, 1 thread each)"}


def run_reference(args, cfg_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cfg = config_table()[cfg_name]
    # size each step's band so that all steps together take about two minutes
    probe_rows = 8
    fn = cfg["oracle_sample"](probe_rows)
    t0 = time.perf_counter()
    fn()
    per_row = (time.perf_counter() - t0) / probe_rows
    rows = int(max(1, min(cfg["h"], 120.0 / max(args.steps, 1) / per_row)))   # a band of one row at least
    fn = cfg["oracle_sample"](rows)
    for _ in range(min(args.warmup, 1)):
        fn()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fn()
    dt = (time.perf_counter() - t0) / args.steps
    v = round(rows * cfg["w"] / dt / 1e6, 4)
    return {"metric": METRIC, "value": v, "unit": "MPix/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": cfg["workload"], "sample": f"{cfg['w']}x{rows} band per step"},
            "cpu_baseline": {"value": v, "unit": "MPix/s", "cores": 1, "kind": "oracle",
                             "sample": f"FP64 oracle on a {cfg['w']}x{rows} band per step, numpy, 1 thread"},
            "e2e": {"value": v, "unit": "MPix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ serving --
SERVING_SIZES = [(256, 256), (480, 640), (1080, 1920), (1536, 2560), (3072, 4096)]
# The serving arena: large enough that every slot keeps the staging of every
# request shape resident (8 slots x about 1 GB of shapes), so no slot gives a
# region back and re-captures its graph during the timed region.
SERVING_ARENA = 32 << 30


def serving_setup():
    """One pipeline per kind and size, each with the autotuned schedule of
    that size, with pinned host inputs and a ring of pinned host outputs."""
    import torch
    from paper_2012_07145_gb300 import hp, pipelines, synth
    import __graft_entry__
    __graft_entry__.build()
    defaults = {"unsharp": dict(schedule="fused", impl=hp.HP_IMPL_WAVE, tile_w=120, tile_h=16, threads=128),
                "harris": dict(schedule="fused", impl=hp.HP_IMPL_WAVE, tile_w=120, tile_h=14, threads=128),
                "histeq": dict(schedule="fused")}
    kinds = [("unsharp", pipelines.unsharp, 3, hp.HP_F32, 3, torch.float32),
             ("harris", pipelines.harris, 3, hp.HP_F32, 1, torch.float32),
             ("histeq", pipelines.histeq, 1, hp.HP_U8, 1, torch.uint8)]
    ring = 3
    bufs = {}
    for name, build, ic, idt, oc, tdt in kinds:
        for (h, w) in SERVING_SIZES:
            p = build()
            app_schedule(name, w, h, "u8" if name == "histeq" else "f32", defaults[name])(p)
            arr = synth.rgb_f32(h, w, seed=7) if idt == hp.HP_F32 else synth.gray_u8_lowcontrast(h, w, seed=7)
            hin = torch.from_numpy(arr).pin_memory()
            outs = [torch.empty((oc, h, w), dtype=tdt).pin_memory() for _ in range(ring)]
            odt = hp.HP_U8 if idt == hp.HP_U8 else hp.HP_F32
            din = hp.padded_copy(hin, "cuda")
            douts = [hp.padded_empty(oc, h, w, tdt, "cuda") for _ in range(ring)]
            bufs[(name, h, w)] = (p, hp.buffer_from_tensor(hin, idt), [hp.buffer_from_tensor(o, odt) for o in outs],
                                  hin, outs, hp.buffer_from_tensor(din, idt), [hp.buffer_from_tensor(o, odt) for o in douts])
    return [k[0] for k in kinds], bufs, ring


def serve_rate(kinds, bufs, ring, lam, n, rng, device=False):
    """n Poisson arrivals at lam per second, kind and size drawn uniformly,
    through a fresh server; returns the per-rate record.  device: the requests'
    buffers are in device memory (no host copies in the latency)."""
    from paper_2012_07145_gb300 import hp
    picks = [(kinds[rng.integers(len(kinds))],) + SERVING_SIZES[rng.integers(len(SERVING_SIZES))] for _ in range(n)]
    gaps = rng.exponential(1.0 / lam, n)
    srv = hp.Server(hbm_budget_bytes=SERVING_ARENA, slots=8, max_batch=8)
    submit = srv.submit_device if device else srv.submit
    bi_of = (lambda k: bufs[k][5]) if device else (lambda k: bufs[k][1])
    bo_of = (lambda k, j: bufs[k][6][j % ring]) if device else (lambda k, j: bufs[k][2][j % ring])
    # make the slots' pipeline copies resident for every kind and size
    # (lowering, scratch, kernel state), then a few requests per slot and key
    # (kernel attributes are set on a kernel's first launch; a slot's graphs
    # are captured on a shape's second realize)
    for k in bufs:
        srv.prepare(bufs[k][0], [bufs[k][1]])
    warm = [submit(bufs[k][0], [bi_of(k)], bo_of(k, j)) for k in bufs for j in range(16)]
    for t in warm:
        srv.wait(t, 120000)
    base = srv.stats()
    t0 = time.perf_counter()
    due = t0
    tickets = []
    for i, (name, h, w) in enumerate(picks):
        due += gaps[i]
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            if due - now > 2e-4:
                time.sleep((due - now) - 1e-4)
        key = (name, h, w)
        tickets.append(submit(bufs[key][0], [bi_of(key)], bo_of(key, i)))
    lats, per = [], []
    for t, (name, h, w) in zip(tickets, picks):
        st, lat = srv.wait(t, 300000)
        if st == hp.HP_OK:
            lats.append(lat)
            per.append((lat, name, h, w))
    t1 = time.perf_counter()
    stats = srv.stats()
    srv.close()
    mpix = sum(h * w for _, h, w in picks) / 1e6
    return {"rate_per_s": lam, "requests": n, "completed": len(lats), "host_copies": not device,
            "p50_ms": round(float(np.percentile(lats, 50)) / 1e3, 3),
            "p99_ms": round(float(np.percentile(lats, 99)) / 1e3, 3),
            "mpix_per_s": round(mpix / (t1 - t0), 1),
            "batched_launches": int(stats.batched_launches - base.batched_launches),
            "graph_replays": int(stats.graph_replays - base.graph_replays),
            "peak_hbm_bytes": int(stats.peak_bytes),
            "slowest": [f"{n} {w}x{h} {l / 1e3:.2f} ms" for l, n, h, w in sorted(per, reverse=True)[:4]]}


def serving_compact(rate=1000.0, requests=300):
    kinds, bufs, ring = serving_setup()
    host = serve_rate(kinds, bufs, ring, rate, requests, np.random.default_rng(0))
    dev = serve_rate(kinds, bufs, ring, rate, requests, np.random.default_rng(0), device=True)
    return {"workload": "serving_mix_unsharp_harris_histeq_poisson", "slots": 8, "max_batch": 8,
            "hbm_budget_bytes": SERVING_ARENA,
            "latency": "submit to completion observed by the server", "with_host_copies": host,
            "device_buffers": dev}


def run_serving(args):
    """Poisson streams of requests drawn uniformly from {unsharp, Harris,
    histogram equalize} x five image sizes, through the continuous-batching
    server; p50/p99 latency and MPix/s per arrival rate."""
    kinds, bufs, ring = serving_setup()
    rates = [float(r) for r in args.rates.split(",")]
    rng = np.random.default_rng(0)
    per_rate = [serve_rate(kinds, bufs, ring, lam, args.requests, rng) for lam in rates]
    per_rate += [serve_rate(kinds, bufs, ring, lam, args.requests, rng, device=True) for lam in rates]
    top = per_rate[len(rates) - 1]
    return {"metric": METRIC, "value": top["mpix_per_s"], "unit": "MPix/s", "n_gpus": 1, "steps": args.requests,
            "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed (f32 RGB, u8)", "data": "synthetic",
            "config": {"workload": "serving_mix_unsharp_harris_histeq_poisson",
                       "sizes": ["%dx%d" % (w, h) for h, w in SERVING_SIZES], "slots": 8, "max_batch": 8,
                       "schedules": "per kind and size from schedules.json (tuner.py)",
                       "hbm_budget_bytes": SERVING_ARENA,
                       "latency": "submit to completion observed by the server; host_copies: pinned host "
                                  "buffers copied in and out inside the latency, else device buffers"},
            "serving": per_rate}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="chain32", help="workload name, or 'all' (one line per workload)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--rates", default="200,500,1000,2000", help="serving: Poisson arrival rates per second")
    ap.add_argument("--requests", type=int, default=300, help="serving: requests per arrival rate")
    ap.add_argument("--configs", default=DEFAULT_CONFIGS,
                    help="workloads reported compactly in the headline line ('' for none)")
    ap.add_argument("--only-fused", action="store_true",
                    help="time the fused pipeline only (for profiler runs); prints no bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.config == "serving":
        line = run_serving(args) if args.impl == "ours" else {"impl": "reference", "unavailable":
                                                              "the serving loop has no CPU counterpart"}
        print(json.dumps(line), flush=True)
        return
    names = list(config_table().keys()) if args.config == "all" else [args.config]
    for name in names:
        line = run_reference(args, name) if args.impl == "reference" else run_ours(args, name)
        if line is not None:
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
