"""GPU parity of the max filter (exact), interpolate and bilateral grid (FP32
against the FP64 oracle; the grid's counts exact) apps, plus schedule
invariance."""

import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import bilateral_grid as ob
from oracle import interpolate as oi
from oracle import maxfilter as om
from paper_2012_07145_gb300 import hp, pipelines, synth

from gpu_util import bits, rel_err, run, to_device, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


# ------------------------------------------------------------- max filter --
# Window maxima are exact: every schedule and the oracle agree bit for bit.
@pytest.mark.parametrize("h,w", [(1536, 2560), (37, 53), (1, 1), (2, 3), (130, 250)])
@pytest.mark.parametrize("radius", [1, 4])
def test_max_filter_bit_exact(h, w, radius):
    img = synth.rgb_f32(h, w, seed=h + w + radius)
    x = to_device(img, hp.HP_F32)
    p = pipelines.max_filter(radius)
    pipelines.root_schedule(p)
    plain = run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)
    sample = (slice(None), slice(0, min(h, 96)), slice(0, min(w, 96)))
    ref = om.max_filter_planes(img[sample], radius, radius)
    got = to_numpy(plain)[sample]
    if h <= 96 and w <= 96:
        assert np.array_equal(got, ref)
    else:   # the sampled corner: its window maxima only read inside the sample except near its far edges
        m = radius
        assert np.array_equal(got[:, :96 - m, :96 - m], ref[:, :96 - m, :96 - m])
    assert [p.group_info([(w, h)], g).kernel for g in range(2)] == [hp.HP_KERNEL_MAX_ROWS] * 2
    for rows, t in [(0, 256), (1, 32), (7, 96), (64, 128)]:      # the streaming kernel, fused
        p.schedule([0, 0], tile_h=[rows], threads=[t])
        assert p.group_info([(w, h)], 0).kernel == hp.HP_KERNEL_MAX_ROWS
        assert torch.equal(bits(run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)), bits(plain))
    for tw, th, t in [(64, 32, 256), (32, 8, 128), (128, 16, 512)]:   # the generic interpreter
        p.schedule([0, 0], tile_w=[tw], tile_h=[th], threads=[t], impl=[hp.HP_IMPL_GENERIC])
        assert torch.equal(bits(run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)), bits(plain))


def test_max_filter_full_size_against_oracle_everywhere():
    h, w = 300, 500
    img = synth.rgb_f32(h, w, seed=9)
    p = pipelines.max_filter(4)
    p.schedule([0, 0])
    got = to_numpy(run(p, [to_device(img, hp.HP_F32)], [hp.HP_F32], (3, h, w), hp.HP_F32))
    assert np.array_equal(got, om.max_filter_planes(img, 4, 4))
    # one square stage on the streaming kernel: the same values
    q = hp.Pipeline([hp.HP_F32], [3])
    q.set_output(q.add_stage(hp.HP_MAX_STENCIL, [q.input(0)], 3, hp.HP_F32, rx=4, ry=4))
    assert q.group_info([(w, h)], 0).kernel == hp.HP_KERNEL_MAX_ROWS
    got = to_numpy(run(q, [to_device(img, hp.HP_F32)], [hp.HP_F32], (3, h, w), hp.HP_F32))
    assert np.array_equal(got, om.max_filter_planes(img, 4, 4))


@pytest.mark.parametrize("h,w,radius,rows", [(61, 77, 3, 16), (130, 250, 4, 5), (257, 365, 2, 0)])
def test_max_filter_bf16_io(h, w, radius, rows):
    """bf16 input rows reach the streaming kernel as TMA boxes that start four
    columns left of the strip's halo lane (16-byte alignment): several strips,
    runs cut at every offset against the 4-row boxes, and the clamped edges."""
    img = torch.from_numpy(synth.rgb_f32(h, w, seed=10 + h)).to(torch.bfloat16).float().numpy()
    p = pipelines.max_filter(radius, io_storage=hp.HP_BF16)
    ref = om.max_filter_planes(img, radius, radius)   # maxima of bf16 values are bf16 values
    for impl in (None, [hp.HP_IMPL_GENERIC]):
        p.schedule([0, 0], tile_w=[32], tile_h=[rows if impl is None else 16], threads=[128], impl=impl)
        got = to_numpy(run(p, [to_device(img, hp.HP_BF16)], [hp.HP_BF16], (3, h, w), hp.HP_BF16))
        assert np.array_equal(got, ref)


# ------------------------------------------------------------ interpolate --
# FP32 arithmetic against the FP64 oracle; the final division by the coverage
# (at least the sample density's order) amplifies the pyramid's rounding, so
# the bound is stated on the output range [0, 1]: 1e-5.
INTERP_TOL = 1e-5


@pytest.mark.parametrize("h,w,levels", [(96, 160, 6), (37, 53, 4), (1, 1, 1), (2, 3, 2), (257, 131, 7)])
def test_interpolate_against_oracle_and_schedules(h, w, levels):
    img = synth.rgba_sparse_f32(h, w, seed=h * 3 + w)
    x = to_device(img, hp.HP_F32)
    p, ids = pipelines.interpolate(levels)
    plain = run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)
    ref = oi.interpolate(img.astype(np.float64), levels)
    err = float(np.abs(to_numpy(plain).astype(np.float64) - ref).max())
    print(f"interpolate {w}x{h} J={levels}: max abs err {err:.3e}")
    assert err <= INTERP_TOL
    for kw in (dict(), dict(down_tile=16), dict(impl=hp.HP_IMPL_GENERIC, tile=16), dict(tile=64, threads=128),
               dict(level_tile=1, threads=32), dict(level_tile=3, threads=96), dict(level_tile=40)):
        pipelines.interpolate_fused_schedule(p, ids, **kw)
        if levels > 1 and not kw.get("impl"):   # the composites run on the streaming level kernel
            assert p.group_info([(w, h)], p.group_count() - 1).kernel == hp.HP_KERNEL_INTERP_ROWS
        assert torch.equal(bits(run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)), bits(plain)), kw


def test_interpolate_full_size():
    h, w = 1536, 2560
    img = synth.rgba_sparse_f32(h, w, seed=0)
    x = to_device(img, hp.HP_F32)
    p, ids = pipelines.interpolate(10)
    plain = run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)
    pipelines.interpolate_fused_schedule(p, ids)
    fused = run(p, [x], [hp.HP_F32], (3, h, w), hp.HP_F32)
    assert torch.equal(bits(fused), bits(plain))
    # covered pixels keep their colour exactly; a sampled band against the oracle
    got = to_numpy(fused)
    cov = img[3] > 0
    assert np.array_equal(got[:, cov], img[:3][:, cov])
    ref = oi.interpolate(img.astype(np.float64), 10)
    assert float(np.abs(got.astype(np.float64) - ref).max()) <= INTERP_TOL


def test_interpolate_full_coverage_is_identity():
    h, w = 45, 67
    img = synth.rgba_sparse_f32(h, w, seed=3, coverage=1.0)
    p, ids = pipelines.interpolate(5)
    pipelines.interpolate_fused_schedule(p, ids)
    got = to_numpy(run(p, [to_device(img, hp.HP_F32)], [hp.HP_F32], (3, h, w), hp.HP_F32))
    assert np.array_equal(got, img[:3])


# --------------------------------------------------------- bilateral grid --
def _splat_only(s, r):
    gz = ob.levels(r)
    p = hp.Pipeline([hp.HP_F32], [1])
    p.set_output(p.add_stage(hp.HP_GRID_SPLAT, [p.input(0)], 2 * gz, hp.HP_F32, params=[s, r]))
    return p, gz


@pytest.mark.parametrize("h,w,s,r", [(37, 53, 4, 0.2), (96, 160, 8, 0.1), (1, 1, 2, 0.5), (130, 250, 8, 0.05)])
def test_grid_splat_counts_exact(h, w, s, r):
    """The splat's counts are exact integers, so every cell's count per range
    level (decided in f32 on both sides) must match the oracle's exactly; the
    sums of values within FP32 rounding."""
    img = synth.gray_f32_gradient_noise(h, w, seed=h + w)
    p, gz = _splat_only(s, r)
    GX, GY = ob.grid_size(w, h, s)
    got = to_numpy(run(p, [to_device(img, hp.HP_F32)], [hp.HP_F32], (2 * gz, GY, GX), hp.HP_F32))
    ref = ob.splat(img[0], s, r)                        # [GY][GX][GZ][2]
    counts = got[1::2].transpose(1, 2, 0)
    sums = got[0::2].transpose(1, 2, 0)
    assert np.array_equal(counts, ref[..., 1])
    assert np.abs(sums - ref[..., 0]).max() <= 1e-5 * s * s


@pytest.mark.parametrize("h,w,s,r", [(37, 53, 4, 0.2), (96, 160, 8, 0.1), (1, 1, 2, 0.5), (257, 131, 8, 0.1)])
def test_bilateral_grid_against_oracle_and_schedules(h, w, s, r):
    img = synth.gray_f32_gradient_noise(h, w, seed=3 * h + w)
    x = to_device(img, hp.HP_F32)
    p = pipelines.bilateral_grid(s, r)
    plain = run(p, [x], [hp.HP_F32], (1, h, w), hp.HP_F32)
    ref = ob.bilateral_grid(img[0], s, r)
    err = float(np.abs(to_numpy(plain)[0].astype(np.float64) - ref).max())
    print(f"bilateral grid {w}x{h} s={s} r={r}: max abs err {err:.3e}")
    assert err <= 1e-5
    for tile, threads, impl in ((0, 256, None), (1, 256, None), (7, 256, None), (64, 256, None),
                                (16, 128, hp.HP_IMPL_GENERIC), (32, 512, hp.HP_IMPL_GENERIC)):
        pipelines.bilateral_grid_fused_schedule(p, tile, threads, impl)
        blur = p.group_info([(w, h)], 1).kernel
        assert blur == (hp.HP_KERNEL_GENERIC if impl else hp.HP_KERNEL_GRID_BLUR)
        assert torch.equal(bits(run(p, [x], [hp.HP_F32], (1, h, w), hp.HP_F32)), bits(plain))


def test_bilateral_grid_full_size_and_edges():
    h, w = 1536, 2560
    img = synth.gray_f32_gradient_noise(h, w, seed=0)
    p = pipelines.bilateral_grid(8, 0.1)
    pipelines.bilateral_grid_fused_schedule(p)
    got = to_numpy(run(p, [to_device(img, hp.HP_F32)], [hp.HP_F32], (1, h, w), hp.HP_F32))[0]
    band = slice(0, 96)
    ref = ob.bilateral_grid(img[0][band], 8, 0.1)
    # the band's last grid rows see the clamped band edge instead of the image below
    assert float(np.abs(got[band][:64].astype(np.float64) - ref[:64]).max()) <= 1e-5
    step = np.full((1, 64, 96), 0.2, dtype=np.float32)
    step[:, :, 48:] = 0.8     # six range cells apart: each side keeps its value
    out = to_numpy(run(p, [to_device(step, hp.HP_F32)], [hp.HP_F32], (1, 64, 96), hp.HP_F32))[0]
    assert np.abs(out[:, :48] - np.float32(0.2)).max() <= 1e-6 and np.abs(out[:, 48:] - np.float32(0.8)).max() <= 1e-6
