"""C ABI checks that need no GPU: the library loads and exports every symbol
include/hp.h declares; stage/schedule validation; bounds inference; lowering."""

import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2012_07145_gb300 import hp, pipelines

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:hp_status|const char\*|unsigned long long)\s+(hp_\w+)\(", text, re.M)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 12
    L = ctypes.CDLL(hp.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(hp.EXPORTS)


def test_stage_validation_errors():
    p = hp.Pipeline([hp.HP_F32], [1])
    with pytest.raises(hp.HPError) as e:
        p.add_stage(hp.HP_STENCIL, [p.input(3)], 1, rx=2, ry=2, wx=[0.2] * 5, wy=[0.2] * 5)
    assert e.value.status == hp.HP_ERR_INVALID_ARG
    with pytest.raises(hp.HPError):
        p.add_stage(hp.HP_STENCIL, [p.input(0)], 1, rx=9, ry=2, wx=[0.1] * 19, wy=[0.2] * 5)
    with pytest.raises(hp.HPError):  # gray needs 3 channels
        p.add_stage(hp.HP_POINTWISE, [p.input(0)], 1, op=hp.HP_OP_GRAY, params=[1.0])
    with pytest.raises(hp.HPError):  # histogram of a float image
        p.add_stage(hp.HP_HISTOGRAM, [p.input(0)], 1, hp.HP_U32)
    s = p.add_stage(hp.HP_STENCIL, [p.input(0)], 1, rx=2, ry=2, wx=[0.2] * 5, wy=[0.2] * 5)
    assert s == 0


def test_schedule_validation():
    p = pipelines.stencil_chain(4, "binomial")
    with pytest.raises(hp.HPError) as e:  # stencils cannot be inlined
        p.schedule([0, hp.HP_INLINE, 1, 1])
    assert e.value.status == hp.HP_ERR_SCHEDULE
    with pytest.raises(hp.HPError):  # group 0 would export two stages
        p.schedule([0, 1, 0, 1])
    p.schedule([0, 0, 1, 1])
    assert p.group_count() == 2
    # a tile that needs more shared memory than a CTA has fails at lowering
    p.schedule([0, 0, 0, 0], tile_w=[512], tile_h=[512])
    with pytest.raises(hp.HPError) as e:
        p.group_info([(512, 512)], 0)
    assert e.value.status == hp.HP_ERR_SCHEDULE


def test_lowering_picks_kernels():
    p = pipelines.stencil_chain(32, "alternate")
    assert p.group_count() == 32
    # a single 5x5 stencil defaults to the streaming kernel (120-column strips);
    # another tile width selects the tiled chain kernel
    info = p.group_info([(2560, 1536)], 0)
    assert info.kernel == hp.HP_KERNEL_STENCIL_ROWS and info.n_members == 1 and info.tile_w == 120
    p.schedule(list(range(32)), tile_w=[64] * 32, tile_h=[32] * 32)
    assert p.group_info([(2560, 1536)], 0).kernel == hp.HP_KERNEL_STENCIL_CHAIN
    p.schedule(list(range(32)), tile_w=[64] * 32, impl=[hp.HP_IMPL_WAVE] * 32)
    with pytest.raises(hp.HPError) as e:   # the streaming kernel's strip width is fixed
        p.group_info([(2560, 1536)], 0)
    assert e.value.status == hp.HP_ERR_SCHEDULE
    pipelines.chain_schedule(p, depth=8, tile_w=64, tile_h=32)
    info = p.group_info([(2560, 1536)], 0)
    assert info.kernel == hp.HP_KERNEL_STENCIL_CHAIN and info.n_members == 8
    assert (info.grid_x, info.grid_y, info.grid_z) == (40, 48, 1)
    u = pipelines.unsharp()
    pipelines.fused_schedule(u)
    assert u.group_info([(64, 48)], 0).kernel == hp.HP_KERNEL_UNSHARP
    pipelines.fused_schedule(u, tile_w=120, tile_h=96)
    assert u.group_info([(4096, 3072)], 0).kernel == hp.HP_KERNEL_STENCIL_ROWS
    h = pipelines.histeq()
    kinds = [h.group_info([(100, 50)], g).kernel for g in range(3)]
    assert kinds == [hp.HP_KERNEL_HISTOGRAM, hp.HP_KERNEL_CDF_LUT, hp.HP_KERNEL_LUT_APPLY]
    pipelines.fused_schedule(h)   # all three in one group: one cooperative kernel
    info = h.group_info([(4096, 3072)], 0)
    assert h.group_count() == 1 and info.kernel == hp.HP_KERNEL_HISTEQ and info.threads == 1024
    assert 1 <= info.grid_x <= 4096 * 3072 // 16 // 2048 + 1
    hr = pipelines.harris()
    pipelines.fused_schedule(hr, impl=hp.HP_IMPL_GENERIC)
    assert hr.group_info([(64, 48)], 0).kernel == hp.HP_KERNEL_GENERIC
    pipelines.fused_schedule(hr)
    assert hr.group_info([(64, 48)], 0).kernel == hp.HP_KERNEL_HARRIS
    pipelines.fused_schedule(hr, inline_pointwise=True)
    info = hr.group_info([(64, 48)], 0)
    assert info.kernel == hp.HP_KERNEL_HARRIS and info.n_members == 10
    # the streaming Harris kernel: 120-column strips for 4-byte input, 112 for 2-byte
    pipelines.fused_schedule(hr, tile_w=120, tile_h=28, threads=256)
    info = hr.group_info([(2560, 1536)], 0)
    assert info.kernel == hp.HP_KERNEL_HARRIS_ROWS and info.grid_x >= 1
    pipelines.fused_schedule(hr, tile_w=112, tile_h=28, impl=hp.HP_IMPL_WAVE)
    with pytest.raises(hp.HPError) as e:
        hr.group_info([(64, 48)], 0)
    assert e.value.status == hp.HP_ERR_SCHEDULE
    hb = pipelines.harris(io_storage=hp.HP_BF16)
    pipelines.fused_schedule(hb, tile_w=112, tile_h=3, impl=hp.HP_IMPL_WAVE)
    with pytest.raises(hp.HPError):
        hb.group_info([(64, 48)], 0)
    pipelines.fused_schedule(hb, tile_w=112, tile_h=8)
    assert hb.group_info([(64, 48)], 0).kernel == hp.HP_KERNEL_HARRIS_ROWS


def test_lowering_line_buffer_chain():
    """HP_IMPL_LINES puts an even-depth chain on the line-buffer kernel, with
    one block per tile and threads for every stage's 8-column blocks; chains
    outside its limits keep the tiled kernel."""
    p = pipelines.stencil_chain(32, "alternate")
    pipelines.chain_schedule(p, depth=8, tile_w=128, tile_h=64, impl=hp.HP_IMPL_LINES)
    info = p.group_info([(2560, 1536)], 0)
    assert info.kernel == hp.HP_KERNEL_STENCIL_LINES and info.n_members == 8
    assert (info.grid_x, info.grid_y, info.grid_z) == (20, 24, 1)
    # stages 1..8 are 156, 152, ..., 128 columns wide; pairs take the wider one's
    # 8-column blocks twice: 2 * (20 + 19 + 18 + 17) = 148 threads, rounded to 160
    assert info.threads == 160
    for depth, tw, th in ((3, 64, 32), (8, 128, 17), (8, 232, 64), (2, 64, 5)):
        q = pipelines.stencil_chain(24, "alternate")
        pipelines.chain_schedule(q, depth=depth, tile_w=tw, tile_h=th, impl=hp.HP_IMPL_LINES)
        assert q.group_info([(640, 480)], 0).kernel == hp.HP_KERNEL_STENCIL_CHAIN, (depth, tw, th)
    # 16-bit chains: 4 or 8 stages (the box start stays 16-byte aligned)
    for depth, kern in ((2, hp.HP_KERNEL_STENCIL_CHAIN), (4, hp.HP_KERNEL_STENCIL_LINES)):
        q = pipelines.stencil_chain(8, "alternate", storage=hp.HP_F16)
        pipelines.chain_schedule(q, depth=depth, tile_w=64, tile_h=32, impl=hp.HP_IMPL_LINES)
        assert q.group_info([(640, 480)], 0).kernel == kern


def test_async_host_realize_refuses_bad_arguments_before_any_cuda_call():
    """hp_realize_host_async checks its arguments (and every host pointer) before
    lowering or touching the device; waiting with nothing enqueued returns at once."""
    L = hp.lib()
    assert L.hp_realize_host_async(None, None, 0, None, None) == hp.HP_ERR_INVALID_ARG
    assert L.hp_realize_host_wait(None) == hp.HP_ERR_INVALID_ARG
    p = pipelines.stencil_chain(4, "binomial")
    inp = hp.Buffer(None, hp.HP_F32, 1, 64, 32, 256, 256 * 32)
    out = hp.Buffer(None, hp.HP_F32, 1, 64, 32, 256, 256 * 32)
    with pytest.raises(hp.HPError) as e:
        p.realize_host_async([inp], out)
    assert e.value.status == hp.HP_ERR_INVALID_ARG
    p.realize_host_wait()


def test_bounds_inference_stencil_chain():
    # Fusing d 5x5 stages: stage k of the group needs the tile grown by 2(d-1-k) per side, clamped.
    p = pipelines.stencil_chain(4, "binomial")
    p.schedule([0, 0, 0, 0])
    W, H = 100, 60
    r = p.infer_bounds([(W, H)], 0, 32, 16, 16, 8)
    assert r[3] == (32, 16, 48, 24)
    assert r[2] == (30, 14, 50, 26)
    assert r[1] == (28, 12, 52, 28)
    assert r[0] == (26, 10, 54, 30)
    r = p.infer_bounds([(W, H)], 0, 0, 0, 16, 8)     # corner tile: clamped to the image
    assert r[0] == (0, 0, 22, 14)
    r = p.infer_bounds([(W, H)], 0, 96, 56, 16, 8)   # ragged corner tile
    assert r[3] == (96, 56, 100, 60)
    assert r[0] == (90, 50, 100, 60)


def test_bounds_inference_pyramid_and_harris():
    pl, ids = pipelines.local_laplacian(levels=3, k_levels=4)
    pipelines.local_laplacian_fused_schedule(pl, ids, tile=16)
    # group 0 computes G1 (downsample) from the inlined remap of gray
    r = pl.infer_bounds([(64, 40)], 0, 8, 4, 8, 4)
    assert r[ids["G"][1]] == (8, 4, 16, 8)
    assert r[ids["G"][0]] == (14, 6, 33, 17)      # [2*8-2, 2*16+1) x [2*4-2, 2*8+1)
    assert r[ids["gray"]] == r[ids["G"][0]]
    hr = pipelines.harris()
    pipelines.fused_schedule(hr)
    r = hr.infer_bounds([(50, 40)], 0, 16, 8, 16, 8)
    assert r[9] == (16, 8, 32, 16)                 # response
    assert r[6] == r[7] == r[8] == (16, 8, 32, 16)  # box sums
    assert r[3] == (15, 7, 33, 17)                 # products: +1 for the box
    assert r[1] == (15, 7, 33, 17)
    assert r[0] == (14, 6, 34, 18)                 # gray: +1 more for Sobel


def test_local_laplacian_lowering():
    J = 5
    pl, ids = pipelines.local_laplacian(levels=J, k_levels=8)
    pipelines.local_laplacian_fused_schedule(pl, ids, tile=16)
    n = pl.group_count()
    assert n == 2 * J - 2
    kinds = [pl.group_info([(160, 96)], g).kernel for g in range(n)]
    # level 1 straight from the input: the streaming remap downsample by default
    assert kinds == ([hp.HP_KERNEL_LL_REMAP_ROWS] + [hp.HP_KERNEL_LL_DOWN_ROWS] * (J - 2) +
                     [hp.HP_KERNEL_LL_LEVEL_ROWS] * (J - 1))
    assert pl.group_info([(160, 96)], 0).n_members == 3          # gray and remap inlined
    info = pl.group_info([(160, 96)], 0)
    assert info.tile_w == 30 and info.tile_h >= 1 and info.threads == 256
    # an explicit power-of-two tile takes the tiled kernel
    pipelines.local_laplacian_fused_schedule(pl, ids, tile=16, down_tile=16, level_tile=32)
    assert all(pl.group_info([(160, 96)], g).kernel == hp.HP_KERNEL_DOWNSAMPLE for g in range(J - 1))
    assert all(pl.group_info([(160, 96)], g).kernel == hp.HP_KERNEL_LL_LEVEL for g in range(J - 1, n))
    pipelines.local_laplacian_fused_schedule(pl, ids, tile=16, impl=hp.HP_IMPL_WAVE, down_tile=16)
    assert pl.group_info([(160, 96)], 0).kernel == hp.HP_KERNEL_LL_REMAP_ROWS
    # a band as wide as the level spacing: three levels could hold one gray value
    wide, wide_ids = pipelines.local_laplacian(levels=J, k_levels=8, sigma_r=0.15)
    pipelines.local_laplacian_fused_schedule(wide, wide_ids, tile=16)
    assert wide.group_info([(160, 96)], 0).kernel == hp.HP_KERNEL_DOWNSAMPLE
    assert wide.group_info([(160, 96)], 1).kernel == hp.HP_KERNEL_LL_DOWN_ROWS
    # the boundary: sigma just below the spacing 1/7 takes the streaming remap
    # kernel (its two-level band logic holds), sigma = 1/7 does not
    for sigma, streaming in ((0.142, True), (1.0 / 7.0, False)):
        q, q_ids = pipelines.local_laplacian(levels=J, k_levels=8, sigma_r=sigma)
        pipelines.local_laplacian_fused_schedule(q, q_ids, tile=16)
        assert (q.group_info([(160, 96)], 0).kernel == hp.HP_KERNEL_LL_REMAP_ROWS) == streaming, sigma
    pipelines.local_laplacian_fused_schedule(pl, ids, tile=16)
    assert pl.group_info([(160, 96)], n - 1).n_members == 8      # level 0: + colour, gray, remap
    pipelines.local_laplacian_fused_schedule(pl, ids, tile=16, impl=hp.HP_IMPL_GENERIC)
    assert all(pl.group_info([(160, 96)], g).kernel == hp.HP_KERNEL_GENERIC for g in range(n))


def test_options():
    """Options need no GPU to set; unknown ones are rejected."""
    p = pipelines.stencil_chain(4, "binomial")
    p.use_cuda_graph(True)
    p.overlap_launches(False)
    p.overlap_launches(True)
    p.set_option(hp.HP_OPT_OVERLAP, 0)
    with pytest.raises(hp.HPError):
        p.set_option(99, 1)


def test_new_stage_kinds_validation_and_lowering():
    """Max stencil, interpolate ops and the bilateral grid's stages: argument
    rules, domains and kernel choice (no GPU needed)."""
    p = hp.Pipeline([hp.HP_F32], [3])
    with pytest.raises(hp.HPError):  # radius beyond HP_MAX_RADIUS
        p.add_stage(hp.HP_MAX_STENCIL, [p.input(0)], 3, rx=5, ry=0)
    with pytest.raises(hp.HPError):  # channel count must follow the input
        p.add_stage(hp.HP_MAX_STENCIL, [p.input(0)], 1, rx=2, ry=2)
    with pytest.raises(hp.HPError):  # premultiply needs RGBA
        p.add_stage(hp.HP_POINTWISE, [p.input(0)], 4, op=hp.HP_OP_PREMUL)
    m = pipelines.max_filter(2)
    m.schedule([0, 0])
    assert m.group_info([(50, 40)], 0).kernel == hp.HP_KERNEL_MAX_ROWS
    m.schedule([0, 0], impl=[hp.HP_IMPL_GENERIC])
    assert m.group_info([(50, 40)], 0).kernel == hp.HP_KERNEL_GENERIC

    g = hp.Pipeline([hp.HP_F32], [1])
    with pytest.raises(hp.HPError):  # s must be an integer in [1, 64]
        g.add_stage(hp.HP_GRID_SPLAT, [g.input(0)], 22, params=[2.5, 0.1])
    with pytest.raises(hp.HPError):  # 2 GZ channels: GZ = floor(1/r + 1/2) + 1 = 11
        g.add_stage(hp.HP_GRID_SPLAT, [g.input(0)], 20, params=[8, 0.1])
    b = pipelines.bilateral_grid(8, 0.1)
    kinds = [b.group_info([(100, 70)], k).kernel for k in range(b.group_count())]
    assert kinds == [hp.HP_KERNEL_GRID_SPLAT, hp.HP_KERNEL_POINTWISE, hp.HP_KERNEL_GENERIC, hp.HP_KERNEL_GENERIC,
                     hp.HP_KERNEL_GRID_SLICE]
    pipelines.bilateral_grid_fused_schedule(b)
    assert [b.group_info([(100, 70)], k).kernel for k in range(3)] == [
        hp.HP_KERNEL_GRID_SPLAT, hp.HP_KERNEL_GRID_BLUR, hp.HP_KERNEL_GRID_SLICE]
    with pytest.raises(hp.HPError):  # the splat cannot share a kernel with other stages
        b.schedule([0, 0, 1, 1, 2])
        b.group_info([(100, 70)], 0)

    q, ids = pipelines.interpolate(4)
    pipelines.interpolate_fused_schedule(q, ids)
    ks = [q.group_info([(64, 48)], k).kernel for k in range(q.group_count())]
    assert ks[0] == hp.HP_KERNEL_PW_ROWS and ks[-1] == hp.HP_KERNEL_INTERP_ROWS
    assert q.group_info([(64, 48)], q.group_count() - 1).n_members == 3   # upsample, over, division


def test_histogram_refuses_images_beyond_its_32_bit_counters():
    """The bin counters and the table's running sums are 32-bit: an image of
    2^32 - 1 pixels or fewer lowers, one of more is refused with a message."""
    h = pipelines.histeq()
    assert h.group_info([(65535, 65537)], 0).kernel == hp.HP_KERNEL_HISTOGRAM   # 2^32 - 1 pixels
    with pytest.raises(hp.HPError) as e:
        h.group_info([(65536, 65536)], 0)
    assert e.value.status == hp.HP_ERR_UNSUPPORTED and "2^32 - 1" in str(e.value)
    pipelines.fused_schedule(h)
    with pytest.raises(hp.HPError):
        h.group_info([(65536, 65536)], 0)


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: with libhp.so absent, the first call raises and names the
    build step (run in a child process so this process keeps its library)."""
    import subprocess
    import sys
    code = ("from paper_2012_07145_gb300 import hp\n"
            "hp.LIB_PATH = '/nonexistent/libhp.so'\n"
            "try:\n"
            "    hp.Pipeline([hp.HP_F32], [1])\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('no error')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert "raised:" in r.stdout and "build" in r.stdout, r.stdout + r.stderr


def test_server_argument_validation_needs_no_gpu():
    """Out-of-range server arguments are refused before any CUDA call, and the
    calls on a null server handle return errors instead of crashing."""
    for budget, slots, batch in ((1 << 19, 4, 8), (1 << 30, 0, 8), (1 << 30, 65, 8), (1 << 30, 4, 0), (1 << 30, 4, 65)):
        with pytest.raises(hp.HPError) as e:
            hp.Server(budget, slots, batch)
        assert e.value.status == hp.HP_ERR_INVALID_ARG
    L = hp.lib()
    t = ctypes.c_ulonglong()
    assert L.hp_server_submit(None, None, None, 0, None, ctypes.byref(t)) == hp.HP_ERR_INVALID_ARG
    stats = hp.ServerStats()
    assert L.hp_server_stats_get(None, ctypes.byref(stats)) != hp.HP_OK
    lat = ctypes.c_double()
    assert L.hp_server_wait(None, 1, 0, ctypes.byref(lat)) != hp.HP_OK


def test_bounds_inference_max_filter_and_upsample():
    # max filter fused: the horizontal stage is needed on the tile grown by the
    # vertical radius in y only, clamped to the image
    p = pipelines.max_filter(3)
    p.schedule([0, 0])
    r = p.infer_bounds([(100, 60)], 0, 32, 16, 16, 8)
    assert r[1] == (32, 16, 48, 24)
    assert r[0] == (32, 13, 48, 27)
    r = p.infer_bounds([(100, 60)], 0, 0, 56, 16, 8)    # ragged bottom tile
    assert r[1] == (0, 56, 16, 60) and r[0] == (0, 53, 16, 60)
    # interpolate's finest level fused (upsample of I_1, composite, division):
    # the point-wise consumers need the upsample exactly on the tile, and a
    # ragged tile is clamped to the fine domain
    q = pipelines.interpolate_finest()
    out = q.infer_bounds([(64, 40), (32, 20)], 0, 16, 8, 16, 8)
    assert out == [(16, 8, 32, 16)] * 3
    out = q.infer_bounds([(63, 39), (32, 20)], 0, 48, 32, 16, 8)
    assert out == [(48, 32, 63, 39)] * 3


def test_realize_rejects_bad_buffers_before_touching_the_device():
    """Null, misaligned, wrongly typed, wrongly shaped or too tightly strided
    buffers are refused with HP_ERR_INVALID_ARG by the host checks, before any
    CUDA call (the addresses are never dereferenced)."""
    p = pipelines.stencil_chain(2)
    W, H = 40, 24
    A = 1 << 20                      # a 16-byte-aligned address that is never read

    def buf(data=A, dtype=hp.HP_F32, c=1, w=W, h=H, rs=192, ps=192 * H):
        return hp.Buffer(data, dtype, c, w, h, rs, ps)

    good = buf()
    cases = {
        "null input": ([buf(data=0)], good),
        "misaligned input": ([buf(data=A + 4)], good),
        "row stride not a multiple of 16": ([buf(rs=168, ps=168 * H)], good),
        "row stride below the width": ([buf(rs=144, ps=144 * H)], good),
        "input dtype": ([buf(dtype=hp.HP_F16)], good),
        "input channels": ([buf(c=3, ps=192 * H)], good),
        "empty input": ([buf(w=0)], good),
        "output size": ([good], buf(w=W - 1)),
        "output dtype": ([good], buf(dtype=hp.HP_U8)),
        "null output": ([good], buf(data=0)),
        "input count": ([good, good], good),
    }
    for name, (ins, out) in cases.items():
        with pytest.raises(hp.HPError) as e:
            p.realize(ins, out)
        assert e.value.status == hp.HP_ERR_INVALID_ARG, (name, str(e.value))


def test_binding_constants_equal_the_header():
    """Every enumerator of include/hp.h has the same value in the binding, and
    the kernel names follow the HP_KERNEL_* ids."""
    text = open(os.path.join(ROOT, "include", "hp.h")).read()
    pairs = re.findall(r"\b(HP_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)
    assert len(pairs) >= 60
    for name, value in pairs:
        assert getattr(hp, name) == int(value), name
    assert hp.HP_INLINE == -1
    kernels = sorted((int(v), n) for n, v in pairs if n.startswith("HP_KERNEL_"))
    assert [v for v, _ in kernels] == list(range(len(hp.KERNEL_NAMES)))
    assert [n[len("HP_KERNEL_"):].lower() for _, n in kernels] == list(hp.KERNEL_NAMES)


def test_fp32_probe_refuses_bad_arguments_before_any_cuda_call():
    L = hp.lib()
    f, ms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    assert L.hp_measure_fp32_peak(0, 16, 1, None, None, ctypes.byref(ms), ctypes.byref(sms)) == hp.HP_ERR_INVALID_ARG
    assert L.hp_measure_fp32_peak(0, 0, 1, None, ctypes.byref(f), None, None) == hp.HP_ERR_INVALID_ARG
    assert L.hp_measure_fp32_peak(1, 16, 0, None, ctypes.byref(f), None, None) == hp.HP_ERR_INVALID_ARG
