"""Builders of the imaging pipelines of the paper's evaluation (Sec. 6) as hp
pipelines, with their stage-per-kernel and fused schedules.

Each builder states the algorithm once (stages, footprints, storage types);
schedules only regroup stages into kernels and retile them (Sec. 1, Sec. 4).
"""

import numpy as np

from . import hp

BINOMIAL16 = [0.0625, 0.25, 0.375, 0.25, 0.0625]   # [1,4,6,4,1]/16, per axis
BOX5 = [0.2] * 5                                    # 1/5 per axis -> 1/25 in 2-D
SOBEL_SMOOTH = [1.0, 2.0, 1.0]
SOBEL_DIFF = [-1.0, 0.0, 1.0]
BOX3_SUM = [1.0, 1.0, 1.0]


def chain_kinds(n_stages: int, pattern: str):
    if pattern == "binomial":
        return ["binomial"] * n_stages
    if pattern == "alternate":
        return ["binomial" if k % 2 == 0 else "box" for k in range(n_stages)]
    raise ValueError(pattern)


def stencil_chain(n_stages: int = 32, pattern: str = "alternate", storage: int = hp.HP_F32) -> hp.Pipeline:
    """Chain of 5x5 separable stencils on a 1-channel image (Sec. 2, Fig. 1; the
    32-stage stencil chain of Sec. 6).  Input and every stage use `storage`."""
    p = hp.Pipeline([storage], [1])
    prev = p.input(0)
    for kind in chain_kinds(n_stages, pattern):
        w = BINOMIAL16 if kind == "binomial" else BOX5
        prev = p.add_stage(hp.HP_STENCIL, [prev], 1, storage, rx=2, ry=2, wx=w, wy=w)
    p.set_output(prev)
    return p


def chain_schedule(p: hp.Pipeline, depth: int, tile_w: int = 64, tile_h: int = 32, threads: int = 256,
                   serial_y: int = 8, impl: int = hp.HP_IMPL_AUTO):
    """Fuse consecutive runs of `depth` stages into one kernel each.  With
    impl = HP_IMPL_WAVE the groups run on the streaming kernel (one warp per
    stage; threads and serial_y do not apply)."""
    n = len(p.stages)
    groups = [k // depth for k in range(n)]
    ng = groups[-1] + 1
    p.schedule(groups, tile_w=[tile_w] * ng, tile_h=[tile_h] * ng, threads=[threads] * ng,
               serial_y=[serial_y] * ng, impl=[impl] * ng)


def root_schedule(p: hp.Pipeline, impl=None):
    """Every stage in its own kernel (compute root, Sec. 2 "Separate Kernels")."""
    n = len(p.stages)
    p.schedule(list(range(n)), impl=impl)


def harris(io_storage: int = hp.HP_F32, inner_storage: int = hp.HP_F32, k: float = 0.04) -> hp.Pipeline:
    """Harris corner response of an RGB image: gray, Sobel gradients, products,
    3x3 box sums, det - k tr^2 (every stencil clamped on its own producer)."""
    p = hp.Pipeline([io_storage], [3])
    s = inner_storage
    g = p.add_stage(hp.HP_POINTWISE, [p.input(0)], 1, s, op=hp.HP_OP_GRAY, params=[1.0])
    ix = p.add_stage(hp.HP_STENCIL, [g], 1, s, rx=1, ry=1, wx=SOBEL_DIFF, wy=SOBEL_SMOOTH)
    iy = p.add_stage(hp.HP_STENCIL, [g], 1, s, rx=1, ry=1, wx=SOBEL_SMOOTH, wy=SOBEL_DIFF)
    ixx = p.add_stage(hp.HP_POINTWISE, [ix, ix], 1, s, op=hp.HP_OP_MUL)
    iyy = p.add_stage(hp.HP_POINTWISE, [iy, iy], 1, s, op=hp.HP_OP_MUL)
    ixy = p.add_stage(hp.HP_POINTWISE, [ix, iy], 1, s, op=hp.HP_OP_MUL)
    sxx = p.add_stage(hp.HP_STENCIL, [ixx], 1, s, rx=1, ry=1, wx=BOX3_SUM, wy=BOX3_SUM)
    syy = p.add_stage(hp.HP_STENCIL, [iyy], 1, s, rx=1, ry=1, wx=BOX3_SUM, wy=BOX3_SUM)
    sxy = p.add_stage(hp.HP_STENCIL, [ixy], 1, s, rx=1, ry=1, wx=BOX3_SUM, wy=BOX3_SUM)
    r = p.add_stage(hp.HP_POINTWISE, [sxx, syy, sxy], 1, io_storage, op=hp.HP_OP_HARRIS, params=[k])
    p.set_output(r)
    return p


def fused_schedule(p: hp.Pipeline, tile_w: int = 32, tile_h: int = 32, threads: int = 256, impl=None,
                   inline_pointwise: bool = False):
    """All stages in one kernel (optionally with point-wise producers inlined)."""
    n = len(p.stages)
    groups = []
    for i, st in enumerate(p.stages):
        inl = inline_pointwise and st["kind"] == hp.HP_POINTWISE and i != n - 1
        groups.append(hp.HP_INLINE if inl else 0)
    p.schedule(groups, tile_w=[tile_w], tile_h=[tile_h], threads=[threads],
               impl=[impl] if impl is not None else None)


def unsharp(storage: int = hp.HP_F32, amount: float = 1.5, channels: int = 3) -> hp.Pipeline:
    """Per channel: blur = 5x5 binomial (clamped); out = in + amount (in - blur)."""
    p = hp.Pipeline([storage], [channels])
    blur = p.add_stage(hp.HP_STENCIL, [p.input(0)], channels, storage, rx=2, ry=2, wx=BINOMIAL16, wy=BINOMIAL16)
    out = p.add_stage(hp.HP_POINTWISE, [p.input(0), blur], channels, storage, op=hp.HP_OP_UNSHARP, params=[amount])
    p.set_output(out)
    return p


def histeq() -> hp.Pipeline:
    """256-bin histogram -> CDF lookup table -> table lookup, on a u8 image."""
    p = hp.Pipeline([hp.HP_U8], [1])
    h = p.add_stage(hp.HP_HISTOGRAM, [p.input(0)], 1, hp.HP_U32)
    lut = p.add_stage(hp.HP_CDF_LUT, [h], 1, hp.HP_U8)
    out = p.add_stage(hp.HP_LUT_APPLY, [p.input(0), lut], 1, hp.HP_U8)
    p.set_output(out)
    return p


def local_laplacian(levels: int = 8, k_levels: int = 8, sigma_r: float = 0.1, alpha: float = 1.0,
                    beta: float = 1.0, out_storage: int = hp.HP_U16, fine_storage: int = hp.HP_F32,
                    fine_levels: int = 0):
    """Local Laplacian filter (Paris et al.; K discrete intensity levels) of a
    u16 RGB image.  The output is u16 (rounded from out * 65535), or with
    out_storage = HP_F32 the float result in [0, 1] units before quantisation.
    fine_storage / fine_levels: the stages of pyramid levels l < fine_levels
    (remapped and gray pyramid level, upsample, Laplacian, interpolated level,
    collapse step) are stored in fine_storage (HP_F16 / HP_BF16; the
    arithmetic stays f32); the coarser levels and the gray image stay f32.
    Returns (pipeline, stage-id map)."""
    J, K = levels, k_levels
    p = hp.Pipeline([hp.HP_U16], [3])
    ids = {}
    F = hp.HP_F32

    def st(l):
        return fine_storage if l < fine_levels else F

    gray = p.add_stage(hp.HP_POINTWISE, [p.input(0)], 1, F, op=hp.HP_OP_GRAY, params=[1.0 / 65535.0])
    G = [p.add_stage(hp.HP_POINTWISE, [gray], K + 1, st(0), op=hp.HP_OP_LL_REMAP, params=[sigma_r, alpha, beta, K])]
    for l in range(1, J):
        G.append(p.add_stage(hp.HP_DOWNSAMPLE2, [G[-1]], K + 1, st(l)))
    U, L, Lout = [], [], []
    for l in range(J - 1):
        U.append(p.add_stage(hp.HP_UPSAMPLE2, [G[l + 1], G[l]], K + 1, st(l)))
        L.append(p.add_stage(hp.HP_POINTWISE, [G[l], U[l]], K + 1, st(l), op=hp.HP_OP_SUB))
        Lout.append(p.add_stage(hp.HP_POINTWISE, [G[l], L[l]], 1, st(l), op=hp.HP_OP_LL_INTERP, params=[K]))
    R = [None] * J
    UR = [None] * (J - 1)
    R[J - 1] = p.add_stage(hp.HP_POINTWISE, [G[J - 1]], 1, st(J - 1), op=hp.HP_OP_SELECT, params=[K])
    for l in range(J - 2, -1, -1):
        UR[l] = p.add_stage(hp.HP_UPSAMPLE2, [R[l + 1], Lout[l]], 1, st(l))
        R[l] = p.add_stage(hp.HP_POINTWISE, [Lout[l], UR[l]], 1, st(l), op=hp.HP_OP_ADD)
    out_scale = 65535.0 if out_storage == hp.HP_U16 else 1.0
    out = p.add_stage(hp.HP_POINTWISE, [p.input(0), gray, R[0]], 3, out_storage, op=hp.HP_OP_LL_COLOUR,
                      params=[1.0 / 65535.0, out_scale])
    p.set_output(out)
    ids.update(gray=gray, G=G, U=U, L=L, Lout=Lout, R=R, UR=UR, out=out)
    return p, ids


def remap_pyramid_level1(k_levels: int = 8, sigma_r: float = 0.1, alpha: float = 1.0, beta: float = 1.0,
                         in_dtype: int = hp.HP_U16, scale: float = 1.0 / 65535.0,
                         storages=(hp.HP_F32, hp.HP_F32, hp.HP_F32)) -> hp.Pipeline:
    """Level 1 of the local-Laplacian remap pyramid on its own: gray of an RGB
    input, its K remaps and gray (K+1 channels), one downsample; gray and the
    remap inlined into the downsample group (the first group of the local
    Laplacian pipeline).  storages: (gray, remap, downsample)."""
    p = hp.Pipeline([in_dtype], [3])
    g = p.add_stage(hp.HP_POINTWISE, [p.input(0)], 1, storages[0], op=hp.HP_OP_GRAY, params=[scale])
    r = p.add_stage(hp.HP_POINTWISE, [g], k_levels + 1, storages[1], op=hp.HP_OP_LL_REMAP,
                    params=[sigma_r, alpha, beta, k_levels])
    d = p.add_stage(hp.HP_DOWNSAMPLE2, [r], k_levels + 1, storages[2])
    p.set_output(d)
    p.schedule([hp.HP_INLINE, hp.HP_INLINE, 0])
    return p


def local_laplacian_fused_schedule(p: hp.Pipeline, ids: dict, tile: int = 32, threads: int = 256, impl=None,
                                   down_tile: int = 0, level_tile: int = 0, rows: int = 0):
    """Per-level fusion: level 1 of the remapped pyramid from the input in one
    kernel (gray and remap inlined); one downsample kernel per coarser level;
    one kernel per level for Laplacian + interpolation + collapse step; the
    finest level fused with the colour reconstruction.  down_tile and
    level_tile = 0 take each kernel's default (the streaming kernels, with run
    lengths sized per level so that small levels still spread over the SMs);
    another value picks the tiled downsample / per-pixel level kernel.  rows
    sets the streaming kernels' coarse rows per run (0: their default).  tile
    sizes the groups under the generic interpreter."""
    J = len(ids["G"])
    n = len(p.stages)
    groups = [None] * n
    gid = 0
    groups[ids["gray"]] = hp.HP_INLINE
    groups[ids["G"][0]] = hp.HP_INLINE
    down_groups = []
    for l in range(1, J):
        groups[ids["G"][l]] = gid
        down_groups.append(gid)
        gid += 1
    groups[ids["R"][J - 1]] = hp.HP_INLINE
    for l in range(J - 2, -1, -1):
        for key in ("U", "L", "Lout", "UR", "R"):
            groups[ids[key][l]] = gid
        if l == 0:
            groups[ids["out"]] = gid
        gid += 1
    assert all(g is not None for g in groups)
    generic = impl == hp.HP_IMPL_GENERIC
    tiles = [tile if generic else (down_tile if g in down_groups else level_tile) for g in range(gid)]
    heights = [t if (generic or t) else rows for t in tiles]
    p.schedule(groups, tile_w=tiles, tile_h=heights, threads=[threads] * gid,
               impl=[impl] * gid if impl is not None else None)


def max_filter(radius: int = 4, channels: int = 3, storage: int = hp.HP_F32, io_storage: int = None) -> hp.Pipeline:
    """Max filter (Sec. 6 app list): per channel, the maximum over the
    (2 radius + 1)^2 window at clamped coordinates, as a horizontal and a
    vertical window-maximum stage (radius <= HP_MAX_RADIUS each)."""
    io = storage if io_storage is None else io_storage
    p = hp.Pipeline([io], [channels])
    h = p.add_stage(hp.HP_MAX_STENCIL, [p.input(0)], channels, storage, rx=radius, ry=0)
    v = p.add_stage(hp.HP_MAX_STENCIL, [h], channels, io, rx=0, ry=radius)
    p.set_output(v)
    return p


def interpolate(levels: int = 10) -> tuple:
    """Interpolate (Sec. 6 app list): fill the uncovered pixels of an RGBA f32
    image (alpha = coverage) from premultiplied pyramids:
    D_0 = premultiply(in), D_l = downsample(D_{l-1}); I_{J-1} = D_{J-1},
    I_l = D_l over upsample(I_{l+1}); out = I_0.rgb / I_0.a (0 where a = 0).
    Returns (pipeline, stage-id map)."""
    J = levels
    F = hp.HP_F32
    p = hp.Pipeline([F], [4])
    D = [p.add_stage(hp.HP_POINTWISE, [p.input(0)], 4, F, op=hp.HP_OP_PREMUL)]
    for _ in range(1, J):
        D.append(p.add_stage(hp.HP_DOWNSAMPLE2, [D[-1]], 4, F))
    I = [None] * J
    U = [None] * J
    I[J - 1] = D[J - 1]
    for l in range(J - 2, -1, -1):
        U[l] = p.add_stage(hp.HP_UPSAMPLE2, [I[l + 1], D[l]], 4, F)
        I[l] = p.add_stage(hp.HP_POINTWISE, [D[l], U[l]], 4, F, op=hp.HP_OP_OVER)
    out = p.add_stage(hp.HP_POINTWISE, [I[0]], 3, F, op=hp.HP_OP_UNPREMUL)
    p.set_output(out)
    return p, dict(D=D, U=U, I=I, out=out)


def interpolate_fused_schedule(p: hp.Pipeline, ids: dict, tile: int = 32, threads: int = 256, impl=None,
                               down_tile: int = 0, level_tile: int = 0):
    """Per level: the premultiplied image in its own kernel (read by the first
    downsample and the finest composite); one downsample kernel per coarser
    level (default: the streaming plane kernel); one kernel per level for the
    upsample and the composite, the finest one with the final division.
    down_tile / level_tile = 0 take each kernel's default (the streaming
    kernels with run lengths sized per level); tile sizes the premultiply and,
    under the generic interpreter, every group."""
    D, U, I, out = ids["D"], ids["U"], ids["I"], ids["out"]
    J = len(D)
    n = len(p.stages)
    groups = [None] * n
    groups[D[0]] = 0
    gid = 1
    down_groups = []
    for l in range(1, J):
        groups[D[l]] = gid
        down_groups.append(gid)
        gid += 1
    for l in range(J - 2, -1, -1):
        groups[U[l]] = gid
        groups[I[l]] = gid
        if l == 0:
            groups[out] = gid
        gid += 1
    if J == 1:   # no pyramid: the premultiply and the division
        groups[out] = gid
        gid += 1
    assert all(g is not None for g in groups)
    generic = impl == hp.HP_IMPL_GENERIC
    tiles = [tile if (generic or g == 0) else (down_tile if g in down_groups else level_tile) for g in range(gid)]
    p.schedule(groups, tile_w=tiles, tile_h=tiles, threads=[threads] * gid,
               impl=[impl] * gid if impl is not None else None)


def interpolate_finest() -> hp.Pipeline:
    """The finest group of the interpolate pipeline on its own: inputs D_0
    (the premultiplied RGBA image) and I_1 (4 channels at half size); upsample
    of I_1, composite, division by coverage, in one kernel."""
    F = hp.HP_F32
    p = hp.Pipeline([F, F], [4, 4])
    u0 = p.add_stage(hp.HP_UPSAMPLE2, [p.input(1), p.input(0)], 4, F)
    i0 = p.add_stage(hp.HP_POINTWISE, [p.input(0), u0], 4, F, op=hp.HP_OP_OVER)
    out = p.add_stage(hp.HP_POINTWISE, [i0], 3, F, op=hp.HP_OP_UNPREMUL)
    p.set_output(out)
    p.schedule([0, 0, 0])
    return p


def bilateral_grid(s: int = 8, r: float = 0.1) -> hp.Pipeline:
    """Bilateral grid (Sec. 6 app list): splat the clamped gray values into
    s x s pixel cells and range levels of size r, blur the grid with
    [1,4,6,4,1]/16 along the range levels, then x, then y, and slice it back
    (trilinear; value / weight).  Input and output: 1-channel f32."""
    F = hp.HP_F32
    gz = int(np.floor(1.0 / float(np.float32(r)) + 0.5)) + 1
    p = hp.Pipeline([F], [1])
    g = p.add_stage(hp.HP_GRID_SPLAT, [p.input(0)], 2 * gz, F, params=[s, r])
    bz = p.add_stage(hp.HP_POINTWISE, [g], 2 * gz, F, op=hp.HP_OP_ZBLUR, params=[gz])
    bx = p.add_stage(hp.HP_STENCIL, [bz], 2 * gz, F, rx=2, ry=0, wx=BINOMIAL16, wy=[1.0])
    by = p.add_stage(hp.HP_STENCIL, [bx], 2 * gz, F, rx=0, ry=2, wx=[1.0], wy=BINOMIAL16)
    out = p.add_stage(hp.HP_GRID_SLICE, [by, p.input(0)], 1, F, params=[s, r])
    p.set_output(out)
    return p


def bilateral_grid_fused_schedule(p: hp.Pipeline, tile: int = 0, threads: int = 256, impl=None):
    """Splat, the three blurs fused in one kernel (the streaming grid-blur
    kernel; tile = its grid rows per run, 0: sized to spread over the SMs;
    under the generic interpreter 16 x 16 tiles by default), slice."""
    t = tile or (16 if impl == hp.HP_IMPL_GENERIC else 0)
    p.schedule([0, 1, 1, 1, 2], tile_w=[0, t, 0], tile_h=[0, t, 0], threads=[0, threads, 0],
               impl=[hp.HP_IMPL_AUTO, impl, hp.HP_IMPL_AUTO] if impl is not None else None)


def bilateral_grid_slice_only(s: int = 8, r: float = 0.1) -> hp.Pipeline:
    """The slice of the bilateral grid on its own: inputs the blurred grid
    (2 GZ channels) and the image; one kernel."""
    F = hp.HP_F32
    gz = int(np.floor(1.0 / float(np.float32(r)) + 0.5)) + 1
    p = hp.Pipeline([F, F], [2 * gz, 1])
    p.set_output(p.add_stage(hp.HP_GRID_SLICE, [p.input(0), p.input(1)], 1, F, params=[s, r]))
    return p
