"""FP16 / BF16 storage with FP32 arithmetic, per pipeline: every stage value is
rounded to the 16-bit type wherever it is stored, so the result is still
bit-identical across schedules (checked), and its error against the FP64
oracle is stated twice (printed as a LOWP line, recorded in the design notes):

  rounded_input  -- the oracle fed the same 16-bit-rounded input, so the error
                    is the one the 16-bit intermediates add;
  original_input -- the oracle fed the original FP32 input, so the error also
                    holds the rounding of the input itself.

Both are max |gpu - oracle| / (max - min of the oracle output).  They are
stated, not gated: the assertions are sanity bounds only.  The local
Laplacian keeps its coarse pyramid levels (and gray) in FP32 and stores only
the finest levels in 16 bits; its u16 input is exact in either case.
"""

import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import harris as ohr
from oracle import local_laplacian as oll
from oracle import stencil as ost
from oracle import unsharp as ous
from paper_2012_07145_gb300 import hp, pipelines, synth

from gpu_util import bits, rel_err, run, to_device, to_numpy

pytestmark = pytest.mark.gpu
NAMES = {hp.HP_F16: "f16", hp.HP_BF16: "bf16"}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def _rounded(img, dt):
    return to_numpy(to_device(img, dt)).astype(np.float64)


def _state(name, dt, e1, e2):
    print(f"LOWP {name} {NAMES[dt]} rounded_input={e1:.3e} original_input={e2:.3e}")


@pytest.mark.parametrize("dt", [hp.HP_F16, hp.HP_BF16])
def test_chain32_16bit(dt):
    H, W = 192, 320
    img = synth.stencil_input(H, W, seed=2)
    p = pipelines.stencil_chain(32, "alternate", storage=dt)
    plain = run(p, [to_device(img, dt)], [dt], (1, H, W), dt)
    for kw in (dict(depth=4, tile_w=64, tile_h=64, threads=256, serial_y=8),
               dict(depth=4, tile_w=112, tile_h=0, threads=128, impl=hp.HP_IMPL_WAVE)):
        pipelines.chain_schedule(p, **kw)
        assert torch.equal(bits(run(p, [to_device(img, dt)], [dt], (1, H, W), dt)), bits(plain)), kw
    kinds = ost.chain_kinds(32, "alternate")
    got = to_numpy(plain)[0]
    e1 = rel_err(got, ost.stencil_chain(_rounded(img, dt)[0], kinds))
    e2 = rel_err(got, ost.stencil_chain(img[0].astype(np.float64), kinds))
    _state("stencil_chain_32", dt, e1, e2)
    assert np.isfinite(e1) and e1 < (0.3 if dt == hp.HP_BF16 else 0.05)


@pytest.mark.parametrize("dt", [hp.HP_F16, hp.HP_BF16])
def test_harris_16bit(dt):
    H, W = 192, 320
    img = synth.rgb_f32(H, W, seed=4)
    p = pipelines.harris(io_storage=dt, inner_storage=dt)
    x = to_device(img, dt)
    plain = run(p, [x], [dt], (1, H, W), dt)
    for kw in (dict(), dict(impl=hp.HP_IMPL_WAVE, tile_w=112, tile_h=14, threads=128)):
        pipelines.fused_schedule(p, **kw)
        assert torch.equal(bits(run(p, [x], [dt], (1, H, W), dt)), bits(plain)), kw
    got = to_numpy(plain)[0]
    e1 = rel_err(got, ohr.harris(_rounded(img, dt)))
    e2 = rel_err(got, ohr.harris(img.astype(np.float64)))
    _state("harris", dt, e1, e2)
    assert np.isfinite(e1) and e1 < 0.1


@pytest.mark.parametrize("dt", [hp.HP_F16, hp.HP_BF16])
def test_unsharp_16bit(dt):
    H, W = 192, 320
    img = synth.rgb_f32(H, W, seed=5)
    p = pipelines.unsharp(storage=dt)
    x = to_device(img, dt)
    plain = run(p, [x], [dt], (3, H, W), dt)
    for kw in (dict(tile_w=64, tile_h=16, threads=128), dict(impl=hp.HP_IMPL_WAVE, tile_w=112, tile_h=16, threads=128)):
        pipelines.fused_schedule(p, **kw)
        assert torch.equal(bits(run(p, [x], [dt], (3, H, W), dt)), bits(plain)), kw
    got = to_numpy(plain)
    r1, r2 = ous.unsharp(_rounded(img, dt)), ous.unsharp(img.astype(np.float64))
    e1 = max(rel_err(got[c], r1[c]) for c in range(3))
    e2 = max(rel_err(got[c], r2[c]) for c in range(3))
    _state("unsharp", dt, e1, e2)
    assert np.isfinite(e1) and e1 < 0.05


@pytest.mark.parametrize("dt", [hp.HP_F16, hp.HP_BF16])
def test_local_laplacian_16bit_fine_levels(dt):
    """Levels 0 and 1 (the two largest) in 16 bits, levels 2.. in f32; alpha =
    0.5 (detail enhancement) so that the filter does real work."""
    H, W, J = 192, 320, 6
    img = synth.rgb_u16_gradient_noise(H, W, seed=1)
    ref = oll.local_laplacian_float(img, levels=J, k_levels=8, sigma_r=0.1, alpha=0.5, beta=1.0)
    p, ids = pipelines.local_laplacian(levels=J, k_levels=8, sigma_r=0.1, alpha=0.5, beta=1.0,
                                       out_storage=hp.HP_F32, fine_storage=dt, fine_levels=2)
    x = to_device(img, hp.HP_U16)
    plain = run(p, [x], [hp.HP_U16], (3, H, W), hp.HP_F32)
    pipelines.local_laplacian_fused_schedule(p, ids)
    assert torch.equal(bits(run(p, [x], [hp.HP_U16], (3, H, W), hp.HP_F32)), bits(plain))
    got = to_numpy(plain)
    e = max(rel_err(got[c], ref[c]) for c in range(3))
    _state("local_laplacian_fine2", dt, e, e)          # the u16 input is exact in both cases
    assert np.isfinite(e) and e < 0.05
