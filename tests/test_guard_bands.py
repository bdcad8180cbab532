"""CPU check of the GPU tests' output guard bands (gpu_util.guarded_empty and
outside_writes): a write inside the image is allowed, one byte past a row, in
the guard row of a plane, or before or after the image is found."""

import torch

from paper_2012_07145_gb300 import hp

from gpu_util import CANARY, guarded_empty, outside_writes


def test_guard_bands_find_writes_outside_the_image_only():
    for dtype, val in ((hp.HP_F32, 1.5), (hp.HP_U8, 7), (hp.HP_BF16, 2.0)):
        out = guarded_empty(3, 5, 13, dtype, device="cpu")
        es = out.element_size()
        assert out.stride(1) * es % 16 == 0 and out.stride(0) * es % 16 == 0
        assert out.data_ptr() % 16 == 0 or out.storage_offset() * es % 16 == 0
        out.fill_(val)                                   # every pixel of the image
        assert outside_writes(out) == 0
        raw = out.guard[0]
        base = raw.data_ptr()
        img0 = out.data_ptr() - base                     # byte offset of pixel (0, 0, 0)
        rs, ps = out.stride(1) * es, out.stride(0) * es
        probes = [img0 - 1,                              # just before the image
                  img0 + 13 * es,                        # just past row 0
                  img0 + 4 * rs + 13 * es,               # past the last row of plane 0
                  img0 + 5 * rs,                         # the guard row of plane 0
                  img0 + 2 * ps + 5 * rs,                # the guard row of the last plane
                  raw.numel() - 1]                       # the last guard byte
        for off in probes:
            raw[off] = CANARY ^ 0xFF
            assert outside_writes(out) == 1, off
            raw[off] = CANARY
        assert outside_writes(out) == 0
