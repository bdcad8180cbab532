"""The allocation-free histogram-equalization entry point, through the C ABI.

Some callers cannot allocate device memory when they run (a framework that
owns all device memory, a loop that must not block on cudaMalloc); they call
hp_histeq_u8_noalloc, which takes its scratch from a fixed array in the
library's device image.  Its output must equal the pipeline entry point's,
bit for bit (the tolerance of every integer path here), on consecutive calls.
This file is collected last so a failure here never hides another test.
"""

import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
from paper_2012_07145_gb300 import hp, pipelines, synth

pytestmark = pytest.mark.gpu


def _u8_device(arr):
    return hp.padded_copy(torch.from_numpy(np.ascontiguousarray(arr)))


def test_noalloc_matches_pipeline_on_two_calls_in_a_row():
    __graft_entry__.build()
    stream = torch.cuda.current_stream().cuda_stream
    p = pipelines.histeq()
    for seed, (h, w) in [(1, (480, 640)), (2, (1080, 1920))]:
        img = synth.gray_u8_lowcontrast(h, w, seed=seed)
        x = _u8_device(img)
        ref = hp.padded_empty(1, h, w, torch.uint8)
        got = hp.padded_empty(1, h, w, torch.uint8)
        got.fill_(7)
        p.realize([hp.buffer_from_tensor(x, hp.HP_U8)], hp.buffer_from_tensor(ref, hp.HP_U8), stream)
        status = hp.lib().hp_histeq_u8_noalloc(ctypes.byref(hp.buffer_from_tensor(x, hp.HP_U8)),
                                               ctypes.byref(hp.buffer_from_tensor(got, hp.HP_U8)),
                                               ctypes.c_void_p(stream))
        assert status == hp.HP_OK, hp.lib().hp_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_rejects_images_beyond_the_counter_capacity():
    __graft_entry__.build()
    x = hp.padded_empty(1, 16, 16, torch.uint8)
    big = hp.buffer_from_tensor(x, hp.HP_U8)
    big.width, big.height = 1 << 17, 1 << 16          # 2^33 pixels: never touched, rejected first
    big.row_stride_bytes = 1 << 17
    status = hp.lib().hp_histeq_u8_noalloc(ctypes.byref(big), ctypes.byref(big), None)
    assert status == hp.HP_ERR_INVALID_ARG
    assert b"HP_NOALLOC_MAX_PIXELS" in hp.lib().hp_last_error()
