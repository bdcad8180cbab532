"""The allocation-free histogram-equalization entry point, through the C ABI.

Some callers cannot allocate device memory when they run (a framework that
owns all device memory, a loop that must not block on cudaMalloc); they call
hp_histeq_u8_noalloc, which takes its scratch from a fixed array in the
library's device image.  Its output must equal the exact integer oracle bit
for bit (the tolerance of every integer path here) and the pipeline entry
point's output, on consecutive calls: full-width rows, a ragged width whose
rows end inside a 16-byte chunk (the byte-by-byte tail of the kernels), and an
in-place call (input and output the same buffer).  This file is collected
last so a failure here never hides another test.
"""

import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import histeq as ohe
from paper_2012_07145_gb300 import hp, pipelines, synth

pytestmark = pytest.mark.gpu


def _u8_device(arr):
    return hp.padded_copy(torch.from_numpy(np.ascontiguousarray(arr)))


def _noalloc(x, y, stream):
    return hp.lib().hp_histeq_u8_noalloc(ctypes.byref(hp.buffer_from_tensor(x, hp.HP_U8)),
                                         ctypes.byref(hp.buffer_from_tensor(y, hp.HP_U8)), ctypes.c_void_p(stream))


@pytest.mark.parametrize("sizes", [[(480, 640), (1080, 1920)], [(53, 37), (53, 37)], [(1, 1), (7, 100)]])
def test_noalloc_matches_oracle_and_pipeline_on_two_calls_in_a_row(sizes):
    __graft_entry__.build()
    stream = torch.cuda.current_stream().cuda_stream
    p = pipelines.histeq()
    for seed, (h, w) in enumerate(sizes):
        img = synth.gray_u8_lowcontrast(h, w, seed=seed + 1)
        x = _u8_device(img)
        ref = hp.padded_empty(1, h, w, torch.uint8)
        got = hp.padded_empty(1, h, w, torch.uint8)
        got.fill_(7)
        p.realize([hp.buffer_from_tensor(x, hp.HP_U8)], hp.buffer_from_tensor(ref, hp.HP_U8), stream)
        status = _noalloc(x, got, stream)
        assert status == hp.HP_OK, hp.lib().hp_last_error()
        torch.cuda.synchronize()
        expect = ohe.equalize(img[0])[2]
        assert np.array_equal(got.cpu().numpy()[0], expect)
        assert torch.equal(got, ref)


def test_noalloc_in_place_on_a_ragged_width():
    """Input and output the same buffer: every thread reads its 16-byte chunk
    (or its tail bytes) before it writes them, after the histogram is complete."""
    __graft_entry__.build()
    stream = torch.cuda.current_stream().cuda_stream
    for seed, (h, w) in enumerate([(53, 37), (300, 333)]):
        img = synth.gray_u8_lowcontrast(h, w, seed=seed + 11)
        x = _u8_device(img)
        assert _noalloc(x, x, stream) == hp.HP_OK, hp.lib().hp_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy()[0], ohe.equalize(img[0])[2])


def test_noalloc_rejects_images_beyond_the_counter_capacity():
    __graft_entry__.build()
    x = hp.padded_empty(1, 16, 16, torch.uint8)
    big = hp.buffer_from_tensor(x, hp.HP_U8)
    big.width, big.height = 1 << 17, 1 << 16          # 2^33 pixels: never touched, rejected first
    big.row_stride_bytes = 1 << 17
    status = hp.lib().hp_histeq_u8_noalloc(ctypes.byref(big), ctypes.byref(big), None)
    assert status == hp.HP_ERR_INVALID_ARG
    assert b"HP_NOALLOC_MAX_PIXELS" in hp.lib().hp_last_error()
