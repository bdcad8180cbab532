"""The pipelined host-buffer entry point (hp_realize_host_async / _wait): a
stream of images copied in, realized and copied back with the copies of one
image overlapping the realize of the next gives, image by image, the bits of
the synchronous hp_realize_host, over two rounds through the same buffers
(the two staging sets alternate) and with CUDA-graph replay."""

import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import stencil as ost
from paper_2012_07145_gb300 import hp, pipelines, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("kind,h,w,graph", [("chain", 300, 517, False), ("chain", 300, 517, True),
                                            ("unsharp", 97, 131, True), ("chain", 1, 1, False)])
def test_async_stream_equals_synchronous_calls(kind, h, w, graph):
    if kind == "chain":
        p = pipelines.stencil_chain(8, "alternate")
        pipelines.chain_schedule(p, depth=4, tile_w=64, tile_h=64)
        imgs = [synth.stencil_input(h, w, seed=s) for s in range(5)]
        oc = 1
    else:
        p = pipelines.unsharp()
        pipelines.fused_schedule(p)
        imgs = [synth.rgb_f32(h, w, seed=s) for s in range(5)]
        oc = 3
    p.use_cuda_graph(graph)
    s = torch.cuda.current_stream().cuda_stream
    hin = [_pinned(a) for a in imgs]
    ref = []
    for t in hin:
        o = torch.empty((oc, h, w), dtype=torch.float32).pin_memory()
        p.realize_host([hp.buffer_from_tensor(t, hp.HP_F32)], hp.buffer_from_tensor(o, hp.HP_F32), s)
        ref.append(o.clone())
    for rnd in range(2):
        hout = [torch.full((oc, h, w), float("nan")).pin_memory() for _ in hin]
        for t, o in zip(hin, hout):
            p.realize_host_async([hp.buffer_from_tensor(t, hp.HP_F32)], hp.buffer_from_tensor(o, hp.HP_F32), s)
        p.realize_host_wait()
        assert p.device_error() == 0
        for o, r in zip(hout, ref):
            assert torch.equal(o.view(torch.int32), r.view(torch.int32)), rnd
    if kind == "chain" and h * w > 1:
        got = ref[0].numpy()[0].astype(np.float64)
        want = ost.stencil_chain(imgs[0][0].astype(np.float64), ost.chain_kinds(8, "alternate"))
        assert np.abs(got - want).max() / (want.max() - want.min()) <= 1e-5
    p.realize_host_wait()   # nothing in flight: returns at once
