"""The continuous-batching serving loop (hp_server_*): every result in a mixed
stream equals the request's solo result; admission respects the HBM budget;
waits time out on the host without touching the GPU."""

import numpy as np
import pytest
import torch

import __graft_entry__
from paper_2012_07145_gb300 import hp, pipelines, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def _pinned(arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()


def _kinds():
    un = pipelines.unsharp()
    pipelines.fused_schedule(un, tile_w=64, tile_h=32)
    hr = pipelines.harris()
    pipelines.fused_schedule(hr, tile_w=120, tile_h=16, threads=128)
    he = pipelines.histeq()
    return {
        "unsharp": (un, lambda h, w, s: (synth.rgb_f32(h, w, seed=s), hp.HP_F32), (3, hp.HP_F32, torch.float32)),
        "harris": (hr, lambda h, w, s: (synth.rgb_f32(h, w, seed=s), hp.HP_F32), (1, hp.HP_F32, torch.float32)),
        "histeq": (he, lambda h, w, s: (synth.gray_u8_lowcontrast(h, w, seed=s), hp.HP_U8), (1, hp.HP_U8, torch.uint8)),
    }


def test_mixed_stream_results_equal_solo_results():
    kinds = _kinds()
    sizes = [(48, 64), (256, 256), (200, 320), (480, 640)]
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(40):
        name = ["unsharp", "harris", "histeq"][rng.integers(3)]
        h, w = sizes[rng.integers(len(sizes))]
        p, gen, (oc, odt, tdt) = kinds[name]
        arr, idt = gen(h, w, 100 + i)
        hin = _pinned(arr)
        hout = torch.zeros((oc, h, w), dtype=tdt).pin_memory()
        solo = torch.zeros((oc, h, w), dtype=tdt).pin_memory()
        p.realize_host([hp.buffer_from_tensor(hin, idt)], hp.buffer_from_tensor(solo, odt))
        reqs.append((p, hin, idt, hout, odt, solo))
    srv = hp.Server(hbm_budget_bytes=256 << 20, slots=4, max_batch=4)
    for p, hin, idt, hout, odt, _ in reqs[:6]:   # some shapes made resident ahead, the rest on first use
        srv.prepare(p, [hp.buffer_from_tensor(hin, idt)])
    tickets = [srv.submit(p, [hp.buffer_from_tensor(hin, idt)], hp.buffer_from_tensor(hout, odt))
               for p, hin, idt, hout, odt, _ in reqs]
    for t in tickets:
        st, lat = srv.wait(t, 60000)
        assert st == hp.HP_OK and lat > 0
    stats = srv.stats()
    srv.close()
    assert stats.completed == len(reqs) and stats.failed == 0
    assert stats.peak_bytes <= 256 << 20
    for p, hin, idt, hout, odt, solo in reqs:
        assert torch.equal(hout, solo)
    print(f"serving test: batched launches {stats.batched_launches}, p50 {stats.p50_us:.0f} us, "
          f"p99 {stats.p99_us:.0f} us")


def test_admission_waits_for_memory_and_oversized_requests_are_refused():
    p = pipelines.unsharp()
    pipelines.fused_schedule(p, tile_w=64, tile_h=32)
    h, w = 256, 256
    per_request = 2 * 3 * h * w * 4                          # input + output, f32 RGB
    budget = int(2.5 * per_request) + (1 << 20)
    srv = hp.Server(hbm_budget_bytes=budget, slots=8, max_batch=1)
    bufs = []
    for i in range(12):
        hin = _pinned(synth.rgb_f32(h, w, seed=i))
        hout = torch.zeros((3, h, w), dtype=torch.float32).pin_memory()
        bufs.append((hin, hout))
    tickets = [srv.submit(p, [hp.buffer_from_tensor(a, hp.HP_F32)], hp.buffer_from_tensor(b, hp.HP_F32))
               for a, b in bufs]
    for t in tickets:
        assert srv.wait(t, 60000)[0] == hp.HP_OK
    stats = srv.stats()
    assert stats.completed == 12 and stats.peak_bytes <= budget
    big_in = torch.zeros((3, 1024, 1024), dtype=torch.float32)
    big_out = torch.zeros((3, 1024, 1024), dtype=torch.float32)
    with pytest.raises(hp.HPError) as e:
        srv.submit(p, [hp.buffer_from_tensor(big_in, hp.HP_F32)], hp.buffer_from_tensor(big_out, hp.HP_F32))
    assert e.value.status == hp.HP_ERR_OOM
    srv.close()


def test_wait_times_out_on_the_host():
    p = pipelines.unsharp()
    pipelines.fused_schedule(p, tile_w=64, tile_h=32)
    # 2048x2048 RGB f32: 50 MB to copy in and out, milliseconds of work; a
    # zero timeout right after submit must come back at once with a timeout
    hin = _pinned(synth.rgb_f32(2048, 2048, seed=1))
    hout = torch.zeros((3, 2048, 2048), dtype=torch.float32).pin_memory()
    srv = hp.Server(hbm_budget_bytes=256 << 20, slots=1, max_batch=1)
    t = srv.submit(p, [hp.buffer_from_tensor(hin, hp.HP_F32)], hp.buffer_from_tensor(hout, hp.HP_F32))
    st, _ = srv.wait(t, 0)
    assert st == hp.HP_ERR_TIMEOUT
    st, _ = srv.wait(t, 60000)
    assert st == hp.HP_OK
    srv.close()


def _queue_then_serve(srv, p, reqs, device=False):
    """Submits every request at once (a slot of the server is busy with the
    first while the rest queue, so later admissions batch) and waits."""
    sub = srv.submit_device if device else srv.submit
    tickets = [sub(p, [hp.buffer_from_tensor(x, idt)], hp.buffer_from_tensor(y, odt)) for x, idt, y, odt in reqs]
    for t in tickets:
        st, _ = srv.wait(t, 60000)
        assert st == hp.HP_OK


@pytest.mark.parametrize("kind,h,w,sched", [
    ("harris", 96, 160, dict(tile_w=32, tile_h=16, threads=128)),                       # tiled kernel
    ("harris", 200, 333, dict(impl=hp.HP_IMPL_WAVE, tile_w=120, tile_h=14, threads=128)),   # streaming kernel
    ("histeq", 300, 500, None), ("histeq", 37, 53, None)])
def test_batched_harris_and_histeq_equal_solo(kind, h, w, sched):
    """Same-pipeline requests of one size served by one launch (the image as
    the batch index of the fused Harris and histogram-equalization kernels)
    give each request its solo result bit for bit."""
    if kind == "harris":
        p = pipelines.harris()
        pipelines.fused_schedule(p, **sched)
        gen, idt, oc, odt, tdt = (lambda s: synth.rgb_f32(h, w, seed=s)), hp.HP_F32, 1, hp.HP_F32, torch.float32
    else:
        p = pipelines.histeq()
        pipelines.fused_schedule(p)
        gen, idt, oc, odt, tdt = (lambda s: synth.gray_u8_lowcontrast(h, w, seed=s)), hp.HP_U8, 1, hp.HP_U8, torch.uint8
    reqs, solos = [], []
    for i in range(9):
        x = _pinned(gen(200 + i))
        y = torch.zeros((oc, h, w), dtype=tdt).pin_memory()
        solo = torch.zeros((oc, h, w), dtype=tdt).pin_memory()
        p.realize_host([hp.buffer_from_tensor(x, idt)], hp.buffer_from_tensor(solo, odt))
        reqs.append((x, idt, y, odt))
        solos.append(solo)
    srv = hp.Server(hbm_budget_bytes=512 << 20, slots=1, max_batch=4)
    _queue_then_serve(srv, p, reqs)
    stats = srv.stats()
    srv.close()
    assert stats.completed == 9 and stats.batched_launches >= 1
    for (_, _, y, _), solo in zip(reqs, solos):
        assert torch.equal(y, solo)


def test_resident_shapes_replay_as_graphs_and_device_requests_match():
    """A slot keeps a shape's staging resident, so its realize of that shape
    replays as a CUDA graph from the second request on; device-buffer requests
    (served in place alone, gathered when batched) give the host requests'
    results."""
    p = pipelines.unsharp()
    pipelines.fused_schedule(p, tile_w=64, tile_h=32)
    h, w = 128, 192
    srv = hp.Server(hbm_budget_bytes=256 << 20, slots=1, max_batch=1)
    outs = []
    for i in range(5):
        x = _pinned(synth.rgb_f32(h, w, seed=300 + i))
        y = torch.zeros((3, h, w), dtype=torch.float32).pin_memory()
        t = srv.submit(p, [hp.buffer_from_tensor(x, hp.HP_F32)], hp.buffer_from_tensor(y, hp.HP_F32))
        assert srv.wait(t, 60000)[0] == hp.HP_OK
        outs.append((x, y))
    stats = srv.stats()
    assert stats.graph_replays >= 2 and stats.resident_bytes > 0
    # device requests, alone and batched, against the host results
    dev = [(hp.padded_copy(x, "cuda"), hp.padded_empty(3, h, w, torch.float32, "cuda")) for x, _ in outs]
    for (xd, yd), (_, y) in zip(dev, outs):
        t = srv.submit_device(p, [hp.buffer_from_tensor(xd, hp.HP_F32)], hp.buffer_from_tensor(yd, hp.HP_F32))
        assert srv.wait(t, 60000)[0] == hp.HP_OK
        assert torch.equal(yd.cpu(), y)
    srv.close()
    srv = hp.Server(hbm_budget_bytes=256 << 20, slots=1, max_batch=4)
    for _, yd in dev:
        yd.zero_()
    _queue_then_serve(srv, p, [(xd, hp.HP_F32, yd, hp.HP_F32) for xd, yd in dev], device=True)
    stats = srv.stats()
    srv.close()
    assert stats.device_requests == 5 and stats.batched_launches >= 1
    for (_, yd), (_, y) in zip(dev, outs):
        assert torch.equal(yd.cpu(), y)
