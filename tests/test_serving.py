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
