"""The autotuner's host logic, on the CPU: its candidate spaces lower through
the C ABI to the kernels they are meant to time, its mirror of the chain
kernel's shared-memory plan equals the library's, its pruning rules hold, and
every stored schedule still lowers to the kernel it was tuned on."""

import json

import pytest

import __graft_entry__
from paper_2012_07145_gb300 import hp, pipelines, tuner


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def test_chain_candidates_lower_with_the_mirrored_shared_memory():
    W, H = 2560, 1536
    cands = [c for c in tuner.chain_candidates(32, W, H)
             if c.get("impl") not in (hp.HP_IMPL_WAVE, hp.HP_IMPL_LINES)]   # the tiled ones
    assert len(cands) > 100
    p = pipelines.stencil_chain(32)
    for c in cands:
        assert tuner.chain_smem_bytes(c["depth"], c["tile_w"], c["tile_h"]) <= tuner.SMEM_LIMIT
        blocks = -(-W // c["tile_w"]) * -(-H // c["tile_h"])
        assert blocks >= tuner.SMS // 2 or (c["tile_w"] <= 32 and c["tile_h"] <= 16)
        assert (c["tile_w"] // 4) * -(-c["tile_h"] // c["serial_y"]) >= c["threads"] // 2
        pipelines.chain_schedule(p, **c)
        assert p.group_count() == 32 // c["depth"]
        info = p.group_info([(W, H)], 0)
        assert info.kernel == hp.HP_KERNEL_STENCIL_CHAIN, c
        assert (info.tile_w, info.tile_h, info.threads) == (c["tile_w"], c["tile_h"], c["threads"])
        assert info.smem_bytes == tuner.chain_smem_bytes(c["depth"], c["tile_w"], c["tile_h"]), c
        assert info.grid_x * info.grid_y == -(-W // c["tile_w"]) * -(-H // c["tile_h"])


def test_line_buffer_candidates_lower_to_the_line_buffer_kernel():
    for n, W, H in ((32, 2560, 1536), (4, 512, 512)):
        cands = [c for c in tuner.chain_candidates(n, W, H) if c.get("impl") == hp.HP_IMPL_LINES]
        assert len(cands) > 20
        p = pipelines.stencil_chain(n)
        for c in cands:
            pipelines.chain_schedule(p, **c)
            assert p.group_count() == -(-n // c["depth"])
            for g in range(p.group_count()):
                info = p.group_info([(W, H)], g)
                assert info.kernel == hp.HP_KERNEL_STENCIL_LINES, c
                assert (info.grid_x, info.grid_y) == (-(-W // c["tile_w"]), -(-H // c["tile_h"]))
                assert info.threads <= 256 and info.smem_bytes <= tuner.SMEM_LIMIT


def test_chain_candidates_prune_what_the_library_refuses():
    """A tile just past the shared-memory limit is not a candidate, and the
    library refuses it too (the mirror errs on neither side)."""
    p = pipelines.stencil_chain(32)
    refused = 0
    for d in (8, 16, 32):
        for tw, th in ((128, 128), (128, 64), (64, 128)):
            if tuner.chain_smem_bytes(d, tw, th) <= tuner.SMEM_LIMIT:
                continue
            pipelines.chain_schedule(p, d, tile_w=tw, tile_h=th)
            with pytest.raises(hp.HPError) as e:
                p.group_info([(2560, 1536)], 0)
            assert e.value.status == hp.HP_ERR_SCHEDULE
            refused += 1
    assert refused >= 3


def _expected_app_kernel(app, c):
    if c["schedule"] == "root":
        return None
    if app == "histeq":
        return hp.HP_KERNEL_HISTEQ
    if c.get("impl") == hp.HP_IMPL_GENERIC:
        return hp.HP_KERNEL_GENERIC
    if c.get("impl") == hp.HP_IMPL_WAVE:
        return hp.HP_KERNEL_HARRIS_ROWS if app == "harris" else hp.HP_KERNEL_STENCIL_ROWS
    return hp.HP_KERNEL_HARRIS if app == "harris" else hp.HP_KERNEL_UNSHARP


@pytest.mark.parametrize("app,dtype", [("harris", "f32"), ("harris", "bf16"), ("unsharp", "f32"), ("histeq", "u8")])
def test_app_candidates_lower_to_the_kernel_they_time(app, dtype):
    wl = tuner.workload(app, 2560, 1536, dtype)
    p, _ = wl["build"]()
    n = len(p.stages)
    for c in tuner.app_candidates(app, dtype):
        tuner.apply_schedule(p, c)
        want = _expected_app_kernel(app, c)
        if want is None:
            assert p.group_count() == n            # every stage its own kernel
            continue
        assert p.group_count() == 1
        info = p.group_info([(2560, 1536)], 0)
        assert info.kernel == want, (app, c)


@pytest.mark.parametrize("n,dtype", [(32, "f32"), (32, "bf16"), (4, "f32")])
def test_streaming_chain_candidates_lower_to_the_streaming_kernel(n, dtype):
    """The tuner's mirror of the streaming kernel's strip widths (4 or 8
    columns per lane, 2-byte inputs aligned to 8 columns) is the library's."""
    pattern = "alternate" if n == 32 else "binomial"
    W, H = (2560, 1536) if n == 32 else (512, 512)
    wl = tuner.workload(f"stencil_chain_{n}_{pattern}", W, H, dtype)
    p, _ = wl["build"]()
    stream = [c for c in wl["candidates"](False) if c.get("impl") == hp.HP_IMPL_WAVE]
    assert len(stream) >= 18
    for c in stream:
        wl["apply"](p, None, c)
        assert p.group_count() == n // c["depth"]
        assert p.group_info([(W, H)], 0).kernel == hp.HP_KERNEL_STENCIL_WAVE, c


def test_local_laplacian_candidates_lower():
    wl = tuner.workload("local_laplacian_J8_K8", 2560, 1536, "u16")
    p, ids = wl["build"]()
    for c in wl["candidates"](False):
        wl["apply"](p, ids, c)
        assert p.group_count() == 14
        kinds = [p.group_info([(2560, 1536)], g).kernel for g in range(p.group_count())]
        assert all(0 <= k < len(hp.KERNEL_NAMES) for k in kinds)


def test_keys_round_trip():
    for wl in tuner.BENCH_WORKLOADS:
        assert tuner.parse_key(tuner.key(*wl)) == wl


def test_every_stored_schedule_lowers():
    """Every entry of schedules.json is keyed by its workload, lowers through
    the C ABI at its size, and was faster than the stage-per-kernel schedule."""
    db = json.load(open(tuner.DB_PATH))
    assert tuner.key("stencil_chain_32_alternate", 2560, 1536, "f32") in db
    for k, entry in db.items():
        pipeline, w, h, dtype = tuner.parse_key(k)
        assert entry["workload"] == dict(pipeline=pipeline, w=w, h=h, dtype=dtype)
        wl = tuner.workload(pipeline, w, h, dtype)
        p, ids = wl["build"]()
        tuner.apply_entry(p, ids, pipeline, entry)
        kinds = [p.group_info([(w, h)], g).kernel for g in range(p.group_count())]
        assert all(0 <= x < len(hp.KERNEL_NAMES) for x in kinds), k
        if entry.get("plain_ms") is not None:
            assert entry["ms"] <= entry["plain_ms"], k
