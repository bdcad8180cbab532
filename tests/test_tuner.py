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
    cands = tuner.chain_candidates(32, W, H)
    assert len(cands) > 100
    p = pipelines.stencil_chain(32)
    for c in cands:
        assert tuner.chain_smem_bytes(c["depth"], c["tile_w"], c["tile_h"]) <= tuner.SMEM_LIMIT
        blocks = -(-W // c["tile_w"]) * -(-H // c["tile_h"])
        assert blocks >= 2 * tuner.SMS or (c["tile_w"] <= 32 and c["tile_h"] <= 16)
        assert (c["tile_w"] // 4) * -(-c["tile_h"] // c["serial_y"]) >= c["threads"] // 2
        pipelines.chain_schedule(p, **c)
        assert p.group_count() == 32 // c["depth"]
        info = p.group_info([(W, H)], 0)
        assert info.kernel == hp.HP_KERNEL_STENCIL_CHAIN, c
        assert (info.tile_w, info.tile_h, info.threads) == (c["tile_w"], c["tile_h"], c["threads"])
        assert info.smem_bytes == tuner.chain_smem_bytes(c["depth"], c["tile_w"], c["tile_h"]), c
        assert info.grid_x * info.grid_y == -(-W // c["tile_w"]) * -(-H // c["tile_h"])


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
        return hp.HP_KERNEL_HARRIS_ROWS if app.startswith("harris") else hp.HP_KERNEL_STENCIL_ROWS
    return hp.HP_KERNEL_HARRIS if app.startswith("harris") else hp.HP_KERNEL_UNSHARP


def _app_pipeline(app):
    if app == "harris":
        return pipelines.harris()
    if app == "harris_bf16":
        return pipelines.harris(io_storage=hp.HP_BF16, inner_storage=hp.HP_BF16)
    if app == "unsharp":
        return pipelines.unsharp()
    return pipelines.histeq()


@pytest.mark.parametrize("app", ["harris", "harris_bf16", "unsharp", "histeq"])
def test_app_candidates_lower_to_the_kernel_they_time(app):
    p = _app_pipeline(app)
    n = len(p.stages)
    for c in tuner.app_candidates(app):
        tuner.apply_schedule(p, c)
        want = _expected_app_kernel(app, c)
        if want is None:
            assert p.group_count() == n            # every stage its own kernel
            continue
        assert p.group_count() == 1
        info = p.group_info([(2560, 1536)], 0)
        assert info.kernel == want, (app, c)


def test_every_stored_schedule_lowers_to_its_kernel():
    db = json.load(open(tuner.DB_PATH))
    assert "chain32" in db
    for name, entry in db.items():
        c = entry["params"]
        if name == "chain32":
            p = pipelines.stencil_chain(32)
            pipelines.chain_schedule(p, **c)
            assert p.group_info([(2560, 1536)], 0).kernel == hp.HP_KERNEL_STENCIL_CHAIN
            assert entry["ms"] < entry["plain_ms"]
            continue
        app, size = name.rsplit("_", 1)
        W, H = (int(v) for v in size.split("x"))
        p = _app_pipeline(app)
        tuner.apply_schedule(p, c)
        want = _expected_app_kernel(app, c)
        got = [p.group_info([(W, H)], g).kernel for g in range(p.group_count())]
        assert got == ([want] if want is not None else got), (name, got)
        if entry.get("plain_ms") is not None:
            assert entry["ms"] <= entry["plain_ms"], name
