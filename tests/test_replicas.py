"""Host-side logic of the replica (N > 1) path on CPU with gloo, world size 2:
work sharding, the max-over-ranks timing reduction, the whole-job rate, and a
rank that fails before the collective (the others get an error, no hang)."""

import multiprocessing as mp
import socket
import traceback

import pytest

from paper_2012_07145_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_covers_every_item_once():
    for n in (0, 1, 7, 300):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in replicas.shard(n, r, world))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        replicas.shard(5, 2, 2)


def test_job_rate():
    assert replicas.job_rate(3.93, 4, 0.002) == pytest.approx(3.93 * 4 / 0.002)


def _worker_max(rank, world, port, q):
    try:
        replicas.init_gloo(rank, world, port)
        m = replicas.max_over_ranks(1.5 if rank == 0 else 4.25)
        q.put((rank, m))
        import torch.distributed as dist
        dist.destroy_process_group()
    except Exception:
        q.put((rank, traceback.format_exc()))


def test_max_over_ranks_with_gloo_world_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_max, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: 4.25, 1: 4.25}


def _worker_fail(rank, world, port, q):
    try:
        replicas.init_gloo(rank, world, port, timeout_s=5.0)
        if rank == 1:
            raise RuntimeError("rank 1 fails before the timing reduction")
        replicas.max_over_ranks(1.0)
        q.put((rank, "no error"))
    except Exception as e:
        q.put((rank, type(e).__name__))


def test_a_failing_rank_ends_the_others_collective_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "RuntimeError"
    assert res[0] != "no error"   # rank 0's reduction fails (peer gone / timeout) instead of hanging
