"""The multi-rank host logic of the weak-scaling runs, on CPU with two gloo ranks.

Every rank owns a disjoint block of independent solves; the throughput of the job is
(units of all ranks) / (the slowest rank's time).  The ranks exchange only the timing
scalars (all-reduce max / sum), which is what these tests exercise.
"""
import os
import socket

import pytest

from paper_2308_11469_gb300 import dist as D

torch = pytest.importorskip("torch")


def test_shard_partitions_every_count():
    for ws in (1, 2, 3, 4, 8):
        for count in (0, 1, 2, 7, 8, 512, 513):
            owned = [list(D.shard(count, r, ws)) for r in range(ws)]
            flat = [i for blk in owned for i in blk]
            assert flat == list(range(count))                     # disjoint, ordered, complete
            sizes = [len(b) for b in owned]
            assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)
    with pytest.raises(ValueError):
        D.shard(4, 0, 0)


def test_single_process_identity():
    assert D.max_over_ranks(3.5) == 3.5
    assert D.throughput(4, 2.0) == 2.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        blk = D.shard(512, rank, ws)
        # rank r "takes" 1 + r seconds for its block; the job time is the slowest rank's
        secs = 1.0 + rank
        mx = D.max_over_ranks(secs, dist)
        tot = D.sum_over_ranks(len(blk), dist)
        thr = D.throughput(len(blk), secs, dist)
        gathered = [None] * ws
        dist.all_gather_object(gathered, list(blk))
        dist.barrier()
        q.put((rank, mx, tot, thr, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_protocol():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    ws = 2
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, tot, thr, gathered in out:
        assert mx == 2.0                                   # max over ranks, on every rank
        assert tot == 512.0
        assert thr == pytest.approx(512.0 / 2.0)
        assert sorted(i for blk in gathered for i in blk) == list(range(512))
