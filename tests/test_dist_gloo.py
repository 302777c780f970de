"""The multi-rank host logic on CPU: two gloo ranks shard work, reduce times
with MAX and aggregate units with SUM, as bench.py does across GPUs."""
import os
import socket

import pytest

from paper_1611_06906_gb300 import dist as D


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = D.shard(n, r, world)
                assert 0 <= lo <= hi <= n
                seen += list(range(lo, hi))
            assert seen == list(range(n))
            sizes = [D.shard(n, r, world)[1] - D.shard(n, r, world)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = D.rank_info()
    lo, hi = D.shard(64, r, w)
    ms = 10.0 + 5.0 * r  # rank 1 is slower
    dist.barrier()
    q.put((r, lo, hi, D.max_over_ranks(ms), D.sum_over_ranks(hi - lo), D.rank_seed(3000, r)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1:3] == (0, 32) and out[1][1:3] == (32, 64)
    assert out[0][3] == out[1][3] == 15.0       # max of 10 and 15
    assert out[0][4] == out[1][4] == 64.0       # all units accounted for
    assert out[0][5] != out[1][5]               # each rank has its own images
