"""The multi-rank path on CPU: two gloo ranks get disjoint counter-event ranges and agree on
the max-over-ranks timing; the split of an integral on segment boundaries covers it once."""
import os

import pytest
import torch.multiprocessing as mp

from paper_1711_05683_b300 import shard


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off = shard.rank_event_offset(rank, 1000)
    t = shard.max_over_ranks(10.0 + rank)
    import torch
    offs = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(offs, torch.tensor([off]))
    q.put((rank, t, [int(o.item()) for o in offs]))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, offs in out:
        assert t == 11.0
        assert offs == [0, 1000]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_rank_slices_cover_once(world):
    total, q = 10 * 2 ** 21 + 12345, 2 ** 21
    covered = []
    for r in range(world):
        lo, hi = shard.rank_slice(r, world, total, q)
        assert lo % q == 0
        covered.append((lo, hi))
    assert covered[0][0] == 0 and covered[-1][1] == total
    for (a, b), (c, d) in zip(covered, covered[1:]):
        assert b == c


def test_single_process_max_is_identity():
    assert shard.max_over_ranks(3.5) == 3.5
