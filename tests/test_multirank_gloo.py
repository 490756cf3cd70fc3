"""The multi-rank path on CPU (gloo, world size 2): ranks take disjoint,
contiguous stream ranges of one seeded job, their first streams are the job's
streams at those indices (checked with the oracle), and the step time is the
maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PER_RANK = 1000
GENS = ["MRG32K3A", "LFSR113", "GM19", "GM61", "MT19937"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_1307_5869_gb300 import workloads as W
        first, n = W.shard_range(rank, world, PER_RANK)
        ranges = [None] * world
        dist.all_gather_object(ranges, (first, n))
        # this rank's first stream, from its own shard
        mine = {g: O.Streams(g, W.bulk_seed(0), first, 1).state(0).u32(8).tolist() for g in GENS}
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = torch.tensor([1.5 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            # rank r's first stream = stream r * PER_RANK of the whole job
            job = {g: [O.Streams(g, W.bulk_seed(0), 0, world * PER_RANK).state(r * PER_RANK).u32(8).tolist()
                       for r in range(world)] for g in GENS}
            q.put((ranges, got, job, float(t.item())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ranges, got, job, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ranges == [(0, PER_RANK), (PER_RANK, PER_RANK)]
    for g in GENS:
        assert [got[r][g] for r in range(2)] == job[g], g
    assert tmax == 2.5


def test_shard_range_covers_the_job():
    from paper_1307_5869_gb300 import workloads as W
    for world in (1, 2, 3, 8):
        spans = [W.shard_range(r, world, 7, first=5) for r in range(world)]
        assert spans[0][0] == 5
        for (a, n), (b, _) in zip(spans, spans[1:]):
            assert a + n == b
        assert sum(n for _, n in spans) == 7 * world
    with pytest.raises(ValueError):
        W.shard_range(2, 2, 7)
