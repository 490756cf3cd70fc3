"""Sharding by stream range: handles over the ranges that shard_range gives
ranks 0 and 1 reproduce, concatenated, one handle over the whole range (the
multi-GPU partition, run here as two handles on one GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1307_5869_gb300 as P  # noqa: E402
from paper_1307_5869_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("gen", ["MT19937", "MRG32K3A", "LFSR113", "GM61", "GQ58_3"])
def test_two_ranks_equal_one_handle(gen):
    P.load()
    per_rank, n_per, seed = 1536, 333, W.bulk_seed(0)
    whole = P.Generator(gen, seed, 0, 2 * per_rank)
    want = [whole.generate(n_per, "u32").cpu().numpy(), whole.generate(n_per, "f32").cpu().numpy()]
    parts = [[], []]
    for rank in range(2):
        first, n = W.shard_range(rank, 2, per_rank)
        g = P.Generator(gen, seed, first, n)
        parts[0].append(g.generate(n_per, "u32").cpu().numpy())
        parts[1].append(g.generate(n_per, "f32").cpu().numpy())
    for w, p in zip(want, parts):
        assert np.array_equal(w.view(np.uint32), np.concatenate(p).view(np.uint32))
