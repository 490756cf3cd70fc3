"""Seeded synthetic workloads (sizes, seeds, request mixes).

This module holds no generator arithmetic: it only fixes the shapes and seeds
of the workloads that the tests and the benchmark feed to both the CUDA path
and the oracle.
"""
from __future__ import annotations

import numpy as np

GENERATORS = ["MT19937", "MRG32K3A", "LFSR113", "GM19", "GM29", "GM31", "GM55",
              "GM61", "GQ58_1", "GQ58_3", "GQ58_4"]

# Bulk fill: three generators, 2^20 block-split streams, 2^10 outputs per stream
# as u32 and then 2^10 more as f32 (2^30 + 2^30 outputs per generator).
BULK_GENERATORS = ["MT19937", "LFSR113", "GM61"]
BULK_STREAMS = 1 << 20
BULK_PER_STREAM = 1 << 10
BULK_SEED_BASE = 0x9E3779B97F4A7C15  # "seed from a 64-bit counter": base + repetition


def bulk_seed(rep: int = 0) -> int:
    return (BULK_SEED_BASE + rep) & 0xFFFFFFFFFFFFFFFF


def shard_range(rank: int, world: int, per_rank: int, first: int = 0):
    """Streams of one rank when a job is sharded by stream index: every rank
    uses the same seed and takes the contiguous range [first + rank * per_rank,
    first + (rank + 1) * per_rank), so the ranks' outputs together are the
    outputs of one job over world * per_rank streams (weak scaling)."""
    if not 0 <= rank < world or per_rank < 0:
        raise ValueError("rank must be in [0, world) and per_rank >= 0")
    return first + rank * per_rank, per_rank


# All eleven generators, 2^16 streams x 2^12 outputs, seed 12345.
TABLE_STREAMS = 1 << 16
TABLE_PER_STREAM = 1 << 12
TABLE_SEED = 12345

# One stream of MRG32K3A from the default state, 2^20 outputs.
SINGLE_LENGTH = 1 << 20

# Skip-ahead study (Table 3): per generator the largest n of the paper's rows
# (2^n values skipped per step); the subsequence is output 0 of 2^22 streams
# spaced 2^n apart (2^20 for MT19937, whose states are 2.5 KB), tested for
# frequency (2^10 cells), serial pairs (2^10 cells) and gaps (hit range
# [0, 2^29), p = 1/8, 49 cells).
STUDY_SKIPS = {"GM19": 21, "GM29": 24, "GM31": 24, "GM55": 60, "GM61": 75, "GQ58_1": 24, "GQ58_3": 24,
               "GQ58_4": 24, "LFSR113": 75, "MRG32K3A": 90, "MT19937": 440}
STUDY_WORDS = 1 << 22
STUDY_WORDS_MT = 1 << 20
STUDY_SEED = 20140401
STUDY_TESTS = (("frequency", dict(bits=10)), ("serial", dict(bits=5)), ("gap", dict(lo=0, hi=1 << 29, t=48)))


def batched_requests(n: int = 10_000, seed: int = 7, max_log2: int = 20):
    """Requests (gen, stream, length, dtype=u32): generator uniform over the
    eleven, stream index uniform in [0, 1e19), length floor(2^(max_log2 * U))
    clamped to [1, 2^max_log2]."""
    rng = np.random.default_rng(seed)
    gens = rng.integers(0, len(GENERATORS), size=n)
    streams = rng.integers(0, 10**19, size=n, dtype=np.uint64)
    lengths = np.clip(np.floor(2.0 ** (max_log2 * rng.random(n))), 1, 2**max_log2).astype(np.int64)
    return [(GENERATORS[int(g)], int(s), int(L), 0) for g, s, L in zip(gens, streams, lengths)]


def serving_arrivals(rate: float = 5e4, seconds: float = 10.0, seed: int = 11):
    """Poisson arrivals: (t_arrival_s, gen, stream, length, dtype) with length
    floor(2^(6 + 16 U)) in [2^6, 2^22] and dtype u32/f32/f64 equiprobable."""
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate * seconds)
    t = np.sort(rng.random(n) * seconds)
    gens = rng.integers(0, len(GENERATORS), size=n)
    streams = rng.integers(0, 10**19, size=n, dtype=np.uint64)
    lengths = np.floor(2.0 ** (6 + 16 * rng.random(n))).astype(np.int64)
    dtypes = rng.integers(0, 3, size=n)
    return [(float(a), GENERATORS[int(g)], int(s), int(L), int(d))
            for a, g, s, L, d in zip(t, gens, streams, lengths, dtypes)]
