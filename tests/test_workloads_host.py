"""The seeded synthetic workloads follow their stated recipes: the request mix
of the batched launch (10^4 requests, generator uniform over the eleven,
stream index uniform in [0, 10^19), length floor(2^(20 U)) in [1, 2^20]) and
the Poisson arrivals of the server (5e4 requests/s for 10 s, length
floor(2^(6 + 16 U)) in [2^6, 2^22], dtype u32/f32/f64 equiprobable).  Means
are checked against the closed form of the log-uniform length,
E[2^(a + b U)] = 2^a (2^b - 1) / (b ln 2), within a few standard errors."""
import math

import numpy as np

from paper_1307_5869_gb300 import workloads as W


def _loguniform_mean(a: int, b: int) -> float:
    return 2.0 ** a * (2.0 ** b - 1) / (b * math.log(2))


def _loguniform_sd(a: int, b: int) -> float:
    m2 = 4.0 ** a * (4.0 ** b - 1) / (2 * b * math.log(2))
    return math.sqrt(m2 - _loguniform_mean(a, b) ** 2)


def test_batched_requests_recipe():
    reqs = W.batched_requests()
    assert reqs == W.batched_requests()  # seeded
    assert len(reqs) == 10_000
    gens = [g for g, _, _, _ in reqs]
    streams = np.array([k for _, k, _, _ in reqs], dtype=np.uint64)
    lengths = np.array([n for _, _, n, _ in reqs], dtype=np.float64)
    assert set(gens) == set(W.GENERATORS)
    assert all(d == 0 for _, _, _, d in reqs)
    assert streams.max() < 10**19 and streams.max() > 9 * 10**18 and streams.min() < 10**18
    assert lengths.min() >= 1 and lengths.max() <= 2**20
    # floor() lowers each length by about 1/2 on average
    mean, se = _loguniform_mean(0, 20) - 0.5, _loguniform_sd(0, 20) / math.sqrt(len(reqs))
    assert abs(lengths.mean() - mean) < 5 * se, (lengths.mean(), mean)
    assert 7.0e8 < lengths.sum() < 8.2e8  # about 7.6e8 outputs in all
    counts = np.bincount([W.GENERATORS.index(g) for g in gens], minlength=11)
    exp = len(reqs) / 11
    assert np.all(np.abs(counts - exp) < 5 * math.sqrt(exp))


def test_serving_arrivals_recipe():
    arr = W.serving_arrivals()
    n = len(arr)
    assert abs(n - 5e5) < 5 * math.sqrt(5e5)  # Poisson(rate * seconds)
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] < 10.0
    lengths = np.array([a[3] for a in arr], dtype=np.float64)
    assert lengths.min() >= 2**6 and lengths.max() <= 2**22
    mean, se = _loguniform_mean(6, 16) - 0.5, _loguniform_sd(6, 16) / math.sqrt(n)
    assert abs(lengths.mean() - mean) < 5 * se, (lengths.mean(), mean)
    dtypes = np.bincount([a[4] for a in arr], minlength=3)
    assert dtypes.size == 3 and np.all(np.abs(dtypes - n / 3) < 5 * math.sqrt(n / 3))
    streams = np.array([a[2] for a in arr], dtype=np.uint64)
    assert streams.max() < 10**19
    # demand: about 1.9e10 samples/s over the 10 s
    assert 1.8e10 < lengths.sum() / 10.0 < 2.0e10


def test_bulk_seed_is_a_64_bit_counter():
    assert W.bulk_seed(0) == 0x9E3779B97F4A7C15
    assert W.bulk_seed(5) == 0x9E3779B97F4A7C15 + 5
    assert W.bulk_seed(2**64 - 0x9E3779B97F4A7C15) == 0  # wraps modulo 2^64
