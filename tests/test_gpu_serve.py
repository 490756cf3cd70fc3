"""GPU parity of the request server: every request returns the next outputs of
its stream (continuing across requests), bit for bit against the oracle, alone
and in a mix of concurrent requests, including streams whose state was moved
to host memory and back."""
import time

import numpy as np
import pytest

import oracle as O
import paper_1307_5869_gb300 as P

pytestmark = pytest.mark.gpu

BITS = {0: np.uint32, 1: np.uint32, 2: np.uint64}
NP = {0: np.int32, 1: np.float32, 2: np.float64}
DT = {0: "u32", 1: "f32", 2: "f64"}


def _fetch(srv, rid, n, dtype, timeout=120.0):
    t0 = time.time()
    while not P.prand_server_query(srv, rid)[0]:
        assert time.time() - t0 < timeout, "request did not complete"
        time.sleep(0.001)
    out = np.empty(n, dtype=NP[dtype])
    P.prand_server_read(srv, rid, out)
    P.prand_server_release(srv, rid)
    return out


def _run(reqs, slots, seed=5150):
    srv = P.prand_server_create(seed, 256 << 20, slots)
    try:
        ids = [P.prand_server_submit(srv, g, k, n, d) for g, k, n, d in reqs]
        outs = [_fetch(srv, i, n, d) for i, (g, k, n, d) in zip(ids, reqs)]
        stats = P.prand_server_stats(srv)
    finally:
        P.prand_server_destroy(srv)
    return outs, stats


def _expected(reqs, seed=5150):
    states, out = {}, []
    for g, k, n, d in reqs:
        st = states.setdefault((g, k), O.State.stream(g, seed, k))
        out.append(getattr(st, DT[d])(n))
    return out


def _mix(seed, count, streams_per_gen=3):
    rng = np.random.default_rng(seed)
    keys = [(g, int(rng.integers(0, 10**19, dtype=np.uint64))) for g in P.GENERATORS for _ in range(streams_per_gen)]
    reqs = []
    for _ in range(count):
        g, k = keys[int(rng.integers(0, len(keys)))]
        n = int(2 ** (6 + 10 * rng.random()))
        reqs.append((g, k, n, int(rng.integers(0, 3))))
    return reqs


def test_server_continues_streams_bit_exact():
    reqs = _mix(1, 150)
    outs, stats = _run(reqs, slots=64)
    for (g, k, n, d), got, want in zip(reqs, outs, _expected(reqs)):
        assert np.array_equal(got.view(BITS[d]), want.view(BITS[d])), (g, k, n, d)
    assert stats["completed"] == len(reqs) and stats["hits"] > 0


def test_server_spill_and_restore_bit_exact():
    # two slots per generator for three streams each: states move to host and back
    reqs = _mix(2, 120)
    outs, stats = _run(reqs, slots=2)
    for (g, k, n, d), got, want in zip(reqs, outs, _expected(reqs)):
        assert np.array_equal(got.view(BITS[d]), want.view(BITS[d])), (g, k, n, d)
    assert stats["spills"] > 0 and stats["restores"] > 0


def test_server_alone_equals_in_the_mix():
    reqs = _mix(3, 60, streams_per_gen=2)
    mixed, _ = _run(reqs, slots=64)
    seen = set()
    for i, (g, k, n, d) in enumerate(reqs):
        if (g, k) in seen:
            continue
        seen.add((g, k))
        alone, _ = _run([(g, k, n, d)], slots=4)
        assert np.array_equal(alone[0].view(BITS[d]), mixed[i].view(BITS[d])), (g, k)


def test_server_long_mt19937_requests_bit_exact():
    # Long MT19937 requests (hundreds of 624-word blocks, generated by the
    # tile's whole team of warps) and the short requests that continue their
    # streams from the state they leave; ragged and whole last blocks, all
    # dtypes, and stream 0 (no digits of the stream index at all).
    rng = np.random.default_rng(12)
    k1, k2 = (int(x) for x in rng.integers(0, 10**19, size=2, dtype=np.uint64))
    reqs = [("MT19937", k1, (1 << 19) + 12345, 0),
            ("MT19937", k1, 1000, 1),
            ("MT19937", k2, 5 << 18, 2),
            ("MT19937", k2, 700, 0),
            ("MT19937", 0, (3 << 18) + 1, 1)]
    outs, _ = _run(reqs, slots=8)
    for (g, k, n, d), got, want in zip(reqs, outs, _expected(reqs)):
        assert np.array_equal(got.view(BITS[d]), want.view(BITS[d])), (g, k, n, d)


def test_server_replay_latencies():
    rng = np.random.default_rng(9)
    reqs = [(P.GENERATORS[i % 11], 0, int(rng.integers(0, 10**19, dtype=np.uint64)), 1024) for i in range(2000)]
    arrivals = list(np.sort(rng.random(2000) * 0.2))
    srv = P.prand_server_create(77, 512 << 20, 4096)
    try:
        lat, wall = P.prand_server_replay(srv, reqs, arrivals)
        st = P.prand_server_stats(srv)
    finally:
        P.prand_server_destroy(srv)
    assert st["completed"] == 2000 and all(x >= 0 for x in lat) and wall > 0
