"""The oracle's spaced streams (Table 3's skip-ahead subsequences) and its
statistical-test cell counts, pinned to brute force, library routines and a
hand-worked example."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("gen", O.GENS)
def test_spaced_stream_is_the_decimated_sequence(gen):
    # output 0 of stream k of spacing 2^s is output k * 2^s of the base, by plain stepping
    s, n = 3, 12
    plain = O.State.spaced(gen, 99, s, 0).u32(n << s)
    dec = O.spaced_outputs(gen, 99, s, 0, n, 1)[:, 0]
    assert np.array_equal(dec, plain[:: 1 << s])
    # and a stream's first outputs continue from there
    two = O.spaced_outputs(gen, 99, s, 5, 2, 4)
    assert np.array_equal(two[0], plain[5 << s: (5 << s) + 4])
    assert np.array_equal(two[1], plain[6 << s: (6 << s) + 4])


@pytest.mark.parametrize("gen,s", [("MRG32K3A", 100), ("LFSR113", 150), ("GM61", 191), ("GM29", 64),
                                   ("MT19937", 300), ("MT19937", 447)])
def test_spaced_stream_composition(gen, s):
    # stream 2k of spacing 2^s is stream k of spacing 2^(s+1) (checked on outputs)
    if s + 1 + 64 > 512:
        s = 447
        a = O.State.spaced(gen, 7, s, 6).u32(8)
        b = O.State.spaced(gen, 7, s - 1, 12).u32(8)
    else:
        a = O.State.spaced(gen, 7, s + 1, 3).u32(8)
        b = O.State.spaced(gen, 7, s, 6).u32(8)
    assert np.array_equal(a, b)


def test_spaced_stream_range_limit():
    with pytest.raises(ValueError):
        O.State.spaced("MRG32K3A", 1, 449, 1)


def test_frequency_counts_match_bincount():
    u = np.random.default_rng(3).integers(0, 2**32, 10007, dtype=np.uint32)
    for b in (1, 4, 8, 12):
        ref = np.bincount((u >> np.uint32(32 - b)).astype(np.int64), minlength=1 << b)
        assert np.array_equal(O.freq_counts(u, b), ref.astype(np.uint64))


def test_serial_counts_match_bincount():
    u = np.random.default_rng(4).integers(0, 2**32, 10007, dtype=np.uint32)  # odd: last word unused
    for b in (1, 3, 6):
        a = (u[0:-1:2] >> np.uint32(32 - b)).astype(np.int64)
        c = (u[1::2] >> np.uint32(32 - b)).astype(np.int64)
        ref = np.bincount(a * (1 << b) + c, minlength=1 << (2 * b))
        assert np.array_equal(O.serial_counts(u, b), ref.astype(np.uint64))


def _golden_gap():
    d = {}
    with open(os.path.join(GOLDEN, "gap_test_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            d[k] = [int(x) for x in v]
    return d


def test_gap_counts_hand_worked_example():
    d = _golden_gap()
    u = np.array(d["words"], dtype=np.uint32)
    c = O.gap_counts(u, d["lo"][0], d["hi"][0], d["t"][0])
    assert c.tolist() == d["counts"]


def test_gap_counts_invariants():
    u = np.random.default_rng(5).integers(0, 2**32, 20000, dtype=np.uint32)
    lo, hi = 1 << 30, 3 << 30
    c = O.gap_counts(u, lo, hi, 10)
    assert int(c.sum()) == int(((u >= lo) & (u < hi)).sum())  # one gap per hit
    # the hit range may run to the top word: [0, 2^32) hits every word, so every gap is 0;
    # [2^32 - 1, 2^32) hits only the top word
    c = O.gap_counts(u, 0, 1 << 32, 3)
    assert c.tolist() == [u.size, 0, 0, 0]
    w = np.array([5, 0xFFFFFFFF, 7, 7, 0xFFFFFFFF], dtype=np.uint32)
    assert O.gap_counts(w, (1 << 32) - 1, 1 << 32, 3).tolist() == [0, 1, 1, 0]
    # hits exactly every m-th word: every gap but the first has length m - 1
    m = 4
    v = np.zeros(400, dtype=np.uint32)
    v[m - 1::m] = 150
    c = O.gap_counts(v, 100, 200, 8)
    assert c[m - 1] == 100 and c.sum() == 100


def test_chi2_closed_forms():
    # exact expectations: statistic 0, tail probability 1
    u = np.arange(1 << 12, dtype=np.uint64) << np.uint64(20)
    stat, p = O.chi2_test("frequency", u.size, O.freq_counts(u.astype(np.uint32), 4), bits=4)
    assert stat == 0.0 and p == 1.0
    # three cells (gap test with t = 2): two degrees of freedom, tail exp(-x / 2)
    counts = np.array([40, 25, 35], dtype=np.uint64)
    stat, p = O.chi2_test("gap", 0, counts, lo=0, hi=1 << 31, t=2)
    e = np.array([50.0, 25.0, 25.0])
    x = float(((counts - e) ** 2 / e).sum())
    assert stat == pytest.approx(x, rel=1e-15)
    assert p == pytest.approx(math.exp(-x / 2), rel=1e-12)
    # expectations of the gap cells sum to the number of gaps (geometric series)
    e = O.expected_counts("gap", 0, counts, lo=123, hi=98765432, t=17)
    assert e.sum() == pytest.approx(100.0, rel=1e-12)


def test_tests_reject_a_biased_sequence_and_accept_a_generator():
    # top bit cleared in every word: the frequency test fails outright
    u = np.random.default_rng(6).integers(0, 2**31, 1 << 16, dtype=np.uint32)
    _, p = O.chi2_test("frequency", u.size, O.freq_counts(u, 4), bits=4)
    assert p < 1e-10
    # every second word repeats the previous one: the serial test fails
    w = np.repeat(np.random.default_rng(7).integers(0, 2**32, 1 << 15, dtype=np.uint32), 2)
    _, p = O.chi2_test("serial", w.size, O.serial_counts(w, 3), bits=3)
    assert p < 1e-10
    # a decimated MRG32K3A subsequence passes all three (fixed seed: deterministic)
    d = O.spaced_outputs("MRG32K3A", 2024, 20, 0, 1 << 13, 1)[:, 0]
    for kind, counts, kw in (("frequency", O.freq_counts(d, 6), dict(bits=6)),
                             ("serial", O.serial_counts(d, 3), dict(bits=3)),
                             ("gap", O.gap_counts(d, 0, 1 << 30, 12), dict(lo=0, hi=1 << 30, t=12))):
        _, p = O.chi2_test(kind, d.size, counts, **kw)
        assert 1e-4 < p < 1 - 1e-4, (kind, p)


def test_gm19_skip_ahead_subsequence_period():
    # GM19's period is p^2 - 1 = 2^20 (2^18 - 1) (Table 2, p = 2^19 - 1), so the
    # subsequence that skips 2^21 values per step repeats after 2^18 - 1 values
    p = (1 << 19) - 1
    assert p * p - 1 == (1 << 20) * ((1 << 18) - 1)
    a = O.spaced_outputs("GM19", 5, 21, 0, 4, 1)[:, 0]
    b = O.spaced_outputs("GM19", 5, 21, (1 << 18) - 1, 4, 1)[:, 0]
    c = O.spaced_outputs("GM19", 5, 21, 1 << 17, 4, 1)[:, 0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)
