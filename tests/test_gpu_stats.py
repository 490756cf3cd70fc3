"""Spaced streams (the skip-ahead layout of Table 3) and the statistical-test
cell counts through the C ABI, against the oracle: outputs and counts bit for
bit, statistics and p-values to rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
import paper_1307_5869_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

CHUNK = 1 << 13  # words per gap chunk on the GPU


def _gen(h, n, m):
    t = torch.empty(n * m, dtype=torch.int32, device="cuda")
    P.prand_generate_u32(h, t.data_ptr(), m, 0)
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32).reshape(n, m)


SPACINGS = {g: (0, 5, 61, 127) for g in O.GENS}
SPACINGS["MT19937"] = (0, 5, 300, 448)


@pytest.mark.parametrize("gen", O.GENS)
def test_spaced_streams_follow_the_oracle(gen):
    P.load()
    seed, first, n, m = 31337, 3, 24, 5
    for sp in SPACINGS[gen]:
        h = P.prand_create(gen, seed)
        try:
            P.prand_init_streams_spaced(h, sp, first, n)
            got = _gen(h, n, m)
            more = _gen(h, n, 3)  # continuation
        finally:
            P.prand_destroy(h)
        ref = O.spaced_outputs(gen, seed, sp, first, n, m + 3)
        assert np.array_equal(got, ref[:, :m]), (gen, sp)
        assert np.array_equal(more, ref[:, m:]), (gen, sp)


def test_spaced_layout_errors_and_checkpoint():
    P.load()
    h = P.prand_create("MRG32K3A", 1)
    try:
        with pytest.raises(P.PrandError):
            P.prand_init_streams_spaced(h, 128, 0, 4)  # above 127 for MRG32K3A
        P.prand_init_streams_spaced(h, 90, 0, 4)
        blob = P.prand_get_state(h)
        a = _gen(h, 4, 16)
        P.prand_set_state(h, blob)
        b = _gen(h, 4, 16)
        assert np.array_equal(a, b)
    finally:
        P.prand_destroy(h)
    h = P.prand_create("MT19937", 1)
    try:
        with pytest.raises(P.PrandError):
            P.prand_init_streams_spaced(h, 449, 0, 2)
    finally:
        P.prand_destroy(h)


def _counts(test, words_dev, n):
    cells = P.prand_test_cells(test)
    c = torch.full((cells,), -1, dtype=torch.int64, device="cuda")
    P.prand_test_counts(test, words_dev, n, c.data_ptr(), 0)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64)


def _oracle_counts(test, u):
    if test.kind == P.TEST_FREQUENCY:
        return O.freq_counts(u, test.bits)
    if test.kind == P.TEST_SERIAL:
        return O.serial_counts(u, test.bits)
    return O.gap_counts(u, test.lo, test.hi, test.t)


TESTS = [P.make_test(P.TEST_FREQUENCY, bits=b) for b in (1, 4, 8, 12)] + \
    [P.make_test(P.TEST_SERIAL, bits=b) for b in (1, 3, 6)] + \
    [P.make_test(P.TEST_GAP, lo=lo, hi=hi, t=t) for lo, hi, t in
     ((0, 1 << 31, 8), (1 << 30, (1 << 30) + (1 << 28), 32), (0, 1 << 32, 1), (5, 6, 4), (0, 1 << 26, 1024),
      ((1 << 32) - 1000, 1 << 32, 7))]


@pytest.mark.parametrize("n", [0, 1, 7, 1000, CHUNK - 1, CHUNK, CHUNK + 1, 3 * CHUNK + 5, (1 << 20) + 3])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_counts_match_the_oracle(n, offset):
    P.load()
    rng = np.random.default_rng(n * 4 + offset)
    u = rng.integers(0, 2**32, n + offset, dtype=np.uint32)
    d = torch.from_numpy(u.view(np.int32)).cuda()
    ptr = d.data_ptr() + 4 * offset  # offsets 1 and 3 leave 16-byte alignment
    for test in TESTS:
        got = _counts(test, ptr, n)
        ref = _oracle_counts(test, u[offset:])
        assert np.array_equal(got, ref), (test.kind, test.bits, test.lo, test.hi, test.t, n, offset)


def test_gap_counts_across_chunk_boundaries():
    P.load()
    n = 6 * CHUNK + 11
    cases = {
        "none": [],
        "boundaries": [CHUNK - 1, CHUNK, 2 * CHUNK - 1, 4 * CHUNK, 6 * CHUNK + 10],
        "last chunk only": [6 * CHUNK + 3, 6 * CHUNK + 9],
        "long gaps": [17, 5 * CHUNK + 1],
        "every word": list(range(n)),
        "first only": [0],
    }
    test = P.make_test(P.TEST_GAP, lo=100, hi=200, t=1024)
    for name, hits in cases.items():
        u = np.full(n, 7, dtype=np.uint32)
        u[hits] = 150
        d = torch.from_numpy(u.view(np.int32)).cuda()
        got = _counts(test, d.data_ptr(), n)
        assert np.array_equal(got, O.gap_counts(u, 100, 200, 1024)), name


def test_evaluate_matches_the_oracle_and_scipy():
    P.load()
    u = np.random.default_rng(9).integers(0, 2**32, 1 << 16, dtype=np.uint32)
    d = torch.from_numpy(u.view(np.int32)).cuda()
    for test, kw in ((P.make_test(P.TEST_FREQUENCY, bits=6), dict(bits=6)),
                     (P.make_test(P.TEST_SERIAL, bits=3), dict(bits=3)),
                     (P.make_test(P.TEST_GAP, lo=0, hi=1 << 30, t=12), dict(lo=0, hi=1 << 30, t=12))):
        kind = {P.TEST_FREQUENCY: "frequency", P.TEST_SERIAL: "serial", P.TEST_GAP: "gap"}[test.kind]
        counts = _counts(test, d.data_ptr(), u.size)
        chi2, dof, p = P.prand_test_evaluate(test, u.size, counts)
        ref_chi2, ref_p = O.chi2_test(kind, u.size, counts, **kw)
        assert dof == P.prand_test_cells(test) - 1
        assert chi2 == pytest.approx(ref_chi2, rel=1e-12)
        assert p == pytest.approx(ref_p, rel=1e-9, abs=1e-300)


# Table 3's skip-ahead subsequences: 2^n values skipped per step, n from the
# paper's rows (MT19937 440 included).
STUDY = [("MRG32K3A", 90), ("LFSR113", 75), ("GM61", 75), ("GM31", 24), ("GQ58_1", 24), ("GM55", 60),
         ("MT19937", 440), ("MT19937", 19)]


@pytest.mark.parametrize("gen,sp", STUDY)
def test_skip_ahead_subsequence_counts_and_pvalues(gen, sp):
    P.load()
    seed, n = 7, 1 << 15
    h = P.prand_create(gen, seed)
    try:
        P.prand_init_streams_spaced(h, sp, 0, n)
        w = torch.empty(n, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(h, w.data_ptr(), 1, 0)  # output 0 of each stream = u[k 2^sp]
        torch.cuda.synchronize()
    finally:
        P.prand_destroy(h)
    u = w.cpu().numpy().view(np.uint32)
    # the subsequence itself, on a prefix the oracle computes quickly
    k = 64 if gen != "MT19937" else 8
    assert np.array_equal(u[:k], O.spaced_outputs(gen, seed, sp, 0, k, 1)[:, 0])
    for test in (P.make_test(P.TEST_FREQUENCY, bits=8), P.make_test(P.TEST_SERIAL, bits=4),
                 P.make_test(P.TEST_GAP, lo=0, hi=1 << 29, t=24)):
        counts = _counts(test, w.data_ptr(), n)
        assert np.array_equal(counts, _oracle_counts(test, u))
        _, _, p = P.prand_test_evaluate(test, n, counts)
        assert 1e-6 < p < 1 - 1e-6, (gen, sp, test.kind, p)


def test_count_errors():
    P.load()
    c = torch.zeros(8, dtype=torch.int64, device="cuda")
    w = torch.zeros(16, dtype=torch.int32, device="cuda")
    bad = [P.make_test(P.TEST_FREQUENCY, bits=0), P.make_test(P.TEST_FREQUENCY, bits=13),
           P.make_test(P.TEST_SERIAL, bits=7), P.make_test(P.TEST_GAP, lo=5, hi=5, t=3),
           P.make_test(P.TEST_GAP, lo=0, hi=(1 << 32) + 1, t=3), P.make_test(P.TEST_GAP, lo=0, hi=9, t=0),
           P.make_test(7, bits=3)]
    for t in bad:
        assert P.prand_test_cells(t) == 0
        with pytest.raises(P.PrandError):
            P.prand_test_counts(t, w.data_ptr(), 16, c.data_ptr(), 0)
    ok = P.make_test(P.TEST_FREQUENCY, bits=2)
    with pytest.raises(P.PrandError):
        P.prand_test_counts(ok, w.data_ptr(), 16, c.data_ptr() + 4, 0)  # counts not 8-byte aligned
    with pytest.raises(P.PrandError):
        P.prand_test_counts(ok, w.data_ptr() + 2, 4, c.data_ptr(), 0)  # words not 4-byte aligned
    with pytest.raises(P.PrandError):
        P.prand_test_counts(ok, w.data_ptr(), 1 << 40, c.data_ptr(), 0)


def test_short_period_subsequence_is_rejected():
    # GM19 skipping 2^21 values per step repeats after 2^18 - 1 values (its period
    # 2^20 (2^18 - 1) shares 2^20 with the skip): 2^20 words hold four copies, and
    # the frequency and serial tests reject the sequence far beyond the paper's
    # 1e-3 threshold (the serial pairs of consecutive copies are offset by one
    # word, the period being odd, so its statistic grows less than the frequency's)
    P.load()
    n = 1 << 20
    h = P.prand_create("GM19", 5)
    try:
        P.prand_init_streams_spaced(h, 21, 0, n)
        w = torch.empty(n, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(h, w.data_ptr(), 1, 0)
        torch.cuda.synchronize()
    finally:
        P.prand_destroy(h)
    u = w.cpu().numpy().view(np.uint32)
    per = (1 << 18) - 1
    assert np.array_equal(u[:per], u[per:2 * per])
    for test in (P.make_test(P.TEST_FREQUENCY, bits=10), P.make_test(P.TEST_SERIAL, bits=5)):
        _, _, p = P.prand_test_evaluate(test, n, _counts(test, w.data_ptr(), n))
        assert p < 1e-6
