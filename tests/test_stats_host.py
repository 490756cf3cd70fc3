"""Host-side parts of the statistical tests (no GPU): the chi-square tail of
the C library against scipy and closed forms, and Pearson's statistic against
the oracle's."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1307_5869_gb300 as P

scipy_stats = pytest.importorskip("scipy.stats")


@pytest.fixture(scope="module")
def lib():
    if not __import__("os").path.exists(P.LIB_PATH):
        pytest.skip("library not built")
    return P.load()


@pytest.mark.parametrize("dof", [1, 2, 3, 7, 15, 63, 255, 1023, 4095])
def test_chi2_tail_against_scipy(lib, dof):
    for q in (1e-12, 1e-6, 1e-3, 0.05, 0.3, 0.5, 0.7, 0.95, 0.999, 1 - 1e-6):
        x = float(scipy_stats.chi2.isf(q, dof))
        assert P.prand_chi2_sf(x, dof) == pytest.approx(q, rel=1e-9), (dof, q)
    assert P.prand_chi2_sf(0.0, dof) == 1.0


def test_chi2_tail_closed_forms(lib):
    for x in (0.01, 0.5, 2.0, 9.0, 40.0, 300.0):
        assert P.prand_chi2_sf(x, 2.0) == pytest.approx(math.exp(-x / 2), rel=1e-12)     # two degrees
        assert P.prand_chi2_sf(x, 1.0) == pytest.approx(math.erfc(math.sqrt(x / 2)), rel=1e-10)  # one degree
    assert math.isnan(P.prand_chi2_sf(-1.0, 3.0)) and math.isnan(P.prand_chi2_sf(1.0, 0.0))
    assert P.prand_chi2_sf(float("inf"), 3.0) == 0.0


def test_cells(lib):
    assert P.prand_test_cells(P.make_test(P.TEST_FREQUENCY, bits=12)) == 4096
    assert P.prand_test_cells(P.make_test(P.TEST_SERIAL, bits=6)) == 4096
    assert P.prand_test_cells(P.make_test(P.TEST_GAP, lo=0, hi=1 << 32, t=1024)) == 1025
    assert P.prand_test_cells(P.make_test(P.TEST_SERIAL, bits=7)) == 0


def test_evaluate_against_the_oracle(lib):
    u = np.random.default_rng(12).integers(0, 2**32, 50001, dtype=np.uint32)
    for test, kind, counts, kw in (
            (P.make_test(P.TEST_FREQUENCY, bits=5), "frequency", O.freq_counts(u, 5), dict(bits=5)),
            (P.make_test(P.TEST_SERIAL, bits=2), "serial", O.serial_counts(u, 2), dict(bits=2)),
            (P.make_test(P.TEST_GAP, lo=7, hi=3 << 29, t=9), "gap", O.gap_counts(u, 7, 3 << 29, 9),
             dict(lo=7, hi=3 << 29, t=9))):
        chi2, dof, p = P.prand_test_evaluate(test, u.size, counts)
        ref_chi2, ref_p = O.chi2_test(kind, u.size, counts, **kw)
        assert chi2 == pytest.approx(ref_chi2, rel=1e-12)
        assert p == pytest.approx(ref_p, rel=1e-9)
        assert dof == len(counts) - 1
    with pytest.raises(P.PrandError):  # no words: no expectation to compare with
        P.prand_test_evaluate(P.make_test(P.TEST_FREQUENCY, bits=2), 0, [0, 0, 0, 0])
