"""Stream-initialisation variants of Table 4 and the a * 2^b skip-ahead,
through the C ABI, against the oracle bit for bit."""
import os
from decimal import Decimal

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
import paper_1307_5869_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    out = []
    for line in open(os.path.join(HERE, "golden", "table4_variants.txt")):
        if line.strip() and not line.startswith("#"):
            g, v, fn, n, L = line.split()
            out.append((g, int(v), int(Decimal(n))))
    return out


ROWS = _rows()


def _gen(h, n, m):
    t = torch.empty(n * m, dtype=torch.int32, device="cuda")
    P.prand_generate_u32(h, t.data_ptr(), m, 0)
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32).reshape(n, m)


@pytest.mark.parametrize("gen,v,nmax", ROWS, ids=[f"{r[0]}-{r[1]}" for r in ROWS])
def test_variant_streams_follow_the_oracle(gen, v, nmax):
    P.load()
    seed, m = 2024, 96
    for first, n in ((0, 3), (nmax - 4, 4)):  # the first streams and the last ones of the variant
        h = P.prand_create(gen, seed)
        try:
            assert P.prand_init_streams_variant(h, v, first, n) == 0
            got = _gen(h, n, m)
        finally:
            P.prand_destroy(h)
        st = O.Streams(gen, seed, first, n, variant=v)
        for j in range(n):
            assert np.array_equal(got[j], st.state(j).u32(m)), (gen, v, first + j)


def test_variant_overlap_warning_and_unlisted_variant():
    P.load()
    h = P.prand_create("GM61", 5)
    try:
        assert P.prand_init_streams_variant(h, P.VARIANT_LONG, 4000000000 - 2, 4) == 7  # past N_max
        with pytest.raises(P.PrandError):
            P.prand_init_streams_variant(h, P.VARIANT_MEDIUM, 0, 1)  # GM61 has no medium variant
    finally:
        P.prand_destroy(h)


def test_switching_variants_and_checkpoint():
    P.load()
    gen, seed, n, m = "GQ58_3", 77, 5, 64
    h = P.prand_create(gen, seed)
    try:
        P.prand_init_streams_variant(h, P.VARIANT_LONG, 10, n)
        a = _gen(h, n, m)
        blob = P.prand_get_state(h)
        P.prand_init_streams(h, 10, n)  # back to the default variant: its own base ensemble
        b = _gen(h, n, m)
        P.prand_set_state(h, blob)  # the long-variant streams, continued
        c = _gen(h, n, m)
    finally:
        P.prand_destroy(h)
    lo = O.Streams(gen, seed, 10, n, variant=2)
    de = O.Streams(gen, seed, 10, n, variant=0)
    for j in range(n):
        s = lo.state(j)
        assert np.array_equal(a[j], s.u32(m))
        assert np.array_equal(c[j], s.u32(m))
        assert np.array_equal(b[j], de.state(j).u32(m))


@pytest.mark.parametrize("gen,a,b", [("MT19937", 3, 440), ("MT19937", 0xFFFFFFFFFFFFFFFF, 448), ("MT19937", 5, 7),
                                     ("MRG32K3A", 12345, 190), ("LFSR113", 7, 100), ("GM61", 3, 120),
                                     ("GM55", 1, 0)])
def test_skipahead_pow2(gen, a, b):
    P.load()
    n, m = 3, 700
    h = P.prand_create(gen, 31)
    try:
        P.prand_init_streams(h, 2, n)
        _gen(h, n, 17)  # mid-block for MT19937
        P.prand_skipahead_pow2(h, a, b)
        got = _gen(h, n, m)
    finally:
        P.prand_destroy(h)
    st = O.Streams(gen, 31, 2, n)
    for j in range(n):
        s = st.state(j)
        s.u32(17)
        s.jump(a << b)
        assert np.array_equal(got[j], s.u32(m)), j


def test_skipahead_pow2_range():
    P.load()
    h = P.prand_create("MRG32K3A", 1)
    m = P.prand_create("MT19937", 1)
    try:
        P.prand_init_streams(h, 0, 1)
        P.prand_init_streams(m, 0, 1)
        with pytest.raises(P.PrandError):
            P.prand_skipahead_pow2(h, 1, 256)  # above 2^256 for a generator other than MT19937
        with pytest.raises(P.PrandError):
            P.prand_skipahead_pow2(m, 2, 511)  # 2^512
        P.prand_skipahead_pow2(m, 1, 511)  # 2^511 < 2^512
        P.prand_skipahead_pow2(m, 0, 600)  # a = 0: nothing to do
    finally:
        P.prand_destroy(h)
        P.prand_destroy(m)
