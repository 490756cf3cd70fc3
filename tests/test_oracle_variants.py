"""The oracle's stream-initialisation variants against Table 4 (all 24 rows):
the printed counts and lengths, the capacity bound (every stream of every
variant fits in the period), the GM/GQ ensembles spaced for their variant, and
block splitting by the variant's length."""
import os
from decimal import Decimal

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    out = []
    for line in open(os.path.join(HERE, "golden", "table4_variants.txt")):
        if line.strip() and not line.startswith("#"):
            g, v, fn, n, L = line.split()
            out.append((g, int(v), fn, int(Decimal(n)), int(Decimal(L))))
    return out


ROWS = _rows()
GMS = ["GM19", "GM29", "GM31", "GM55", "GM61", "GQ58_1", "GQ58_3", "GQ58_4"]


def test_table4_has_24_functions():
    assert len(ROWS) == 24 and len({r[2] for r in ROWS}) == 24


@pytest.mark.parametrize("gen,v,fn,nmax,maxlen", ROWS, ids=[r[2] for r in ROWS])
def test_variant_matches_table4(gen, v, fn, nmax, maxlen):
    n, L = O.variant_info(gen, v)
    assert n == nmax
    if gen in GMS:
        assert L == maxlen  # the printed maximal length is the block length
    else:  # a power of two at least the printed length
        assert L >= maxlen and L & (L - 1) == 0
    # capacity: every stream of the variant ends inside the period
    if gen in GMS:
        p, s = O.gm_param(gen, "p"), O.gm_param(gen, "s")
        assert s * n * L <= p * p - 1
    elif gen == "LFSR113":
        assert n * L <= (2**31 - 1) * (2**29 - 1) * (2**28 - 1) * (2**25 - 1)
    elif gen == "MRG32K3A":
        m1, m2 = 2**32 - 209, 2**32 - 22853
        assert n * L <= (m1**3 - 1) * (m2**3 - 1) // 2
    else:
        assert n * L < 2**19937 - 1


def test_unlisted_variants_are_rejected():
    listed = {(g, v) for g, v, *_ in ROWS}
    for g in O.GENS:
        for v in range(3):
            assert (O.variant_info(g, v) is None) == ((g, v) not in listed), (g, v)
    with pytest.raises(ValueError):
        O.State.stream("GM61", 1, 0, variant=1)


def _point_jump(k, q, g, xp, xc, e):
    import ctypes
    a, b = ctypes.c_uint64(xp), ctypes.c_uint64(xc)
    O.lib().orc_gm_point_jump(k, q, g, ctypes.byref(a), ctypes.byref(b), O.big(e))
    return a.value, b.value


@pytest.mark.parametrize("gen,v", [(g, v) for g, v, *_ in ROWS if g in GMS and v > 0])
def test_ensemble_spacing_of_each_variant(gen, v):
    k, q, g, s = (O.gm_param(gen, x) for x in ("k", "q", "g", "s"))
    n, L = O.variant_info(gen, v)
    st = np.frombuffer(O.State.stream(gen, 4321, 0, variant=v).raw(), dtype=np.uint64)
    x0p, x0c = int(st[0]), int(st[32])
    for i in range(1, s):
        assert (int(st[i]), int(st[32 + i])) == _point_jump(k, q, g, x0p, x0c, i * n * L)


@pytest.mark.parametrize("gen,v", [(g, v) for g, v, *_ in ROWS if v > 0])
def test_block_split_of_each_variant(gen, v):
    n, L = O.variant_info(gen, v)
    s0 = O.State.stream(gen, 777, 0, variant=v)
    for k in (1, 2, 12345, n - 1):
        assert np.array_equal(O.State.stream(gen, 777, k, variant=v).u32(8), s0.copy().jump(k * L).u32(8)), k
