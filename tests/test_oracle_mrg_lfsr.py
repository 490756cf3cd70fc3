"""Pins for the oracle's MRG32K3A (Sec. 5.2) and LFSR113 (Sec. 5.3).

MRG32K3A: the matrix form of Sec. 5.2 evaluated independently in Python
integers, the exact component orders, brute-force jumps, and the
closed-form period (m1^3 - 1)(m2^3 - 1)/2 of Table 2.
LFSR113: the word step against a bit-level simulation of eqs. (lfsrRel1) and
(lfsrOutput), brute-force jumps, the doubling identity (lfsrRel2), and the
component periods 2^p - 1 whose product is Table 2's 1.0e34.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M1 = 2**32 - 209
M2 = 2**32 - 22853


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------------- MRG32K3A

def test_mrg_matrix_form_of_sec_5_2():
    # X_{n+1} = A X_n mod m1, Y_{n+1} = B Y_n mod m2 with the printed a, b, c, d,
    # evaluated with Python integers; output z = (x - y) mod m1, 0 -> m1.
    a, b, c, d = 1403580, -810728, 527612, -1370589
    A = [[0, a, b], [1, 0, 0], [0, 1, 0]]
    B = [[c, 0, d], [1, 0, 0], [0, 1, 0]]
    X = [12345] * 3
    Y = [12345] * 3
    ref = []
    for _ in range(2000):
        X = [sum(A[i][k] * X[k] for k in range(3)) % M1 for i in range(3)]
        Y = [sum(B[i][k] * Y[k] for k in range(3)) % M2 for i in range(3)]
        z = (X[0] - Y[0]) % M1
        ref.append(z if z else M1)
    assert np.array_equal(O.State("MRG32K3A").u32(2000), np.array(ref, dtype=np.uint32))


@pytest.mark.parametrize("seed", [O.SEED_DEFAULT, 12345, 7])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 100, 12345, 10**6 + 7])
def test_mrg_jump_equals_steps(seed, n):
    a = O.State("MRG32K3A", seed)
    b = a.copy()
    if n:
        a.u32(n)
    b.jump(n)
    assert np.array_equal(a.u32(64), b.u32(64))


def test_mrg_period_closed_form():
    rho = (M1**3 - 1) * (M2**3 - 1) // 2
    assert f"{rho:.1e}" == "3.1e+57"  # Table 2
    st = O.State("MRG32K3A", 12345)
    ref = st.copy().u32(50)
    assert np.array_equal(st.copy().jump(rho).u32(50), ref)
    # m1^3 - 1 alone returns the x component but not the combined state
    assert not np.array_equal(st.copy().jump(M1**3 - 1).u32(50), ref)


def test_mrg_component_orders_exact():
    sympy = pytest.importorskip("sympy")
    # A has order exactly m1^3 - 1 mod m1 (and B: m2^3 - 1 mod m2): primitive
    # characteristic polynomials, so every nonzero state has full period.
    def matpow(M, e, m):
        R = sympy.eye(3)
        Bm = sympy.Matrix(M)
        while e:
            if e & 1:
                R = (R * Bm).applyfunc(lambda v: v % m)
            Bm = (Bm * Bm).applyfunc(lambda v: v % m)
            e >>= 1
        return R
    for M, m in (([[0, 1403580, -810728], [1, 0, 0], [0, 1, 0]], M1),
                 ([[527612, 0, -1370589], [1, 0, 0], [0, 1, 0]], M2)):
        order = m**3 - 1
        assert sympy.isprime(m)
        assert matpow(M, order, m) == sympy.eye(3)
        for r in sympy.factorint(order):
            assert matpow(M, order // r, m) != sympy.eye(3)


def test_mrg_output_range():
    out = O.State("MRG32K3A", 5).u32(200000).astype(np.int64)
    assert out.min() >= 1 and out.max() <= M1
    f = O.State("MRG32K3A", 5).f64(200000)
    assert (f > 0).all() and (f < 1).all()


def test_mrg_streams():
    L = O.block_length("MRG32K3A")
    assert L == 2**127 and 10**38 <= L and 10**19 * L < (M1**3 - 1) * (M2**3 - 1) // 2
    s0 = O.State("MRG32K3A", 12345)
    for k in (1, 2, 5, 10**18 + 3):
        assert np.array_equal(O.State.stream("MRG32K3A", 12345, k).u32(32), s0.copy().jump(k * L).u32(32))


# ----------------------------------------------------------------- LFSR113

def _word_from_bits(bits):
    w = 0
    for b in bits:
        w = (w << 1) | int(b)
    return w


@pytest.mark.parametrize("j", range(4))
def test_lfsr_word_step_is_bit_recurrence(j):
    L = O.lib()
    p, q, s = (L.orc_lfsr_param(j, w) for w in range(3))
    rng = np.random.default_rng(100 + j)
    for _ in range(20):
        init = rng.integers(0, 2, size=p).astype(np.uint8)
        if not init.any():
            init[0] = 1
        nb = s * 300 + 64
        x = (ctypes.c_uint8 * nb)()
        L.orc_lfsr_bits(j, (ctypes.c_uint8 * p)(*init.tolist()), x, nb)
        xs = np.frombuffer(x, dtype=np.uint8)
        # independent check of eq. (lfsrRel1) on the simulated bits
        assert all(xs[n] == xs[n - p] ^ xs[n - p + q] for n in range(p, 400))
        z = _word_from_bits(xs[:32])
        for n in range(300):
            assert z == _word_from_bits(xs[n * s:n * s + 32])  # eq. (lfsrOutput)
            z = L.orc_lfsr_comp_step(z, j)


@pytest.mark.parametrize("j", range(4))
def test_lfsr_doubling_identity(j):
    # eq. (lfsrRel2): x_n = x_{n-kp} + x_{n-kp+kq} (mod 2) for k = 2^e
    L = O.lib()
    p, q, _ = (L.orc_lfsr_param(j, w) for w in range(3))
    init = (ctypes.c_uint8 * p)(*([1] + [0] * (p - 1)))
    nb = 40 * p + 200
    x = (ctypes.c_uint8 * nb)()
    L.orc_lfsr_bits(j, init, x, nb)
    for e in range(5):
        k = 2**e
        for n in range(k * p, nb):
            assert x[n] == x[n - k * p] ^ x[n - k * p + k * q]


@pytest.mark.parametrize("j", range(4))
def test_lfsr_component_period(j):
    sympy = pytest.importorskip("sympy")
    L = O.lib()
    p = L.orc_lfsr_param(j, 0)
    z = L.orc_lfsr_comp_step(0xDEADBEEF, j)  # one step makes the word consistent
    per = 2**p - 1
    assert L.orc_lfsr_comp_jump(z, j, O.big(per)) == z
    for r in sympy.factorint(per):
        assert L.orc_lfsr_comp_jump(z, j, O.big(per // r)) != z


def test_lfsr_combined_period_table2():
    per = 1
    for p in (31, 29, 28, 25):
        per *= 2**p - 1
    assert f"{per:.1e}" == "1.0e+34"


@pytest.mark.parametrize("seed", [O.SEED_DEFAULT, 12345, 2**40 + 1])
@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 1000, 2**20 + 5])
def test_lfsr_jump_equals_steps(seed, n):
    a = O.State("LFSR113", seed)
    b = a.copy()
    if n:
        a.u32(n)
    b.jump(n)
    assert np.array_equal(a.u32(64), b.u32(64))


def test_lfsr_streams():
    L = O.block_length("LFSR113")
    assert L == 2**34 and 10**10 <= L
    s0 = O.State("LFSR113", 12345)
    for k in (1, 3, 2**60 + 5):
        assert np.array_equal(O.State.stream("LFSR113", 12345, k).u32(32), s0.copy().jump(k * L).u32(32))
    # Table 4: 3.8e18 sequences of length 2^34 stay inside the 1.0e34 period
    assert 38 * 10**17 * L < (2**31 - 1) * (2**29 - 1) * (2**28 - 1) * (2**25 - 1)


def test_lfsr_seeds_valid():
    L = O.lib()
    for seed in range(200):
        raw = O.State("LFSR113", seed).raw()
        z = np.frombuffer(raw, dtype=np.uint32)
        for j in range(4):
            p = L.orc_lfsr_param(j, 0)
            assert int(z[j]) >> (32 - p) != 0
