"""Pins for the oracle's GM/GQ torus-map ensembles (Sec. 5.1) and the float
conversions.

GM/GQ: the recurrence (rec1) against the paper's own jump identities (rec2:
doubling of (k_n, q_n); rec3: the Lucas form), evaluated here in Python
integers; brute-force jumps; the exact period p^2 - 1 against Table 2; the
dissipative structure of GM55/GQ58 (x = 2^t z on the cycle); and a tiny
modulus whose whole state space is enumerated.  The output map, ensemble size,
seeding and block lengths are readings of gaps in the paper (parity unpinned);
only their invariants are checked.
Floats: exact values as rationals, and MRG32K3A's f64 (two roundings) within
its relative error bound 2^-52 of the exact quotient z / (m1 + 1).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GMS = ["GM19", "GM29", "GM31", "GM55", "GM61", "GQ58_1", "GQ58_3", "GQ58_4"]


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return {ln.split()[0]: ln.split()[1:] for ln in f if ln.strip() and not ln.startswith("#")}


def _params(gen):
    return {nm: O.gm_param(gen, nm) for nm in ("k", "q", "g", "v", "s", "t", "p", "L", "nmax")}


def _point_seq(k, q, g, x0, x1, n):
    import ctypes
    xp, xc = ctypes.c_uint64(x0), ctypes.c_uint64(x1)
    out = [x0, x1]
    for _ in range(n):
        O.lib().orc_gm_point_step(k, q, g, ctypes.byref(xp), ctypes.byref(xc))
        out.append(xc.value)
    return out


def _point_jump(k, q, g, x0, x1, e):
    import ctypes
    xp, xc = ctypes.c_uint64(x0), ctypes.c_uint64(x1)
    O.lib().orc_gm_point_jump(k, q, g, ctypes.byref(xp), ctypes.byref(xc), O.big(e))
    return xp.value, xc.value


@pytest.mark.parametrize("gen", GMS)
def test_table2_parameters(gen):
    P = _params(gen)
    table = {  # Table 2: k, q, g, v
        "GM19": (15, 28, 2**19 - 1, 1), "GM29": (4, 2, 2**29 - 3, 1), "GM31": (11, 14, 2**31 - 1, 1),
        "GM55": (256, 176, 16 * (2**51 - 129), 4), "GM61": (24, 74, 2**61 - 1, 1),
        "GQ58_1": (8, 48, 2**29 * (2**29 - 3), 1), "GQ58_3": (8, 48, 2**29 * (2**29 - 3), 3),
        "GQ58_4": (8, 48, 2**29 * (2**29 - 3), 4)}
    assert (P["k"], P["q"], P["g"], P["v"]) == table[gen]
    assert P["g"] == P["p"] << P["t"]


@pytest.mark.parametrize("gen", GMS)
def test_rec2_doubling_identity(gen):
    # x^(2n+w) = k_n x^(n+w) - q_n x^(w) (mod g) with k_1 = k, q_1 = q,
    # k_2n = k_n^2 - 2 q_n, q_2n = q_n^2 (Sec. 5.1)
    P = _params(gen)
    k, q, g = P["k"], P["q"], P["g"]
    x0, x1 = 3 << P["t"], 5 << P["t"]
    seq = _point_seq(k, q, g, x0, x1, 2 * 256 + 40)
    kn, qn = k % g, q % g
    n = 1
    while n <= 256:
        for w in range(0, 40):
            assert seq[2 * n + w] == (kn * seq[n + w] - qn * seq[w]) % g
        kn, qn = (kn * kn - 2 * qn) % g, (qn * qn) % g
        n *= 2
    # far jumps against rec2 at n = 2^i: jump(2n) = k_n jump(n) - q_n x^(0)
    kn, qn = k % g, q % g
    for i in range(0, 130):
        n = 2**i
        a_p, a_c = _point_jump(k, q, g, x0, x1, n)       # (x^(n), x^(n+1))
        b_p, b_c = _point_jump(k, q, g, x0, x1, 2 * n)   # (x^(2n), x^(2n+1))
        assert b_p == (kn * a_p - qn * x0) % g
        assert b_c == (kn * a_c - qn * x1) % g
        kn, qn = (kn * kn - 2 * qn) % g, (qn * qn) % g


@pytest.mark.parametrize("gen", ["GM19", "GM61", "GQ58_4"])
def test_rec3_lucas_form(gen):
    # k_0 = 2, k_1 = k, k_{n+1} = k k_n - q k_{n-1}; q_n = q^n; then rec2 holds for every n.
    P = _params(gen)
    k, q, g = P["k"], P["q"], P["g"]
    x0, x1 = 7 << P["t"], 11 << P["t"]
    seq = _point_seq(k, q, g, x0, x1, 2 * 70 + 20)
    kk = [2 % g, k % g]
    for n in range(1, 70):
        kk.append((k * kk[n] - q * kk[n - 1]) % g)
    for n in range(1, 70):
        qn = pow(q, n, g)
        for w in range(0, 20):
            assert seq[2 * n + w] == (kk[n] * seq[n + w] - qn * seq[w]) % g


@pytest.mark.parametrize("gen", GMS)
@pytest.mark.parametrize("n", [0, 1, 2, 3, 17, 1000, 54321])
def test_jump_equals_steps(gen, n):
    a = O.State(gen, 12345)
    b = a.copy()
    if n:
        a.u32(n)
    b.jump(n)
    assert np.array_equal(a.u32(40), b.u32(40))


@pytest.mark.parametrize("gen", GMS)
def test_period_is_p2_minus_1_and_table2(gen):
    sympy = pytest.importorskip("sympy")
    P = _params(gen)
    p = P["p"]
    per = p * p - 1
    printed = _golden("table2_periods.txt")[gen][0]
    mant, ex = printed.split("e")
    # Table 2 prints two significant digits (truncated for most rows, rounded for GM55)
    lead = Fraction(per, 10 ** (int(ex) - 1))
    assert int(mant.replace(".", "")) in (int(lead), round(lead))
    assert sympy.isprime(p)
    st = O.State(gen, 12345)
    ref = st.raw()
    assert st.copy().jump(per).raw() == ref
    for r in sympy.factorint(per):
        assert st.copy().jump(per // r).raw() != ref


@pytest.mark.parametrize("gen", ["GM55", "GQ58_1", "GQ58_3", "GQ58_4"])
def test_dissipative_structure(gen):
    # k and q are both even: any state falls onto multiples of 2^t within a few steps,
    # and on that set x = 2^t z with z following the same map mod p.
    P = _params(gen)
    k, q, g, t, p = P["k"], P["q"], P["g"], P["t"], P["p"]
    seq = _point_seq(k, q, g, 12345, 67891, 60)
    steps = next(i for i, x in enumerate(seq) if all(y % (1 << t) == 0 for y in seq[i:]))
    assert steps <= 20
    z = [x >> t for x in seq[steps:]]
    for i in range(2, len(z)):
        assert z[i] == (k * z[i - 1] - q * z[i - 2]) % p
    # seeded ensembles start on that set
    st = np.frombuffer(O.State(gen, 99).raw(), dtype=np.uint64)
    s = P["s"]
    assert all(int(x) % (1 << t) == 0 for x in st[:s]) and all(int(x) % (1 << t) == 0 for x in st[32:32 + s])


def test_small_modulus_whole_state_space():
    # A 2-D torus map mod a small prime whose characteristic polynomial x^2 - kx + q is
    # primitive: every nonzero state lies on the one cycle of length p^2 - 1.
    p = 13

    def order(k, q):
        # order of the companion matrix found by pure-Python powering
        M = [[k % p, (-q) % p], [1, 0]]
        R = [[1, 0], [0, 1]]
        for n in range(1, p * p):
            R = [[(R[0][0] * M[0][0] + R[0][1] * M[1][0]) % p, (R[0][0] * M[0][1] + R[0][1] * M[1][1]) % p],
                 [(R[1][0] * M[0][0] + R[1][1] * M[1][0]) % p, (R[1][0] * M[0][1] + R[1][1] * M[1][1]) % p]]
            if R == [[1, 0], [0, 1]]:
                return n
        return None

    pairs = [(k, q) for k in range(p) for q in range(1, p) if order(k, q) == p * p - 1]
    assert pairs
    for k, q in pairs[:5]:
        seen = set()
        x0, x1 = 0, 1
        seq = _point_seq(k, q, p, x0, x1, p * p)
        for i in range(p * p - 1):
            seen.add((seq[i], seq[i + 1]))
        assert (seq[p * p - 1], seq[p * p]) == (x0, x1)
        assert len(seen) == p * p - 1 and (0, 0) not in seen


@pytest.mark.parametrize("gen", GMS)
def test_table4_capacity_and_ensemble_spacing(gen):
    P = _params(gen)
    t4 = _golden("table4_streams.txt")[gen]
    nmax, maxlen = int(float(t4[1])), int(float(t4[2]))
    assert P["nmax"] == nmax and P["L"] == maxlen == O.block_length(gen)
    # s points spaced D = nmax * L apart fit inside the period p^2 - 1
    assert P["s"] * P["nmax"] * P["L"] <= P["p"] ** 2 - 1
    # point i of the seeded ensemble is point 0 advanced by i * D
    st = np.frombuffer(O.State(gen, 4321).raw(), dtype=np.uint64)
    D = P["nmax"] * P["L"]
    x0p, x0c = int(st[0]), int(st[32])
    for i in range(1, P["s"]):
        assert (int(st[i]), int(st[32 + i])) == _point_jump(P["k"], P["q"], P["g"], x0p, x0c, i * D)


@pytest.mark.parametrize("gen", GMS)
def test_block_split_streams(gen):
    L = O.block_length(gen)
    s0 = O.State(gen, 12345)
    for k in (1, 2, 999, 10**19 - 1):
        assert np.array_equal(O.State.stream(gen, 12345, k).u32(16), s0.copy().jump(k * L).u32(16))


def test_gm19_stream_one_by_single_steps():
    # block splitting by brute force: stream 1 starts 6e6 single steps after stream 0
    s0 = O.State("GM19", 12345)
    s0.u32(6000000)
    assert np.array_equal(s0.u32(64), O.State.stream("GM19", 12345, 1).u32(64))


@pytest.mark.parametrize("gen", GMS)
def test_output_bits_balanced(gen):
    # output map (a reading): each bit of the word is a strip index bit of an
    # equidistributed point, so every bit used is 1 about half the time
    P = _params(gen)
    out = O.State(gen, 2024).u32(20000).astype(np.uint64)
    used = min(32, P["v"] * P["s"])
    for b in range(used):
        frac = float(((out >> b) & 1).mean())
        assert abs(frac - 0.5) < 0.03, (b, frac)


# ----------------------------------------------------------------- floats

def test_f32_exact_values():
    L = O.lib()
    rng = np.random.default_rng(5)
    us = list(rng.integers(0, 2**32, size=5000)) + [0, 1, 255, 256, 2**32 - 1, 2**31]
    for u in us:
        f = L.orc_u32_to_f32(int(u))
        assert 0.0 <= f < 1.0
        assert Fraction(f) == Fraction(int(u) >> 8, 2**24)


def test_f64_exact_values():
    L = O.lib()
    rng = np.random.default_rng(6)
    for u in list(rng.integers(0, 2**32, size=5000)) + [0, 1, 2**32 - 1]:
        f = L.orc_u32_to_f64(int(u))
        assert 0.0 <= f < 1.0 and Fraction(f) == Fraction(int(u), 2**32)


def test_mrg_f64_error_bound():
    L = O.lib()
    m1 = 2**32 - 209
    rng = np.random.default_rng(7)
    for z in list(rng.integers(1, m1 + 1, size=5000)) + [1, 2, m1 - 1, m1]:
        f = L.orc_mrg_to_f64(int(z))
        exact = Fraction(int(z), m1 + 1)
        assert 0.0 < f < 1.0
        # two roundings (the constant, then the product), each of relative error at
        # most 2^-53: relative error of the result at most 2^-52 (+ 2^-106)
        assert abs(Fraction(f) - exact) <= exact * Fraction(1, 2**52) * (1 + Fraction(1, 2**53))
        # and it is the one correctly rounded product of z and the rounded constant
        assert Fraction(f) == Fraction(float(Fraction(int(z)) * Fraction(1.0 / (m1 + 1))))


def test_float_streams_follow_u32():
    for gen in ("MT19937", "LFSR113", "GM31", "MRG32K3A"):
        u = O.State(gen, 3).u32(1000)
        assert np.array_equal(O.State(gen, 3).f32(1000), (u >> 8).astype(np.float32) / np.float32(2**24))
        f64 = O.State(gen, 3).f64(1000)
        if gen == "MRG32K3A":
            assert np.allclose(f64, u / (2**32 - 208), rtol=2**-52, atol=0)
        else:
            assert np.array_equal(f64, u.astype(np.float64) / 2**32)
