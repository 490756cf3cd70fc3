"""Pins for the oracle's MT19937 (step, seeding, jump-ahead of Sec. 5.4).

Each pin is external to the oracle: the C++ standard's check value, two
independent MT19937 implementations (numpy's legacy RandomState, CPython's
random module), brute force (jump == single steps), closed forms of the
characteristic polynomial (degree 19937, x^(2^19937) = x), and numpy's own
MT19937 jump by 2^128 (an independent jump implementation).
"""
import os
import random

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_cxx_standard_check_value():
    (seed, idx, val), = _golden_rows("mt19937_check.txt")
    st = O.State("MT19937", int(seed))
    out = st.u32(int(idx))
    assert int(out[-1]) == int(val)
    # the default seed of the library is the same 5489
    assert (O.State("MT19937").u32(int(idx))[-1]) == int(val)


@pytest.mark.parametrize("seed", [0, 1, 5489, 12345, 2**31 + 7, 2**32 - 1])
def test_init_genrand_matches_numpy_legacy(seed):
    # numpy's RandomState(int) seeds with init_genrand and draws raw 32-bit outputs here.
    ref = np.random.RandomState(seed).randint(0, 2**32, size=3000, dtype=np.uint32)
    assert np.array_equal(O.State("MT19937", seed).u32(3000), ref)


@pytest.mark.parametrize("seed", [2**32, 0x9E3779B97F4A7C15, 2**64 - 2, (7 << 32) | 5])
def test_init_by_array_matches_cpython(seed):
    # CPython's random.seed(int) uses init_by_array with the 32-bit words of the int.
    r = random.Random(seed)
    ref = np.array([r.getrandbits(32) for _ in range(3000)], dtype=np.uint32)
    assert np.array_equal(O.State("MT19937", seed).u32(3000), ref)


def _temper(y: int) -> int:
    y ^= y >> 11
    y ^= (y << 7) & 0x9D2C5680
    y ^= (y << 15) & 0xEFC60000
    return (y ^ (y >> 18)) & 0xFFFFFFFF


def _per_word_outputs(key, pos: int, n: int) -> np.ndarray:
    """Outputs from an MT19937 state held in the per-word form: the 624 most
    recent words x_k .. x_(k+623) stored cyclically from key[pos]; each output
    first makes x_(k+624) = x_(k+397) ^ ((x_k^u | x_(k+1)^l) A) in place of x_k
    (the recurrence of Matsumoto & Nishimura, one word at a time) and tempers it."""
    mt = [int(v) for v in key]
    out = np.empty(n, dtype=np.uint32)
    i = pos % 624
    for t in range(n):
        y = (mt[i] & 0x80000000) | (mt[(i + 1) % 624] & 0x7FFFFFFF)
        mt[i] = mt[(i + 397) % 624] ^ (y >> 1) ^ (0x9908B0DF if y & 1 else 0)
        out[t] = _temper(mt[i])
        i = (i + 1) % 624
    return out


@pytest.mark.parametrize("seed", [5489, 12345, 2**32 - 1])
def test_jump_by_2_pow_128_matches_numpy(seed):
    # numpy's MT19937.jumped() (a polynomial jump with numpy's own stored
    # polynomial) applied to a state fresh from init_genrand (all 624 words
    # unread) returns the state 2^128 outputs later in the per-word form at
    # index pos; decoded that way it must continue exactly like the oracle's
    # jump by 2^128.
    _, key, pos, _, _ = np.random.RandomState(seed).get_state()
    bg = np.random.MT19937()
    bg.state = {"bit_generator": "MT19937", "state": {"key": key, "pos": pos}}
    s = bg.jumped(1).state["state"]
    ref = _per_word_outputs(s["key"], s["pos"], 1500)
    assert np.array_equal(O.State("MT19937", seed).jump(2**128).u32(1500), ref)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 396, 397, 623, 624, 625, 1000, 1247, 1248, 19937, 65536 + 3, 10**6])
def test_jump_equals_single_steps(n):
    a = O.State("MT19937", 12345)
    b = a.copy()
    if n:
        a.u32(n)
    b.jump(n)
    assert np.array_equal(a.u32(1500), b.u32(1500))


@pytest.mark.parametrize("pre", [1, 100, 623])
def test_jump_from_inside_a_twisted_block(pre):
    a = O.State("MT19937", 777)
    a.u32(pre)
    b = a.copy()
    for n in (5, 624 - pre, 624 - pre + 1, 5000):
        a2, b2 = a.copy(), b.copy()
        a2.u32(n)
        b2.jump(n)
        assert np.array_equal(a2.u32(700), b2.u32(700))


def test_jump_composition():
    a = O.State("MT19937", 99)
    b = a.copy()
    a.jump(2**40 + 12345).jump(2**70 + 3)
    b.jump(2**40 + 12345 + 2**70 + 3)
    assert np.array_equal(a.u32(1000), b.u32(1000))


def test_charpoly_closed_forms():
    phi = O.mt_charpoly()
    assert phi.bit_length() - 1 == 19937
    # no root in GF(2): phi(0) = 1 and phi(1) = 1 (odd number of terms)
    assert phi & 1 == 1
    assert bin(phi).count("1") % 2 == 1
    # phi annihilates every output bit sequence, far beyond the 2*19937 bits BM saw
    st = O.State("MT19937", 4242)
    words = st.u32(19937 + 3000).astype(np.uint64)
    coeffs = np.array([(phi >> j) & 1 for j in range(19938)], dtype=bool)
    for bit in (0, 17, 31):
        seq = ((words >> bit) & 1).astype(np.uint8)
        for t in range(0, 3000, 199):
            assert int(np.bitwise_xor.reduce(seq[t:t + 19938][coeffs])) == 0


@pytest.mark.slow
def test_period_is_2_pow_19937_minus_1():
    # x^(2^19937) = x mod phi (19937 squarings).  With phi of prime degree 19937 and
    # no root in GF(2), this makes phi irreducible and the order of x divide the prime
    # 2^19937 - 1, so jumping 2^19937 - 1 steps returns every state (Table 2: 4.3e6001).
    g = O.mt_x_pow2k(19937)
    assert g == 2
    # applying that polynomial to a state is exactly one step
    st = O.State("MT19937", 31337)
    ref = st.copy()
    ref.u32(1)
    O.mt_apply_poly(st, g)
    assert np.array_equal(st.u32(1000), ref.u32(1000))
    import math
    digits = 19937 * math.log10(2)
    assert int(digits) == 6001 and round(10 ** (digits - int(digits)), 1) == 4.3


def test_block_split_streams():
    L = O.block_length("MT19937")
    assert L == 2**432
    # stream k is the seeded state advanced by k * 2^432
    s0 = O.State("MT19937", 12345)
    for k in (1, 2, 3, 10):
        a = O.State.stream("MT19937", 12345, k)
        b = s0.copy().jump(k * L)
        assert np.array_equal(a.u32(800), b.u32(800))
    # contiguous range == individual streams
    rng = O.Streams("MT19937", 12345, 7, 3)
    for j in range(3):
        assert np.array_equal(rng.state(j).u32(700), O.State.stream("MT19937", 12345, 7 + j).u32(700))
    # Table 4: 1e19 streams of length 1e130 fit under 2^432 spacing inside 2^512
    assert 10**130 <= L and 10**19 * L < 2**512
