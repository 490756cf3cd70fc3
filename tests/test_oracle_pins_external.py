"""Oracle pins against values fixed outside the oracle: SplitMix64's published
outputs, a hand-worked MRG32k3a step from the RngStreams default seed, and
hand-worked GM/GQ output words (tests/golden/*.txt, each citing its source).

Each pin names the plausible mistakes it catches; a pin that only retyped the
oracle's own formula would catch none of them."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GM_GENS = ["GM19", "GM29", "GM31", "GM55", "GM61", "GQ58_1", "GQ58_3", "GQ58_4"]


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split("#")[0].strip() for ln in f if ln.split("#")[0].strip()]


def test_splitmix64_published_outputs():
    # catches: a wrong increment or multiplier, the shifts 30/27/31 permuted, or
    # mixing the state before (instead of after) adding the increment
    lines = _lines("splitmix64_check.txt")
    seed = int(lines[0].split()[1])
    want = [int(x) for x in lines[1:]]
    assert O.splitmix64(seed, len(want)) == want


def test_seeded_mrg32k3a_state_comes_from_splitmix64():
    # the seeded MRG32K3A state (reading: six SplitMix64 draws, x mod m1, y mod
    # m2) is built from the pinned SplitMix64 sequence
    m1, m2 = 4294967087, 4294944443
    for seed in (1, 12345, 2**63 + 5):
        d = O.splitmix64(seed, 6)
        raw = np.frombuffer(O.State("MRG32K3A", seed).raw(), dtype=np.uint64)
        assert [int(v) for v in raw[:3]] == [v % m1 for v in d[:3]]
        assert [int(v) for v in raw[3:6]] == [v % m2 for v in d[3:6]]


def test_mrg32k3a_first_step_from_the_rngstreams_seed():
    # a hand-worked step from the paper's constants: catches the sum instead of
    # the difference of the two components, a sign or coefficient error in
    # either recurrence, and a wrong normalisation of the double map
    vals = dict(ln.split() for ln in _lines("mrg32k3a_check.txt"))
    st = O.State("MRG32K3A")  # default state: 12345 in all six words (reading)
    assert np.frombuffer(st.raw(), dtype=np.uint64).tolist() == [12345] * 6
    assert int(st.copy().u32(1)[0]) == int(vals["z3"])
    assert abs(st.copy().f64(1)[0] - float(vals["u3"])) < 1e-15
    # the state after the step holds x_3 and y_3 as its newest words
    st.u32(1)
    raw = np.frombuffer(st.raw(), dtype=np.uint64)
    assert int(raw[0]) == int(vals["x3"]) and int(raw[3]) == int(vals["y3"])


def _worked_cases():
    cases, cur = [], None
    for ln in _lines("gm_words_worked.txt"):
        f = ln.split()
        if f[0] == "case":
            cur = {"gen": f[1], "word": int(f[2], 16), "points": []}
            cases.append(cur)
        else:
            cur["points"].append((f[1], int(f[2]), int(f[3])))
    out = []
    for c in cases:
        s = O.gm_param(c["gen"], "s")
        xp, x = [None] * s, [None] * s
        rest = None
        for lst, a, b in c["points"]:
            if lst == "*":
                rest = (a, b)
                continue
            for i in lst.split(","):
                xp[int(i)], x[int(i)] = a, b
        for i in range(s):
            if xp[i] is None:
                xp[i], x[i] = rest
        out.append((c["gen"], xp, x, c["word"]))
    return out


WORKED = _worked_cases()


@pytest.mark.parametrize("gen,xp,x,word", WORKED, ids=[c[0] for c in WORKED])
def test_gm_hand_worked_words(gen, xp, x, word):
    # one hand-worked word per v (1, 3, 4): catches reversed bit order, the strip
    # of x^(n) or x^(n-1) instead of the new value, + q x_prev, and for GQ58.3
    # a truncation other than bits 0..31 of the 36-bit sum (s = 10 points, or
    # point 10's low bits dropped)
    st = O.gm_state_raw(gen, xp, x)
    assert st.next() == word


def _plain_word(gen, xp, x):
    """The output map restated with Python integers: each point steps by eq.
    (rec1) and contributes floor(2^v x' / g) at bit v*i; bits from 32 up are
    dropped."""
    k, q, g, v = (O.gm_param(gen, n) for n in ("k", "q", "g", "v"))
    w = 0
    for i in range(len(x)):
        n = (k * x[i] - q * xp[i]) % g
        xp[i], x[i] = x[i], n
        w += ((n << v) // g) << (v * i)
    return w % 2**32


@pytest.mark.parametrize("gen", GM_GENS)
def test_gm_words_restated_in_python(gen):
    # every ensemble, seeded streams at block-split positions: the oracle's
    # words equal the Python restatement (word assembly, truncation, and the
    # state update order) over 40 consecutive words
    for seed, k in ((12345, 0), (7, 3), (2**64 - 1, 11)):
        st = O.State.stream(gen, seed, k)
        xp, x = O.gm_state_points(st)
        for _ in range(40):
            assert st.next() == _plain_word(gen, xp, x)
        assert O.gm_state_points(st) == (xp, x)
