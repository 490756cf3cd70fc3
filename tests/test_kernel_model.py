"""The GM/GQ kernels' arithmetic, modelled on the CPU operation by operation
(tests/kernel_model.py), against the exact definitions: every step is eq.
(rec1) mod p and stays in its lazy range; every strip extraction is
floor(2^v z / p) of the canonical residue.  These check the design of the
limb arithmetic before it runs; the GPU parity tests check the kernels."""
import numpy as np
import pytest

import kernel_model as KM

GENS = list(KM.PARAMS)


def _edge_and_random(p, slack, rng, n):
    edge = [0, 1, p - 1, p, p + slack - 1, (p + 1) // 2, (p - 1) // 2]
    return [e for e in edge if e < p + slack] + [int(x) for x in rng.integers(0, p + slack, n)]


@pytest.mark.parametrize("gen", [g for g in GENS if g != "GM61"])
def test_step_is_the_recurrence_and_stays_lazy(gen):
    k, q, p, t, v, s, slack = KM.PARAMS[gen]
    rng = np.random.default_rng(1)
    zs = _edge_and_random(p, slack, rng, 3000)
    ys = _edge_and_random(p, slack, rng, 3000)
    for z in zs[:40]:
        for y in ys[:40]:
            r = KM.step(gen, z, y)
            assert r % p == (k * z - q * y) % p and r < p + slack, (z, y, r)
    for z, y in zip(zs, ys[::-1]):
        r = KM.step(gen, z, y)
        assert r % p == (k * z - q * y) % p and r < p + slack, (z, y, r)


def test_gm61_step_on_rotated_values():
    # u = 2 z + 1 (mod p) obeys u' = 24 u - 74 u_prev + 51; the kernel keeps u in
    # [1, 2^61 + 2^40) and its output bit is floor(2 z' / p)
    p = KM.P61
    rng = np.random.default_rng(2)
    lim = (1 << 61) + (1 << 40)
    us = [1, 2, p - 1, p, lim - 1] + [int(x) for x in rng.integers(1, lim, 4000, dtype=np.uint64)]
    for u, up in zip(us, us[::-1]):
        r, bit = KM.gm61_step(u, up)
        assert 1 <= r < lim
        assert r % p == (24 * u - 74 * up + 51) % p
        z = KM.gm61_leave(r)
        assert bit == (2 * z // p == 1)


def test_gm61_rotation_round_trip():
    rng = np.random.default_rng(3)
    p = KM.P61
    for z in [0, 1, p - 1, 1 << 60, (1 << 60) - 1] + [int(x) for x in rng.integers(0, p, 2000, dtype=np.uint64)]:
        u = KM.gm61_enter(z)
        assert 1 <= u <= p and u == (2 * z) % p + 1 and KM.gm61_leave(u) == z


@pytest.mark.parametrize("gen", ["GM19", "GM29", "GM31", "GQ58_1"])
def test_v1_strip_on_lazy_values(gen):
    p, slack = KM.PARAMS[gen][2], KM.PARAMS[gen][6]
    rng = np.random.default_rng(4)
    for z in KM.strip_boundaries(gen) + list(range(p, p + slack)) + [int(x) for x in rng.integers(0, p, 2000)]:
        assert KM.strip1(gen, z) == (2 * (z % p) // p == 1), z


@pytest.mark.parametrize("gen", ["GM55", "GQ58_3", "GQ58_4"])
def test_strip_insert_is_the_strip(gen):
    k, q, p, t, v, s, slack = KM.PARAMS[gen]
    rng = np.random.default_rng(5)
    zs = KM.strip_boundaries(gen) + [p + d for d in (0, 1, 2, 3, slack // 2, slack - 1)]
    zs += [int(x) for x in rng.integers(0, p, 1500, dtype=np.uint64)]
    for z in zs:
        want = ((z % p) << v) // p
        for i in range(s):
            pos = v * i
            if pos >= 32:
                assert KM.strip_insert(gen, i, z) == 0
                continue
            bits = min(v, 32 - pos)
            got = KM.strip_insert(gen, i, z) >> pos
            assert got == want % (1 << bits), (z, i, got, want)
            # only the point's own bits are written
            assert KM.strip_insert(gen, i, z, 0xFFFFFFFF) == 0xFFFFFFFF


@pytest.mark.parametrize("gen", ["GQ58_3", "GQ58_4"])
def test_gq58_strip_in_32_bits_over_the_whole_lazy_range(gen):
    # The v = 3, 4 kernels take the strip from a 32-bit sum (8 z + 3 (q0 + 1),
    # halved in its constant for v = 4) instead of the 64-bit 2^v z + 3 (q0 + 1).
    # Every lazy residue z in [0, p + slack) is checked against
    # floor(2^v (z mod p) / p) mod 2^v; a wrong shift, constant or wrap fails.
    v, slack = KM.PARAMS[gen][4], KM.PARAMS[gen][6]
    p = KM.PARAMS[gen][2]
    top = 28 if v == 4 else 29
    # uint32 arithmetic wraps mod 2^32 as the kernel's does; the exact strip
    # floor(2^v zm / p) is taken in doubles, exact here (the quotient is never
    # closer than 1/p ~ 2^-29 to an integer, far above the rounding error)
    step = 1 << 25
    for lo in range(0, p + slack, step):
        z = np.arange(lo, min(lo + step, p + slack), dtype=np.uint32)
        q0 = z >> np.uint32(29 - v)
        c = (np.uint32(3) * q0 + np.uint32(3)) >> np.uint32(1) if v == 4 else np.uint32(3) * q0 + np.uint32(3)
        got = ((np.uint32(8) * z + c) >> np.uint32(top)) & np.uint32((1 << v) - 1)
        zm = np.where(z >= np.uint32(p), z - np.uint32(p), z)
        want = np.floor(zm.astype(np.float64) * float(1 << v) / float(p)).astype(np.uint32) & np.uint32((1 << v) - 1)
        assert np.array_equal(got, want), lo


@pytest.mark.parametrize("gen", GENS)
def test_lazy_state_search_reaches_the_lazy_range(gen):
    # the states the GPU edge-case tests import: the model shows that their
    # next value is kept in the lazy range, and that value is the exact residue
    k, q, p = KM.PARAMS[gen][:3]
    rng = np.random.default_rng(6)
    for z, y in KM.lazy_states(gen, 16, rng):
        got, exact = KM.next_lazy(gen, z, y)
        if gen == "GM61":
            assert got >= 1 << 61 and KM.gm61_leave(got) == exact
        else:
            assert got >= p and got - p == exact


@pytest.mark.parametrize("gen", GENS)
def test_boundary_states_hit_every_strip_boundary(gen):
    k, q, p = KM.PARAMS[gen][:3]
    rng = np.random.default_rng(7)
    states = KM.boundary_states(gen, rng)
    assert [(k * z - q * y) % p for z, y in states] == KM.strip_boundaries(gen)
