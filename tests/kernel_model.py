"""A CPU model of the GM/GQ kernels' integer arithmetic, operation by
operation (32-bit registers wrap mod 2^32; carries as in the PTX).

Test infrastructure only.  It is not the oracle and no expected value comes
from it: the oracle computes every expected output.  The model serves two
purposes: checking the kernels' arithmetic design on the CPU (each step is
the recurrence mod p and stays in its lazy range; each strip extraction is
floor(2^v z / p)), and finding states whose next values land in the kernels'
lazy ranges or on strip boundaries, which the GPU parity tests then import.
"""
M32 = (1 << 32) - 1
M64 = (1 << 64) - 1

# generator: (k, q, p, t, v, s, lazy bound: every value the kernel keeps is below p + SLACK)
PARAMS = {
    "GM19": (15, 28, (1 << 19) - 1, 0, 1, 32, 72),
    "GM29": (4, 2, (1 << 29) - 3, 0, 1, 32, 24),
    "GM31": (11, 14, (1 << 31) - 1, 0, 1, 32, 40),
    "GM55": (256, 176, (1 << 51) - 129, 4, 4, 8, 129 << 10),
    "GM61": (24, 74, (1 << 61) - 1, 0, 1, 32, 1 << 40),
    "GQ58_1": (8, 48, (1 << 29) - 3, 29, 1, 32, 312),
    "GQ58_3": (8, 48, (1 << 29) - 3, 29, 3, 12, 312),
    "GQ58_4": (8, 48, (1 << 29) - 3, 29, 4, 8, 312),
}


def _mad32(a, b, c):
    return (a * b + c) & M32


def step(gen, z, y):
    """One step of the kernel on (z, z_prev) -> z' (lazy), for every generator
    but GM61 (whose kernel runs on the rotated values; see gm61_step)."""
    if gen == "GM19":
        a = _mad32(y, 0xFFFFFFE4, 29360072)
        a = _mad32(z, 15, a)
        h = a >> 19
        return _mad32(h, 0xFFF80001, a)
    if gen == "GM29":
        a = _mad32(y, 0xFFFFFFFE, 1610612727)
        a = _mad32(z, 4, a)
        h = a >> 29
        return _mad32(h, 0xE0000003, a)
    if gen == "GM31":
        t = (0xFFFFFFFE - y) & M32
        S = (t * 14 + z * 11) & M64
        lo, hi = S & M32, S >> 32
        h = (((hi << 32) | lo) >> 31) & M32
        return _mad32(h, 0x80000001, lo)
    if gen.startswith("GQ58"):
        t = (1073741818 - y) & M32
        S = (t * 48 + z * 8) & M64
        lo, hi = S & M32, S >> 32
        h = (((hi << 32) | lo) >> 29) & M32
        return _mad32(h, 0xE0000003, lo)
    if gen == "GM55":
        y0, y1, z0, z1 = y & M32, y >> 32, z & M32, z >> 32
        d0 = 0xFFFFFEFE - y0
        t0, borrow = d0 & M32, 1 if d0 < 0 else 0
        t1 = (0x000FFFFF - y1 - borrow) & M32
        U = (t0 * 176 + z0 * 256) & M64
        a0, a1 = U & M32, U >> 32
        a1 = _mad32(t1, 176, a1)
        s1 = _mad32(z1, 256, a1)
        h = s1 >> 19
        r = h * 129 + a0
        r0, carry = r & M32, r >> 32
        r1 = ((s1 & 0x7FFFF) + carry) & M32
        return (r1 << 32) | r0
    raise ValueError(gen)


P61 = (1 << 61) - 1


def gm61_enter(z):
    c = z - P61 if z >= P61 else z
    return (((c << 1) & P61) | (c >> 60)) + 1


def gm61_leave(u):
    w = u - 1
    if w >= P61:
        w -= P61
    return (w >> 1) | ((w & 1) << 60)


def gm61_step(u, up):
    """The GM61 kernel step on the rotated values: (u, u_prev) -> (u', bit).
    The high product B' = 74 t1 + 24 u1 is formed without the low product's
    carry word a1, which is added after the fold."""
    u0, u1, v0, v1 = u & M32, u >> 32, up & M32, up >> 32
    d0 = 0xEB3E4530 - v0
    t0, borrow = d0 & M32, 1 if d0 < 0 else 0
    t1 = (0x23E45306 - v1 - borrow) & M32
    A = (t0 * 74 + u0 * 24) & M64
    a0, a1 = A & M32, A >> 32
    B = (u1 * 24 + t1 * 74) & M64
    b0, b1 = B & M32, B >> 32
    h = (((b1 << 32) | b0) >> 29) & M32
    m = _mad32(h, 0xE0000000, b0)
    r = a0 + h
    r0, carry = r & M32, r >> 32
    r1 = (m + a1 + carry) & M32
    bit = ((((r0 << 29) & M32) ^ (~r1 & M32)) & 0x20000000) != 0
    return (r1 << 32) | r0, bit


def strip1(gen, z):
    """The v = 1 output bit as the kernel tests it (lazy z)."""
    p = PARAMS[gen][2]
    half = (p + 1) // 2
    return ((z - half) & M32) < (p - half)


def strip_insert(gen, i, z, w=0):
    """Point i's strip placed at bit v i of w, as the v = 3, 4 kernels do it."""
    v = PARAMS[gen][4]
    pos = v * i
    if pos >= 32:
        return w
    if gen == "GM55":
        q0 = (z >> 47) & M32
        X = (((z << 4) & M64) + ((129 * q0 + 129) & M32)) & M64
        hi = X >> 32
        x = hi >> (19 - pos) if pos <= 19 else (hi << (pos - 19)) & M32
        return (x & (15 << pos)) | w
    # p = 2^29 - 3: the kernel works in 32 bits, on X mod 2^32 (v = 3) or
    # X / 2 mod 2^32 (v = 4), X = 2^v z + 3 (q0 + 1)
    q0 = z >> (29 - v)
    top = 28 if v == 4 else 29
    x = (8 * z + ((3 * q0 + 3) >> 1 if v == 4 else 3 * q0 + 3)) & M32
    y = x >> (top - pos) if pos <= top else (x << (pos - top)) & M32
    mask = (((1 << v) - 1) << pos) if pos + v <= 32 else (M32 << pos) & M32
    return (y & mask) | w


def next_lazy(gen, z, y):
    """(value the kernel computes, exact canonical value) of the step from the
    canonical pair (z, z_prev) = (z, y)."""
    k, q, p = PARAMS[gen][:3]
    exact = (k * z - q * y) % p
    if gen == "GM61":
        u, _ = gm61_step(gm61_enter(z), gm61_enter(y))
        return u, exact
    return step(gen, z, y), exact


# ---------------------------------------------------------------- state search

def _inv(a, p):
    return pow(a % p, -1, p)


def solve_prev(gen, z, target):
    """z_prev such that the exact next value (k z - q z_prev mod p) is target."""
    k, q, p = PARAMS[gen][:3]
    return ((k * z - target) * _inv(q, p)) % p


def lazy_states(gen, count, rng):
    """`count` canonical pairs (z, z_prev) whose next value, as the kernel
    computes it, lies in the lazy range (>= p; for GM61 the rotated value
    >= 2^61, the XNOR branch of the output bit).  The exact next value is a
    small residue e, which the kernel keeps as e + p when the fold leaves a
    high part it does not subtract (shown by the model for each pair)."""
    k, q, p, t, v, s, slack = PARAMS[gen]
    out = []
    for _ in range(200000):
        if len(out) == count:
            break
        z = int(rng.integers(0, p))
        if gen == "GM61":
            e = int(rng.integers(0, 40))          # u' = 2 e + 1
            y = solve_prev(gen, z, e)
            u, _ = gm61_step(gm61_enter(z), gm61_enter(y))
            if u >= 1 << 61:
                out.append((z, y))
        else:
            e = int(rng.integers(0, min(slack, p)))
            y = solve_prev(gen, z, e)
            if step(gen, z, y) >= p:
                out.append((z, y))
    if len(out) < count:
        raise RuntimeError(f"{gen}: found {len(out)} lazy states of {count}")
    return out


def strip_boundaries(gen):
    """Canonical values on either side of every strip boundary of
    floor(2^v z / p), plus 0 and p - 1."""
    p, v = PARAMS[gen][2], PARAMS[gen][4]
    vals = {0, p - 1}
    for j in range(1, 1 << v):
        b = -(-j * p >> v)  # ceil(j p / 2^v): the first value of strip j
        vals |= {b - 1, b}
    return sorted(vals)


def boundary_states(gen, rng):
    """Canonical pairs (z, z_prev) whose exact next value is each strip
    boundary value in turn."""
    p = PARAMS[gen][2]
    out = []
    for target in strip_boundaries(gen):
        z = int(rng.integers(0, p))
        out.append((z, solve_prev(gen, z, target)))
    return out
