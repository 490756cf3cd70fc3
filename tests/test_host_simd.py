"""Host SIMD generation (prand_host_generate, no GPU) against the oracle: the
MT19937, LFSR113 and MRG32K3A outputs of streams whose states come from the
oracle, bit for bit as u32, f32 and f64, over ragged stream counts (vector
tails), ragged lengths (MT19937 block edges, the 4-output transposes) and
thread counts, and the states left behind continue exactly."""
import numpy as np
import pytest

import oracle as O
import paper_1307_5869_gb300 as P

GENS = ["MT19937", "LFSR113", "MRG32K3A"]
BITS = {"u32": np.uint32, "f32": np.uint32, "f64": np.uint64}
NPDT = {"u32": np.uint32, "f32": np.float32, "f64": np.float64}
DTYPE = {"u32": 0, "f32": 1, "f64": 2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1307_5869_gb300 import build as B
    B.build()
    P.load()


def _device_structs(gen, states):
    """Oracle states -> the prand_device.h layout (one struct per stream)."""
    raw = [st.raw() for st in states]
    if gen == "MRG32K3A":  # oracle: six u64 words; struct: six u32
        return np.concatenate([np.frombuffer(r, dtype=np.uint64).astype(np.uint32) for r in raw])
    return np.concatenate([np.frombuffer(r, dtype=np.uint32) for r in raw]).copy()


def _host(gen, dt, structs, n, nper, threads):
    out = np.zeros(n * nper, dtype=NPDT[dt])
    P.prand_host_generate(gen, DTYPE[dt], structs.ctypes.data, n, out.ctypes.data, nper, threads)
    return out.reshape(n, nper)


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("n", [1, 3, 4, 5, 9, 37])
def test_host_simd_equals_oracle(gen, n):
    seed = 2024 + n
    states = [O.State.stream(gen, seed, 11 + j) for j in range(n)] if gen != "MT19937" else \
        [O.Streams(gen, seed, 11, n).state(j) for j in range(n)]
    structs = _device_structs(gen, states)
    for nper, dt, threads in ((1, "u32", 1), (5, "f32", 3), (623, "u32", 0), (626, "f64", 2), (1300, "u32", 1),
                              (4099, "f32", 0)):
        got = _host(gen, dt, structs, n, nper, threads)
        want = np.stack([getattr(st, dt)(nper) for st in states])
        assert np.array_equal(got.view(BITS[dt]), want.view(BITS[dt])), f"{gen} n={n} nper={nper} {dt}"


def test_host_simd_mrg32k3a_degenerate_output():
    # states whose next x and y are equal give z = m1, the largest output
    m1 = 4294967087
    a, b = 1403580, 810728
    x1 = 77777
    x2 = ((a * x1 - 5) * pow(b, -1, m1)) % m1
    y0 = 4242
    y2 = ((527612 * y0 - 5) * pow(1370589, -1, 4294944443)) % 4294944443
    words = np.array([9, x1, x2, y0, 8, y2] * 3, dtype=np.uint32)
    states = [O.State("MRG32K3A", raw=np.array([9, x1, x2, y0, 8, y2], dtype=np.uint64).tobytes()) for _ in range(3)]
    got = _host("MRG32K3A", "u32", words, 3, 50, 1)
    assert (got[:, 0] == m1).all()
    assert np.array_equal(got, np.stack([st.u32(50) for st in states]))


def test_host_simd_errors():
    L = P.load()
    buf = np.zeros(64, dtype=np.uint32)
    assert L.prand_host_generate(3, 0, buf.ctypes.data, 1, buf.ctypes.data, 4, 0) == 1   # GM19: not on the host
    assert L.prand_host_generate(2, 7, buf.ctypes.data, 1, buf.ctypes.data, 4, 0) == 1   # unknown dtype
    assert L.prand_host_generate(2, 0, buf.ctypes.data, 1, buf.ctypes.data, 4, -1) == 1  # negative threads
    assert L.prand_host_generate(2, 0, None, 1, buf.ctypes.data, 4, 0) == 1
    assert L.prand_host_generate(2, 2, buf.ctypes.data, 1, buf.ctypes.data + 4, 4, 0) == 2  # f64 needs 8-byte alignment
    assert L.prand_host_generate(2, 0, None, 0, None, 4, 0) == 0                         # nothing to do
    mt = np.zeros(625, dtype=np.uint32)
    mt[624] = 700
    assert L.prand_host_generate(0, 0, mt.ctypes.data, 1, buf.ctypes.data, 4, 0) == 5    # index beyond the block
