"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Every comparison is bit-exact: u32 outputs as integers, f32/f64 outputs with
0 ulp (compared as raw bit patterns).  Inputs are seeded and synthetic.
"""
import numpy as np
import pytest

import oracle as O
import paper_1307_5869_gb300 as P

pytestmark = pytest.mark.gpu

GENS = P.GENERATORS
NPDT = {"u32": np.uint32, "f32": np.uint32, "f64": np.uint64}


def _bits(a: np.ndarray, dt: str) -> np.ndarray:
    return np.ascontiguousarray(a).view(NPDT[dt])


def _gpu(t) -> np.ndarray:
    return t.cpu().numpy()


def _assert_same(got, ref, dt, what=""):
    g = _bits(got, dt)
    r = _bits(ref, dt)
    assert g.shape == r.shape, (what, g.shape, r.shape)
    if not np.array_equal(g, r):
        bad = np.argwhere(g != r)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {i}: got {g[i]:#x} want {r[i]:#x}")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    P.load(build_if_missing=True)
    torch.cuda.init()
    yield


@pytest.mark.parametrize("dt", ["u32", "f32", "f64"])
@pytest.mark.parametrize("gen", GENS)
def test_ragged_chunks_many_streams(gen, dt):
    # 37 streams starting at stream 3, consecutive calls of ragged lengths
    g = P.Generator(gen, 12345, 3, 37)
    ref = O.Streams(gen, 12345, 3, 37)
    for n in (1, 5, 127, 4097):
        _assert_same(_gpu(g.generate(n, dt)), ref.generate(dt, n), dt, f"{gen} {dt} chunk {n}")
    g.close()


@pytest.mark.parametrize("dt", ["u32", "f32", "f64"])
@pytest.mark.parametrize("gen", GENS)
def test_aligned_chunks_vector_stores(gen, dt):
    # lengths that are multiples of 4 keep every row 16-byte aligned: the vector
    # and staged-row store paths (the ragged test above covers the scalar ones)
    g = P.Generator(gen, 31, 5, 300)
    ref = O.Streams(gen, 31, 5, 300)
    for n in (64, 1000, 4096):
        _assert_same(_gpu(g.generate(n, dt)), ref.generate(dt, n), dt, f"{gen} {dt} chunk {n}")
    g.close()


@pytest.mark.parametrize("gen", GENS)
def test_long_sections_and_continuation(gen):
    # few streams, long outputs: one stream is split into sections reached by jumps
    nper = 20000 if gen != "MT19937" else 5000
    g = P.Generator(gen, 777, 0, 2)
    ref = O.Streams(gen, 777, 0, 2)
    for n in (nper, 777, 3 * nper + 1):
        _assert_same(_gpu(g.generate(n, "u32")), ref.generate("u32", n), "u32", f"{gen} n={n}")
    g.close()


def test_mrg32k3a_default_state_one_stream_2_pow_20():
    # one stream of MRG32K3A from the paper's default state, 2^20 outputs as u32 and f64
    n = 1 << 20
    for dt in ("u32", "f64"):
        g = P.Generator("MRG32K3A", P.SEED_DEFAULT, 0, 1)
        got = _gpu(g.generate(n, dt))
        g.close()
        ref = O.State("MRG32K3A")
        want = ref.u32(n) if dt == "u32" else ref.f64(n)
        _assert_same(got.reshape(-1), want, dt, f"MRG32K3A default {dt}")
        if dt == "f64":
            assert (got > 0).all() and (got < 1).all()


@pytest.mark.parametrize("gen", GENS)
def test_skipahead_offsets(gen):
    g = P.Generator(gen, 4242, 10, 5)
    states = [O.State.stream(gen, 4242, 10 + j) for j in range(5)]
    got = _gpu(g.generate(100, "u32"))
    want = np.stack([s.u32(100) for s in states])
    _assert_same(got, want, "u32", f"{gen} pre-skip")
    for off in (1, 523, 624, 10**6 + 3, 2**100 + 7):
        g.skipahead(off)
        for s in states:
            s.jump(off)
        got = _gpu(g.generate(300, "u32"))
        want = np.stack([s.u32(300) for s in states])
        _assert_same(got, want, "u32", f"{gen} after skip {off}")
    g.close()


@pytest.mark.parametrize("gen", GENS)
def test_state_checkpoint_resume(gen):
    a = P.Generator(gen, 99, 1, 4)
    a.generate(333, "u32")
    blob = a.get_state()
    cont = _gpu(a.generate(500, "u32"))
    b = P.Generator(gen, 1, 0, 1)
    b.set_state(blob)
    _assert_same(_gpu(b.generate(500, "u32")), cont, "u32", f"{gen} resume")
    a.close()
    b.close()


@pytest.mark.parametrize("gen", GENS)
def test_misaligned_output_scalar_path(gen):
    import torch
    g = P.Generator(gen, 5, 0, 3)
    ref = O.Streams(gen, 5, 0, 3)
    buf = torch.zeros(3 * 1001 + 1, dtype=torch.int32, device="cuda")
    out = buf[1:]  # 4-byte aligned, not 16-byte aligned
    P.prand_generate_u32(g.h, out.data_ptr(), 1001, torch.cuda.current_stream().cuda_stream)
    got = _gpu(out).reshape(3, 1001)
    _assert_same(got, ref.generate("u32", 1001), "u32", f"{gen} misaligned")
    assert int(_gpu(buf)[0]) == 0  # nothing written before the output
    g.close()


def test_error_paths_on_device():
    import torch
    L = P.load()
    import ctypes
    h = ctypes.c_void_p()
    assert L.prand_create(ctypes.byref(h), 1, 1) == 0
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    assert L.prand_generate_u32(h, buf.data_ptr(), 4, None) == 5          # no streams yet
    assert L.prand_init_streams(h, 0, 0) == 1                              # zero streams
    assert L.prand_init_streams(h, 2**64 - 1, 2) == 1                      # index overflow
    assert L.prand_init_streams(h, 0, 4) == 0
    assert L.prand_generate_u32(h, buf.data_ptr() + 1, 4, None) == 2      # misaligned
    assert L.prand_generate_f64(h, buf.data_ptr() + 4, 2, None) == 2      # f64 needs 8 bytes
    assert L.prand_generate_u32(h, buf.data_ptr(), 0, None) == 0           # no-op
    assert L.prand_init_streams(h, 10**19 - 1, 2) == 7                     # beyond Table 4
    assert L.prand_destroy(h) == 0


@pytest.mark.parametrize("gen", ["MT19937", "MRG32K3A", "LFSR113", "GM61"])
def test_refused_allocation_reports_nomem_and_leaves_no_error(gen):
    # 2^38 streams need terabytes of state: the allocation is refused and
    # reported as PRAND_ERR_NOMEM, the handle holds no streams, and the calls
    # after it succeed (the refused allocation leaves no CUDA error behind for
    # a later launch check to report)
    import ctypes
    import torch
    L = P.load()
    h = ctypes.c_void_p()
    assert L.prand_create(ctypes.byref(h), P.GENERATORS.index(gen), 9) == 0
    buf = torch.zeros(4 * 300, dtype=torch.int32, device="cuda")
    assert L.prand_init_streams(h, 0, 1 << 38) == 3
    assert L.prand_generate_u32(h, buf.data_ptr(), 300, None) == 5
    assert L.prand_init_streams(h, 2, 4) == 0
    assert L.prand_generate_u32(h, buf.data_ptr(), 300, None) == 0
    torch.cuda.synchronize()
    _assert_same(_gpu(buf).reshape(4, 300), O.Streams(gen, 9, 2, 4).generate("u32", 300), "u32", f"{gen} after NOMEM")
    assert L.prand_destroy(h) == 0


def test_refused_server_arena_reports_nomem():
    import ctypes
    L = P.load()
    srv = ctypes.c_void_p()
    assert L.prand_server_create(ctypes.byref(srv), ctypes.c_uint64(3), ctypes.c_uint64(1 << 52), 4) == 3
    assert not srv.value
    # a server of ordinary size still works afterwards
    s = P.prand_server_create(3, 64 << 20, 4)
    try:
        rid = P.prand_server_submit(s, "LFSR113", 11, 500, 0)
        import time
        t0 = time.time()
        while not P.prand_server_query(s, rid)[0]:
            assert time.time() - t0 < 60, "request did not complete"
            time.sleep(0.001)
        out = np.empty(500, dtype=np.int32)
        P.prand_server_read(s, rid, out)
    finally:
        P.prand_server_destroy(s)
    _assert_same(out, O.State.stream("LFSR113", 3, 11).u32(500), "u32", "server after NOMEM")


@pytest.mark.parametrize("gen", GENS)
def test_extreme_stream_indices(gen):
    # the largest stream indices the ABI accepts (beyond Table 4, so the call
    # warns): the jump offset (first + j) L needs up to 64 + log2(L) bits,
    # 2^496 for MT19937
    for seed, first, n, dt in ((12345, 2**64 - 3, 2, "u32"), (7, 10**19 - 1, 1, "f64")):
        g = P.Generator(gen, seed, first, n)
        _assert_same(_gpu(g.generate(64, dt)), O.Streams(gen, seed, first, n).generate(dt, 64), dt,
                     f"{gen} streams {first}..{first + n - 1}")
        g.close()


def _sample_streams(gen, n, rng, count=1024):
    """Stream indices to compare at full size: the first and last streams,
    those on both sides of every power-of-two boundary (thread blocks, warps,
    sections of the launch grid), and random ones, `count` in all.  MT19937
    takes runs of 64 consecutive streams (the oracle reaches a run's first
    stream by one jump and each next one by L more)."""
    if gen == "MT19937":
        runs = count // 64
        starts = {0, n - 64, n // 2 - 32}
        while len(starts) < runs:
            starts.add(int(rng.integers(0, n // 64)) * 64)
        return sorted(k for a in starts for k in range(a, a + 64))
    ks = {0, 1, 2, n - 2, n - 1}
    b = 2
    while b < n:
        ks |= {b - 1, b}
        b *= 2
    while len(ks) < count:
        ks.add(int(rng.integers(0, n)))
    return sorted(ks)


def _oracle_rows(gen, seed, ks, nper, dts):
    """Oracle outputs of streams ks (u32 then each later dtype continuing)."""
    out = {dt: [] for dt in dts}
    if gen == "MT19937":
        for a in range(0, len(ks), 64):
            assert ks[a + 63] == ks[a] + 63
            st = O.Streams(gen, seed, ks[a], 64)
            for dt in dts:
                out[dt].append(st.generate(dt, nper))
        return {dt: np.concatenate(v) for dt, v in out.items()}
    for k in ks:
        st = O.State.stream(gen, seed, k)
        for dt in dts:
            out[dt].append(getattr(st, dt)(nper))
    return {dt: np.stack(v) for dt, v in out.items()}


@pytest.mark.parametrize("gen", GENS)
def test_table4_streams_2_pow_16_by_2_pow_12_sampled(gen):
    # all eleven generators, 2^16 block-split streams x 2^12 outputs; u32, then
    # f32 from a fresh identical handle; seed 12345; 1024 sampled streams
    # against the oracle's stream k = base + k * L
    import torch
    n, nper = 1 << 16, 1 << 12
    ks = _sample_streams(gen, n, np.random.default_rng(2024))
    assert len(ks) >= 1024
    ref = _oracle_rows(gen, 12345, ks, nper, ["u32"])["u32"]
    idx = torch.tensor(ks, device="cuda")
    for dt in ("u32", "f32"):
        g = P.Generator(gen, 12345, 0, n)
        out = g.generate(nper, dt)
        got = _gpu(out[idx])
        g.close()
        del out
        want = ref if dt == "u32" else O.convert(ref.reshape(-1), "f32").reshape(ref.shape)
        _assert_same(got, want, dt, f"{gen} {dt} sampled")


@pytest.mark.parametrize("gen", ["MT19937", "LFSR113", "GM61"])
def test_bulk_2_pow_20_streams_sampled(gen):
    # 2^20 streams x 2^10 (2^30 outputs), u32 then f32 continuing; seed from a
    # 64-bit counter; 1024 sampled streams
    import torch
    n, nper = 1 << 20, 1 << 10
    seed = 0x9E3779B97F4A7C15
    ks = _sample_streams(gen, n, np.random.default_rng(7))
    assert len(ks) >= 1024
    g = P.Generator(gen, seed, 0, n)
    idx = torch.tensor(ks, device="cuda")
    u = g.generate(nper, "u32")
    gu = _gpu(u[idx])
    del u
    f = g.generate(nper, "f32")
    gf = _gpu(f[idx])
    del f
    g.close()
    ref = _oracle_rows(gen, seed, ks, nper, ["u32", "f32"])
    _assert_same(gu, ref["u32"], "u32", f"{gen} u32 sampled")
    _assert_same(gf, ref["f32"], "f32", f"{gen} f32 sampled")


def test_batch_run_mixed_requests():
    import torch
    rng = np.random.default_rng(7)
    reqs, bufs, meta = [], [], []
    for i in range(24):
        gen = GENS[i % len(GENS)]
        dt = ["u32", "f32", "f64"][i % 3]
        k = int(rng.integers(0, 10**19, dtype=np.uint64))
        n = int(rng.integers(1, 3000))
        t = torch.empty(n, dtype={"u32": torch.int32, "f32": torch.float32, "f64": torch.float64}[dt], device="cuda")
        bufs.append(t)
        reqs.append((gen, {"u32": 0, "f32": 1, "f64": 2}[dt], k, n, t.data_ptr()))
        meta.append((gen, dt, k, n))
    P.prand_batch_run(reqs, 12345, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for t, (gen, dt, k, n) in zip(bufs, meta):
        st = O.State.stream(gen, 12345, k)
        _assert_same(_gpu(t), getattr(st, dt)(n), dt, f"batch {gen} {dt} stream {k}")
