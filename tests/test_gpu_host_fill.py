"""Host-array fills (prand_generate_host_*) through the C ABI: the outputs
equal a device fill of an identical handle and the oracle, and the streams
continue exactly afterwards.  The shapes drive the blocking: several stream
blocks sharing one section split (more than 65536 streams), many output blocks
(small staging), MT19937's in-block position, pageable and page-locked memory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
import paper_1307_5869_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

TDT = {"u32": torch.int32, "f32": torch.float32, "f64": torch.float64}
NDT = {"u32": np.uint32, "f32": np.float32, "f64": np.float64}
BITS = {"u32": np.uint32, "f32": np.uint32, "f64": np.uint64}
HOST = {"u32": P.prand_generate_host_u32, "f32": P.prand_generate_host_f32, "f64": P.prand_generate_host_f64}
DEV = {"u32": P.prand_generate_u32, "f32": P.prand_generate_f32, "f64": P.prand_generate_f64}

CASES = [
    # gen, streams, outputs per stream, dtype, staging bytes (None: default), page-locked
    ("MRG32K3A", 70000, 2048, "u32", None, True),
    ("LFSR113", 70000, 2048, "f32", None, False),
    ("MRG32K3A", 5, 100000, "f64", 1 << 16, True),
    ("MT19937", 3000, 1000, "u32", 1 << 16, True),
    ("MT19937", 700, 1500, "f64", None, False),
    ("GM61", 3000, 1000, "f32", 1 << 16, True),
    ("GQ58_3", 1000, 777, "u32", 1 << 16, False),
    ("GM19", 9, 50000, "u32", 1 << 16, True),
]


def _host_array(n, dt, pinned):
    if pinned:
        return torch.empty(n, dtype=TDT[dt], pin_memory=True)
    return torch.from_numpy(np.empty(n, dtype=NDT[dt]).view(np.int32) if dt == "u32" else np.empty(n, dtype=NDT[dt]))


@pytest.mark.parametrize("gen,n,nper,dt,stage,pinned", CASES,
                         ids=[f"{c[0]}-{c[1]}x{c[2]}-{c[3]}-{'pin' if c[5] else 'page'}" for c in CASES])
def test_host_fill_equals_device_fill_and_oracle(gen, n, nper, dt, stage, pinned, monkeypatch):
    P.load()
    if stage is not None:
        monkeypatch.setenv("PRAND_HOST_STAGE_BYTES", str(stage))
    else:
        monkeypatch.delenv("PRAND_HOST_STAGE_BYTES", raising=False)
    seed = 4242
    a, b = P.prand_create(gen, seed), P.prand_create(gen, seed)
    try:
        P.prand_init_streams(a, 0, n)
        P.prand_init_streams(b, 0, n)
        host = _host_array(n * nper, dt, pinned)
        HOST[dt](a, host.data_ptr(), nper, 0)
        dev = torch.empty(n * nper, dtype=TDT[dt], device="cuda")
        DEV[dt](b, dev.data_ptr(), nper, 0)
        got = host.numpy().view(BITS[dt])
        want = dev.cpu().numpy().view(BITS[dt])
        assert np.array_equal(got, want)
        # oracle on a few streams, including block edges
        st = O.Streams(gen, seed, 0, n)
        for j in sorted({0, 1, n // 2, min(n - 1, 65535), min(n - 1, 65536), n - 1}):
            o = getattr(st.state(j), dt)(nper)
            assert np.array_equal(got[j * nper:(j + 1) * nper], o.view(BITS[dt])), j
        # the streams continue exactly: one more fill on both handles
        m = 333
        d1 = torch.empty(n * m, dtype=torch.int32, device="cuda")
        d2 = torch.empty(n * m, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(a, d1.data_ptr(), m, 0)
        P.prand_generate_u32(b, d2.data_ptr(), m, 0)
        assert torch.equal(d1, d2)
        assert P.prand_query(a) == P.prand_query(b)
    finally:
        P.prand_destroy(a)
        P.prand_destroy(b)


def test_host_fill_errors():
    P.load()
    h = P.prand_create("LFSR113", 1)
    try:
        buf = np.zeros(16, dtype=np.float64)
        with pytest.raises(P.PrandError):  # no streams yet
            P.prand_generate_host_f64(h, buf.ctypes.data, 2, 0)
        P.prand_init_streams(h, 0, 4)
        with pytest.raises(P.PrandError):  # misaligned host pointer
            P.prand_generate_host_f64(h, buf.ctypes.data + 4, 2, 0)
        with pytest.raises(P.PrandError):
            P.prand_generate_host_u32(h, 0, 2, 0)
        P.prand_generate_host_f64(h, buf.ctypes.data, 0, 0)  # nothing to do
        P.prand_generate_host_f64(h, buf.ctypes.data, 4, 0)
        assert np.all((buf >= 0) & (buf < 1))
    finally:
        P.prand_destroy(h)


@pytest.mark.parametrize("gen", ["LFSR113", "GM55", "MT19937"])
def test_host_fill_into_page_locked_interior_and_registered_memory(gen):
    # page-locked memory is written by the kernels directly: an interior
    # pointer of a page-locked allocation (4-byte but not 16-byte aligned, so
    # the scalar store forms run on host memory) and a pageable numpy array
    # registered with cudaHostRegister both equal a device fill
    P.load()
    n, nper, seed = 300, 1001, 77
    a, b, c = (P.prand_create(gen, seed) for _ in range(3))
    try:
        for h in (a, b, c):
            P.prand_init_streams(h, 5, n)
        pinned = torch.zeros(n * nper + 8, dtype=torch.int32, pin_memory=True)
        P.prand_generate_host_u32(a, pinned.data_ptr() + 3 * 4, nper, 0)
        dev = torch.empty(n * nper, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(b, dev.data_ptr(), nper, 0)
        want = dev.cpu().numpy().view(np.uint32)
        got = pinned.numpy().view(np.uint32)
        assert np.array_equal(got[3:3 + n * nper], want)
        assert not got[:3].any() and not got[3 + n * nper:].any()  # nothing outside the array
        arr = np.zeros(n * nper, dtype=np.uint32)
        rt = torch.cuda.cudart()
        assert int(rt.cudaHostRegister(arr.ctypes.data, arr.nbytes, 0)) == 0
        try:
            P.prand_generate_host_u32(c, arr.ctypes.data, nper, 0)
        finally:
            rt.cudaHostUnregister(arr.ctypes.data)
        assert np.array_equal(arr, want)
    finally:
        for h in (a, b, c):
            P.prand_destroy(h)
