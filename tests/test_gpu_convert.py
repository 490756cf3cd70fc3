"""The float epilogue against the oracle on every 32-bit input: f32 =
(u >> 8) 2^-24, f64 = u 2^-32 and the MRG32K3A double map (one round-to-nearest
multiply), through the C ABI's prand_convert, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
import paper_1307_5869_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

CHUNK = 1 << 27
MAPS = [("f32", P.DTYPE_F32, np.float32, np.uint32), ("f64", P.DTYPE_F64, np.float64, np.uint64),
        ("mrg_f64", P.MAP_MRG_F64, np.float64, np.uint64)]


@pytest.mark.parametrize("kind,map_,dt,bits", MAPS, ids=[m[0] for m in MAPS])
def test_every_u32_input(kind, map_, dt, bits):
    P.load()
    tdt = torch.float32 if dt == np.float32 else torch.float64
    src = torch.empty(CHUNK, dtype=torch.int32, device="cuda")
    dst = torch.empty(CHUNK, dtype=tdt, device="cuda")
    for base in range(0, 1 << 32, CHUNK):
        u = np.arange(base, base + CHUNK, dtype=np.uint64).astype(np.uint32)
        src.copy_(torch.from_numpy(u.view(np.int32)))
        P.prand_convert(src.data_ptr(), CHUNK, map_, dst.data_ptr(), 0)
        got = dst.cpu().numpy().view(bits)
        want = O.convert(u, kind).view(bits)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (kind, hex(int(u[bad[0]])), got[bad[0]], want[bad[0]])


def test_scalar_path_and_tails():
    """Unaligned pointers (scalar path) and lengths that are not multiples of 4."""
    P.load()
    rng = np.random.default_rng(3)
    u = rng.integers(0, 1 << 32, size=4099, dtype=np.uint64).astype(np.uint32)
    src = torch.from_numpy(u.view(np.int32)).cuda()
    for kind, map_, dt, bits in MAPS:
        tdt = torch.float32 if dt == np.float32 else torch.float64
        for off_in, off_out, n in ((0, 0, 4099), (1, 0, 4098), (0, 1, 4098), (3, 2, 17), (0, 0, 3)):
            dst = torch.zeros(n + off_out, dtype=tdt, device="cuda")
            P.prand_convert(src.data_ptr() + 4 * off_in, n, map_, dst.data_ptr() + dst.element_size() * off_out, 0)
            got = dst.cpu().numpy()[off_out:].view(bits)
            want = O.convert(u[off_in:off_in + n], kind).view(bits)
            assert np.array_equal(got, want), (kind, off_in, off_out, n)
