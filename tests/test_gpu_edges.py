"""GPU parity at the method's edge cases, through the C ABI: states imported
into a handle (prand_import_states) whose next values land in the kernels'
lazy residue ranges or on the strip boundaries of the output map, and the
MRG32K3A states whose output is the degenerate z = m1 (x_n = y_n) or whose
components step to 0 or m - 1.  Every output is compared bit for bit with the
oracle continuing the same states.

The states are chosen on the CPU with a model of the kernels' limb arithmetic
(tests/kernel_model.py), which shows that each chosen state reaches the lazy
range (tests/test_kernel_model.py); random streams reach it about once in
2^30 (GM29) to 2^53 (GM61) point steps."""
import numpy as np
import pytest

import kernel_model as KM
import oracle as O
import paper_1307_5869_gb300 as P

pytestmark = pytest.mark.gpu

GM_GENS = list(KM.PARAMS)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    P.load(build_if_missing=True)
    torch.cuda.init()
    yield


def _gm_stream_states(gen, rng, n_streams):
    """n_streams GM/GQ states (x_prev, x per point) mixing lazy-range and
    strip-boundary pairs over the points, plus random canonical points."""
    k, q, p, t, v, s, slack = KM.PARAMS[gen]
    pairs = KM.lazy_states(gen, 3 * s, rng) + KM.boundary_states(gen, rng)
    rng.shuffle(pairs)
    streams = []
    for j in range(n_streams):
        pts = []
        for i in range(s):
            idx = j * s + i
            if idx < len(pairs):
                pts.append(pairs[idx])
            else:
                pts.append((int(rng.integers(0, p)), int(rng.integers(0, p))))
        # (z, z_prev) pairs -> (x_prev, x) = 2^t (z_prev, z)
        streams.append(([y << t for z, y in pts], [z << t for z, y in pts]))
    return streams


def _import(gen, structs_u64, n):
    import torch
    g = P.Generator(gen, 1, 0, n)
    dev = torch.from_numpy(structs_u64.view(np.int64)).cuda()
    P.prand_import_states(g.h, dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("dt", ["u32", "f32"])
@pytest.mark.parametrize("gen", GM_GENS)
def test_gm_lazy_ranges_and_strip_boundaries(gen, dt):
    rng = np.random.default_rng(20240 + GM_GENS.index(gen))
    n = 8
    states = _gm_stream_states(gen, rng, n)
    structs = np.zeros((n, 64), dtype=np.uint64)
    for j, (xp, x) in enumerate(states):
        structs[j, :len(xp)] = xp
        structs[j, 32:32 + len(x)] = x
    g = _import(gen, structs, n)
    # two calls: the first continues from the imported states (vector and
    # staged-row stores), the second from the states the first wrote back
    for nper in (256, 100):
        got = g.generate(nper, dt).cpu().numpy()
        want = []
        for j, (xp, x) in enumerate(states):
            st = O.gm_state_raw(gen, xp, x)
            want.append(getattr(st, dt)(nper))
            states[j] = O.gm_state_points(st)
        want = np.stack(want)
        gb, wb = got.view(np.uint32), want.view(np.uint32)
        bad = np.argwhere(gb != wb)
        assert bad.size == 0, f"{gen} {dt} n={nper}: {len(bad)} mismatches, first at {tuple(bad[0])}"
    g.close()


@pytest.mark.parametrize("gen", GM_GENS)
def test_gm_hand_worked_words_on_the_gpu(gen):
    # the oracle's hand-worked golden words (tests/golden/gm_words_worked.txt),
    # imported into the kernels
    import test_oracle_pins_external as T
    cases = [c for c in T.WORKED if c[0] == gen]
    if not cases:
        pytest.skip("no hand-worked word for this ensemble")
    for _, xp, x, word in cases:
        structs = np.zeros((1, 64), dtype=np.uint64)
        structs[0, :len(xp)] = xp
        structs[0, 32:32 + len(x)] = x
        g = _import(gen, structs, 1)
        got = g.generate(8, "u32").cpu().numpy().view(np.uint32)[0]
        g.close()
        assert int(got[0]) == word
        assert np.array_equal(got, O.gm_state_raw(gen, xp, x).u32(8))


def _mrg_edge_states(rng):
    """MRG32K3A states (x_n, x_{n-1}, x_{n-2}, y_n, y_{n-1}, y_{n-2}) whose next
    x and y are chosen: equal (output z = m1), 0, m - 1, 1."""
    m1, m2 = 4294967087, 4294944443
    a, b, c, d = 1403580, 810728, 527612, 1370589
    targets = [(5, 5), (m1 - 1, m1 - 1), (0, 0), (0, m2 - 1), (m1 - 1, 0), (1, 0), (0, 1), (m1 - 1, m2 - 1),
               (12345, 12345), (m2 - 1, m2 - 1)]
    out = []
    for tx, ty in targets:
        x1, y0 = int(rng.integers(1, m1)), int(rng.integers(1, m2))
        # x_{n+1} = a x_{n-1} - b x_{n-2}; y_{n+1} = c y_n - d y_{n-2}
        x2 = ((a * x1 - tx) * pow(b, -1, m1)) % m1
        y2 = ((c * y0 - ty) * pow(d, -1, m2)) % m2
        out.append([int(rng.integers(0, m1)), x1, x2, y0, int(rng.integers(0, m2)), y2])
    return out


@pytest.mark.parametrize("dt", ["u32", "f64"])
def test_mrg32k3a_degenerate_outputs(dt):
    rng = np.random.default_rng(99)
    st = _mrg_edge_states(rng)
    n = len(st)
    structs = np.array(st, dtype=np.uint32)
    import torch
    g = P.Generator("MRG32K3A", 1, 0, n)
    dev = torch.from_numpy(structs.view(np.int32).copy()).cuda()
    P.prand_import_states(g.h, dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = g.generate(64, dt).cpu().numpy()
    g.close()
    want = []
    for words in st:
        raw = np.array(words, dtype=np.uint64).tobytes()
        want.append(getattr(O.State("MRG32K3A", raw=raw), dt)(64))
    want = np.stack(want)
    w64 = want.view(np.uint32 if dt == "u32" else np.uint64)
    assert np.array_equal(got.view(w64.dtype), w64)
    if dt == "u32":
        assert int(got.view(np.uint32)[0, 0]) == 4294967087  # x = y: z = m1
    else:
        assert (got > 0).all() and (got < 1).all()
