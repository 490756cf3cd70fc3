"""Host SIMD generation against the GPU (on the GPU machine the host code is the
AArch64 NEON build): streams exported from a handle (prand_export_states) and
filled on the host equal the GPU's fill of the same streams, bit for bit, and
the states the host leaves behind equal the handle's."""
import numpy as np
import pytest

import paper_1307_5869_gb300 as P

pytestmark = pytest.mark.gpu
TDT = {"u32": "int32", "f32": "float32", "f64": "float64"}
BITS = {"u32": np.uint32, "f32": np.uint32, "f64": np.uint64}
DTYPE = {"u32": 0, "f32": 1, "f64": 2}


@pytest.mark.parametrize("gen", ["MT19937", "LFSR113", "MRG32K3A"])
@pytest.mark.parametrize("dt", ["u32", "f32", "f64"])
def test_host_simd_equals_gpu_fill(gen, dt):
    import torch
    P.load(build_if_missing=True)
    n = 1027
    g = P.Generator(gen, 99, 123456, n)
    g.generate(333, "u32")  # mid-block MT19937 positions, continued states
    sb = P.prand_device_state_bytes(gen)
    dev = torch.empty(n * sb // 4, dtype=torch.int32, device="cuda")
    P.prand_export_states(g.h, dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    structs = dev.cpu().numpy().copy()
    for nper in (1000, 77):
        want = g.generate(nper, dt).cpu().numpy()
        out = np.zeros(n * nper, dtype=getattr(np, TDT[dt]))
        P.prand_host_generate(gen, DTYPE[dt], structs.ctypes.data, n, out.ctypes.data, nper, 0)
        assert np.array_equal(out.view(BITS[dt]).reshape(n, nper), want.view(BITS[dt])), f"{gen} {dt} {nper}"
    P.prand_export_states(g.h, dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), structs)
    g.close()
