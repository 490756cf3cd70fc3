"""Single-stream generation in user device code: a handle's streams exported
as prand_device.h states, advanced by a user kernel (one thread per stream)
and imported back.  The user kernel's outputs equal the handle's own fills,
and the handle continues exactly where the user code left the streams."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1307_5869_gb300 as P  # noqa: E402
from paper_1307_5869_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kern(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    so = str(tmp_path_factory.mktemp("devapi") / "kern.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "device_api_kernel.cu"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.dev_api_kernel.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_ulonglong]
    return L


@pytest.mark.parametrize("gen", W.GENERATORS)
def test_export_advance_import(kern, gen):
    P.load()
    n = 192
    m = 700 if not gen.startswith(("GM", "GQ")) else 40
    a, b = P.prand_create(gen, 99), P.prand_create(gen, 99)
    try:
        P.prand_init_streams(a, 5, n)
        P.prand_init_streams(b, 5, n)
        # both handles first fill a ragged stretch (the export starts mid-block)
        for h in (a, b):
            t = torch.empty(n * 37, dtype=torch.int32, device="cuda")
            P.prand_generate_u32(h, t.data_ptr(), 37, 0)
        sb = P.prand_device_state_bytes(gen)
        states = torch.zeros(n * sb // 4 + 2, dtype=torch.int32, device="cuda")
        P.prand_export_states(a, states.data_ptr(), 0)
        torch.cuda.synchronize()
        user = torch.empty(n * m, dtype=torch.int32, device="cuda")
        assert kern.dev_api_kernel(W.GENERATORS.index(gen), states.data_ptr(), n, user.data_ptr(), m) == 0
        ref = torch.empty(n * m, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(b, ref.data_ptr(), m, 0)
        torch.cuda.synchronize()
        assert torch.equal(user, ref)
        P.prand_import_states(a, states.data_ptr(), 0)
        c1 = torch.empty(n * 333, dtype=torch.int32, device="cuda")
        c2 = torch.empty(n * 333, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(a, c1.data_ptr(), 333, 0)
        P.prand_generate_u32(b, c2.data_ptr(), 333, 0)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2)
    finally:
        P.prand_destroy(a)
        P.prand_destroy(b)


def test_mt_import_rejects_mixed_positions():
    P.load()
    n = 4
    h = P.prand_create("MT19937", 1)
    try:
        P.prand_init_streams(h, 0, n)
        sb = P.prand_device_state_bytes("MT19937")
        assert sb == 625 * 4
        states = torch.zeros(n * sb // 4, dtype=torch.int32, device="cuda")
        P.prand_export_states(h, states.data_ptr(), 0)
        host = states.cpu()
        host[1 * 625 + 624] = 3  # stream 1 at another in-block position
        states.copy_(host)
        before = torch.empty(n * 10, dtype=torch.int32, device="cuda")
        with pytest.raises(P.PrandError):
            P.prand_import_states(h, states.data_ptr(), 0)
        # nothing changed: the handle still produces its own next outputs
        twin = P.prand_create("MT19937", 1)
        P.prand_init_streams(twin, 0, n)
        ref = torch.empty(n * 10, dtype=torch.int32, device="cuda")
        P.prand_generate_u32(h, before.data_ptr(), 10, 0)
        P.prand_generate_u32(twin, ref.data_ptr(), 10, 0)
        torch.cuda.synchronize()
        assert torch.equal(before, ref)
        P.prand_destroy(twin)
    finally:
        P.prand_destroy(h)
