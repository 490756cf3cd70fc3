"""The single-stream functions of include/prand_device.h (the paper's
single-threaded interface, Sec. 7.3), compiled for the host: from a stream's
oracle state they produce the oracle's outputs, integer and float, bit for
bit."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1307_5869_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN_ID = {g: i for i, g in enumerate(W.GENERATORS)}


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    so = str(tmp_path_factory.mktemp("devapi") / "shim.so")
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "device_api_shim.cpp"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.dev_api_run.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_ulonglong]
    return L


def device_struct(gen, raw: bytes) -> bytearray:
    """The oracle's state bytes in the prand_device.h layout."""
    if gen == "MRG32K3A":  # oracle: uint64 x[3], y[3]; device: uint32 x[3], y[3]
        w = np.frombuffer(raw, dtype=np.uint64)
        return bytearray(w.astype(np.uint32).tobytes())
    return bytearray(raw)  # MT19937 {mt[624], idx}, LFSR113 {z[4]}, GM/GQ {x_prev[32], x[32]} already match


@pytest.mark.parametrize("gen", W.GENERATORS)
@pytest.mark.parametrize("kind", ["u32", "f32", "f64"])
def test_single_stream_functions_follow_the_oracle(shim, gen, kind):
    n = 1000 if gen.startswith(("GM", "GQ")) else 3000  # MT19937: several twists
    for seed, k in ((W.TABLE_SEED, 0), (W.TABLE_SEED, 7), (O.SEED_DEFAULT, 3)):
        st = O.State.stream(gen, seed, k)
        buf = (ctypes.c_char * 4096).from_buffer(device_struct(gen, st.raw()) + bytearray(4096))
        want = getattr(st.copy(), kind)(n)
        got = np.empty(n, dtype={"u32": np.uint32, "f32": np.float32, "f64": np.float64}[kind])
        assert shim.dev_api_run(GEN_ID[gen], ctypes.addressof(buf), ["u32", "f32", "f64"].index(kind), got.ctypes.data, n) == 0
        bits = {"u32": np.uint32, "f32": np.uint32, "f64": np.uint64}[kind]
        assert np.array_equal(got.view(bits), want.view(bits)), (gen, seed, k)
