"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/prand.h declares, and rejects
bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

import paper_1307_5869_gb300 as P
from paper_1307_5869_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "prand.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(prand_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert _declared() == sorted(P.EXPORTS)


def test_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for code in range(8):
        s = P.prand_status_string(code)
        assert s and s != "unknown status"
    assert P.prand_status_string(99) == "unknown status"


def test_argument_errors_without_device(lib):
    L = lib
    h = ctypes.c_void_p()
    assert L.prand_create(None, 0, 0) == 1                       # NULL out
    assert L.prand_create(ctypes.byref(h), 11, 0) == 1           # gen out of range
    assert L.prand_create(ctypes.byref(h), -1, 0) == 1
    assert L.prand_init_streams(None, 0, 1) == 1
    assert L.prand_generate_u32(None, None, 1, None) == 1
    assert L.prand_generate_f64(None, None, 1, None) == 1
    assert L.prand_skipahead(None, None) == 1
    n = ctypes.c_size_t(0)
    assert L.prand_get_state(None, None, ctypes.byref(n)) == 1
    assert L.prand_set_state(None, None, 0) == 1
    assert L.prand_query(None, None, None, None) == 1
    assert L.prand_destroy(None) == 0
    bad = (P.Request * 1)(P.Request(42, 0, 0, 1, 0))
    assert L.prand_batch_run(bad, 1, 0, None) == 1
    bad = (P.Request * 1)(P.Request(0, 7, 0, 1, 0))
    assert L.prand_batch_run(bad, 1, 0, None) == 1
    assert L.prand_batch_run(None, 0, 0, None) == 0              # empty batch
    vp = ctypes.c_void_p
    assert L.prand_convert(None, 1, 1, vp(0x1000), None) == 1    # NULL input
    assert L.prand_convert(vp(0x1000), 1, 7, vp(0x2000), None) == 1  # unknown map
    assert L.prand_convert(None, 0, 1, None, None) == 0           # nothing to do
    assert L.prand_convert(vp(0x1002), 4, 1, vp(0x2000), None) == 2  # input not 4-byte aligned
    assert L.prand_convert(vp(0x1000), 4, 2, vp(0x2004), None) == 2  # doubles not 8-byte aligned
    assert L.prand_export_states(None, vp(0x1000), None) == 1
    assert L.prand_import_states(None, vp(0x1000), None) == 1
    assert [L.prand_device_state_bytes(g) for g in range(11)] == [2500, 24, 16] + [512] * 8
    assert L.prand_device_state_bytes(11) == 0
    assert L.prand_init_streams_variant(None, 0, 0, 1) == 1
    assert L.prand_skipahead_pow2(None, 1, 0) == 1


def test_binding_raises_on_error(lib):
    with pytest.raises(P.PrandError):
        P._check(1, "prand_init_streams")
    assert P._check(7, "prand_init_streams", allow_warn=True) == 7
    with pytest.raises(ValueError):
        P.prand_skipahead(0, -1)


def _compile_alone(tmp_path, compiler, std, header, ext):
    import shutil
    import subprocess
    if not shutil.which(compiler):
        pytest.skip(f"{compiler} not found")
    src = tmp_path / f"only_{header.replace('.', '_')}.{ext}"
    src.write_text(f'#include "{header}"\nint main(void) {{ return 0; }}\n')
    res = subprocess.run([compiler, f"-std={std}", "-Wall", "-Werror", "-fsyntax-only",
                          "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


@pytest.mark.parametrize("std", ["c99", "c11"])
def test_prand_h_is_a_self_contained_c_header(tmp_path, std):
    # a C translation unit that includes only prand.h must compile: every type
    # the declarations use (streams included) comes from the header itself
    _compile_alone(tmp_path, "gcc", std, "prand.h", "c")


def test_prand_h_compiles_as_cpp(tmp_path):
    _compile_alone(tmp_path, "g++", "c++17", "prand.h", "cpp")


def test_prand_device_h_compiles_with_a_host_compiler(tmp_path):
    _compile_alone(tmp_path, "g++", "c++17", "prand_device.h", "cpp")


def test_mt_jump_polynomials_match_the_oracle(lib):
    # The library's host precomputation of x^(2^b) mod phi (Berlekamp-Massey,
    # then squarings reduced eight coefficients per pass from byte tables)
    # against the oracle's bit-serial squarings.  A wrong table entry, shift or
    # pass order changes every later power.
    import oracle as O
    for b in (0, 1, 2, 31, 432, 511):
        assert P.prand_mt_jump_polynomial(b) == O.mt_x_pow2k(b), b
    buf = (ctypes.c_uint32 * 624)()
    assert lib.prand_mt_jump_polynomial(512, ctypes.cast(buf, ctypes.c_void_p)) == 1
    assert lib.prand_mt_jump_polynomial(0, None) == 1
