"""Python binding of the prand C ABI (``include/prand.h``).

Argument marshalling only: every step of generation, jump-ahead and stream
initialisation runs in the CUDA kernels of ``libprand_gb300.so``.  There is no
CPU fallback; importing the binding without the built library raises.

The functions keep the C names.  Device buffers are passed as integer device
pointers (e.g. ``tensor.data_ptr()``) and streams as integer ``cudaStream_t``
handles (e.g. ``torch.cuda.current_stream().cuda_stream``).  ``Generator`` is
a small convenience wrapper over one handle that returns torch tensors.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libprand_gb300.so")

GENERATORS = ["MT19937", "MRG32K3A", "LFSR113", "GM19", "GM29", "GM31", "GM55",
              "GM61", "GQ58_1", "GQ58_3", "GQ58_4"]
GEN_ID = {g: i for i, g in enumerate(GENERATORS)}
SEED_DEFAULT = 2**64 - 1
DTYPE_U32, DTYPE_F32, DTYPE_F64 = 0, 1, 2

PRAND_OK = 0
PRAND_WARN_STREAM_OVERLAP = 7
STATUS = {0: "PRAND_OK", 1: "PRAND_ERR_ARG", 2: "PRAND_ERR_ALIGN", 3: "PRAND_ERR_NOMEM",
          4: "PRAND_ERR_CUDA", 5: "PRAND_ERR_STATE", 6: "PRAND_ERR_TIMEOUT",
          7: "PRAND_WARN_STREAM_OVERLAP"}

# Every symbol include/prand.h declares.
EXPORTS = ["prand_create", "prand_init_streams", "prand_generate_u32", "prand_generate_f32",
           "prand_generate_f64", "prand_skipahead", "prand_get_state", "prand_set_state",
           "prand_query", "prand_destroy", "prand_status_string", "prand_kernel_launches",
           "prand_batch_run", "prand_batch_run_per_request", "prand_batch_plan_create",
           "prand_batch_plan_launch", "prand_batch_plan_destroy", "prand_batch_autotune",
           "prand_mrg32k3a_generate_u32_noalloc", "prand_server_create", "prand_server_submit",
           "prand_server_query", "prand_server_read", "prand_server_completed", "prand_server_release", "prand_server_stats",
           "prand_server_destroy", "prand_server_replay", "prand_convert", "prand_generate_host_u32",
           "prand_generate_host_f32", "prand_generate_host_f64", "prand_device_state_bytes", "prand_export_states",
           "prand_import_states", "prand_init_streams_variant", "prand_skipahead_pow2", "prand_init_streams_spaced",
           "prand_test_cells", "prand_test_counts", "prand_test_evaluate", "prand_chi2_sf", "prand_host_generate",
           "prand_batch_set_params", "prand_mt_jump_polynomial"]


class PrandError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_status_text(status)})")


class ServerStats(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_uint64) for nm in ("completed", "samples", "hits", "misses", "spills", "restores",
                                                 "batches", "pending", "tiles")] + [("worker_busy_s", ctypes.c_double)] + \
        [(nm, ctypes.c_uint64) for nm in ("arena_used_bytes", "arena_free_blocks", "arena_top_bytes", "flights_busy")] + \
        [("gpu_busy_s", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("gen", ctypes.c_int32), ("dtype", ctypes.c_int32), ("stream", ctypes.c_uint64),
                ("length", ctypes.c_uint64), ("dev_out", ctypes.c_void_p)]


class Test(ctypes.Structure):
    """prand_test_t: kind (TEST_*), bits (frequency, serial), t, lo, hi (gap)."""
    _fields_ = [("kind", ctypes.c_int32), ("bits", ctypes.c_uint32), ("t", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]


TEST_FREQUENCY, TEST_SERIAL, TEST_GAP = 0, 1, 2

_lib = None


def load(build_if_missing: bool = False):
    """Load the shared library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"prand CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        from . import build as _b
        _b.build()
    L = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    u64 = ctypes.c_uint64
    L.prand_create.argtypes = [ctypes.POINTER(H), ctypes.c_int, u64]
    L.prand_init_streams.argtypes = [H, u64, u64]
    L.prand_init_streams_variant.argtypes = [H, ctypes.c_int32, u64, u64]
    L.prand_skipahead_pow2.argtypes = [H, u64, ctypes.c_uint32]
    L.prand_init_streams_spaced.argtypes = [H, ctypes.c_uint32, u64, u64]
    L.prand_test_cells.argtypes = [ctypes.POINTER(Test)]
    L.prand_test_cells.restype = ctypes.c_uint32
    L.prand_test_counts.argtypes = [ctypes.POINTER(Test), ctypes.c_void_p, u64, ctypes.c_void_p, ctypes.c_void_p]
    L.prand_test_evaluate.argtypes = [ctypes.POINTER(Test), u64, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.prand_chi2_sf.argtypes = [ctypes.c_double, ctypes.c_double]
    L.prand_chi2_sf.restype = ctypes.c_double
    for nm in ("prand_generate_u32", "prand_generate_f32", "prand_generate_f64", "prand_generate_host_u32",
               "prand_generate_host_f32", "prand_generate_host_f64"):
        getattr(L, nm).argtypes = [H, ctypes.c_void_p, u64, ctypes.c_void_p]
    L.prand_skipahead.argtypes = [H, ctypes.POINTER(u64)]
    L.prand_get_state.argtypes = [H, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    L.prand_set_state.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
    L.prand_query.argtypes = [H, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.prand_destroy.argtypes = [H]
    L.prand_status_string.argtypes = [ctypes.c_int]
    L.prand_status_string.restype = ctypes.c_char_p
    L.prand_kernel_launches.argtypes = []
    L.prand_kernel_launches.restype = u64
    L.prand_batch_run.argtypes = [ctypes.POINTER(Request), ctypes.c_size_t, u64, ctypes.c_void_p]
    L.prand_mrg32k3a_generate_u32_noalloc.argtypes = [ctypes.c_void_p, u64, ctypes.c_void_p, u64, ctypes.c_void_p]
    L.prand_batch_set_params.argtypes = [ctypes.c_uint32] * 4
    L.prand_host_generate.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_void_p, u64, ctypes.c_void_p, u64,
                                      ctypes.c_int32]
    L.prand_convert.argtypes = [ctypes.c_void_p, u64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    L.prand_mt_jump_polynomial.argtypes = [ctypes.c_uint32, ctypes.c_void_p]
    L.prand_device_state_bytes.argtypes = [ctypes.c_int]
    L.prand_device_state_bytes.restype = u64
    L.prand_export_states.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    L.prand_import_states.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    vp = ctypes.c_void_p
    L.prand_server_create.argtypes = [ctypes.POINTER(vp), u64, u64, ctypes.c_uint32]
    L.prand_server_submit.argtypes = [vp, ctypes.c_int32, u64, u64, ctypes.c_int32, ctypes.POINTER(u64)]
    L.prand_server_query.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(vp),
                                     ctypes.POINTER(ctypes.c_double)]
    L.prand_server_completed.argtypes = [vp, ctypes.POINTER(u64), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.prand_server_release.argtypes = [vp, u64]
    L.prand_server_read.argtypes = [vp, u64, vp, u64]
    L.prand_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.prand_server_destroy.argtypes = [vp]
    L.prand_server_replay.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.prand_batch_run_per_request.argtypes = [ctypes.POINTER(Request), ctypes.c_size_t, u64, ctypes.c_void_p]
    L.prand_batch_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Request), ctypes.c_size_t, u64]
    L.prand_batch_plan_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.prand_batch_plan_destroy.argtypes = [ctypes.c_void_p]
    L.prand_batch_autotune.argtypes = [ctypes.POINTER(Request), ctypes.c_size_t, u64, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_float)]
    for nm in EXPORTS:
        if nm not in ("prand_status_string", "prand_kernel_launches", "prand_device_state_bytes", "prand_test_cells",
                      "prand_chi2_sf"):
            getattr(L, nm).restype = ctypes.c_int
    _lib = L
    return L


def _status_text(s: int) -> str:
    try:
        return load().prand_status_string(s).decode()
    except Exception:  # pragma: no cover
        return "?"


def _check(status: int, where: str, allow_warn: bool = False) -> int:
    if status == PRAND_OK or (allow_warn and status == PRAND_WARN_STREAM_OVERLAP):
        return status
    raise PrandError(status, where)


def _gid(gen) -> int:
    return GEN_ID[gen] if isinstance(gen, str) else int(gen)


# ----------------------------------------------------------------- C names

def prand_create(gen, seed: int = SEED_DEFAULT) -> int:
    h = ctypes.c_void_p()
    _check(load().prand_create(ctypes.byref(h), _gid(gen), ctypes.c_uint64(seed)), "prand_create")
    return h.value


def prand_init_streams(h: int, first_stream: int, n_streams: int) -> int:
    return _check(load().prand_init_streams(h, first_stream, n_streams), "prand_init_streams", allow_warn=True)


def prand_generate_u32(h: int, dev_out: int, n_per_stream: int, stream: int = 0) -> None:
    _check(load().prand_generate_u32(h, dev_out, n_per_stream, stream), "prand_generate_u32")


def prand_generate_f32(h: int, dev_out: int, n_per_stream: int, stream: int = 0) -> None:
    _check(load().prand_generate_f32(h, dev_out, n_per_stream, stream), "prand_generate_f32")


def prand_generate_f64(h: int, dev_out: int, n_per_stream: int, stream: int = 0) -> None:
    _check(load().prand_generate_f64(h, dev_out, n_per_stream, stream), "prand_generate_f64")


def prand_generate_host_u32(h: int, host_out: int, n_per_stream: int, stream: int = 0) -> None:
    _check(load().prand_generate_host_u32(h, host_out, n_per_stream, stream), "prand_generate_host_u32")


def prand_generate_host_f32(h: int, host_out: int, n_per_stream: int, stream: int = 0) -> None:
    _check(load().prand_generate_host_f32(h, host_out, n_per_stream, stream), "prand_generate_host_f32")


def prand_generate_host_f64(h: int, host_out: int, n_per_stream: int, stream: int = 0) -> None:
    _check(load().prand_generate_host_f64(h, host_out, n_per_stream, stream), "prand_generate_host_f64")


def prand_mt_jump_polynomial(b: int) -> int:
    """x^(2^b) mod phi for MT19937 as a Python int (bit i = coefficient of x^i)."""
    buf = (ctypes.c_uint32 * 624)()
    _check(load().prand_mt_jump_polynomial(b, ctypes.cast(buf, ctypes.c_void_p)), "prand_mt_jump_polynomial")
    return sum(int(w) << (32 * i) for i, w in enumerate(buf))


def prand_device_state_bytes(gen) -> int:
    return int(load().prand_device_state_bytes(_gid(gen)))


def prand_export_states(h: int, dev_states: int, stream: int = 0) -> None:
    _check(load().prand_export_states(h, dev_states, stream), "prand_export_states")


def prand_import_states(h: int, dev_states: int, stream: int = 0) -> None:
    _check(load().prand_import_states(h, dev_states, stream), "prand_import_states")


VARIANT_DEFAULT, VARIANT_MEDIUM, VARIANT_LONG = 0, 1, 2


def prand_init_streams_variant(h: int, variant: int, first: int, n: int) -> int:
    """Streams first..first+n-1 of a Table 4 variant; returns the status (7 = overlap warning)."""
    return _check(load().prand_init_streams_variant(h, variant, first, n), "prand_init_streams_variant", allow_warn=True)


def prand_skipahead_pow2(h: int, a: int, b: int) -> None:
    _check(load().prand_skipahead_pow2(h, ctypes.c_uint64(a), b), "prand_skipahead_pow2")


def prand_skipahead(h: int, offset: int) -> None:
    if offset < 0 or offset >= 1 << 256:
        raise ValueError("offset must be in [0, 2^256)")
    arr = (ctypes.c_uint64 * 4)(*[(offset >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)])
    _check(load().prand_skipahead(h, arr), "prand_skipahead")


def prand_get_state(h: int) -> bytes:
    n = ctypes.c_size_t(0)
    _check(load().prand_get_state(h, None, ctypes.byref(n)), "prand_get_state")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().prand_get_state(h, buf, ctypes.byref(n)), "prand_get_state")
    return buf.raw[:n.value]


def prand_set_state(h: int, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().prand_set_state(h, buf, len(blob)), "prand_set_state")


def prand_query(h: int):
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().prand_query(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "prand_query")
    return a.value, b.value, c.value


def prand_destroy(h: int) -> None:
    if h:
        _check(load().prand_destroy(h), "prand_destroy")


def prand_status_string(status: int) -> str:
    return _status_text(status)


def prand_kernel_launches() -> int:
    return int(load().prand_kernel_launches())


def requests_array(requests):
    """(gen, dtype, stream_index, length, dev_ptr) tuples -> a prand_request_t array."""
    reqs = list(requests)
    arr = (Request * max(1, len(reqs)))()
    for i, (g, dt, s, n, p) in enumerate(reqs):
        arr[i] = Request(_gid(g), dt, s, n, p)
    return arr, len(reqs)


def prand_batch_run(requests, seed: int, stream: int = 0) -> None:
    """requests: iterable of (gen, dtype, stream_index, length, dev_ptr)."""
    arr, n = requests_array(requests)
    _check(load().prand_batch_run(arr, n, ctypes.c_uint64(seed), stream), "prand_batch_run")


def prand_batch_run_per_request(requests, seed: int, stream: int = 0) -> None:
    arr, n = requests_array(requests)
    _check(load().prand_batch_run_per_request(arr, n, ctypes.c_uint64(seed), stream), "prand_batch_run_per_request")


def prand_batch_plan_create(requests, seed: int) -> int:
    arr, n = requests_array(requests)
    p = ctypes.c_void_p()
    _check(load().prand_batch_plan_create(ctypes.byref(p), arr, n, ctypes.c_uint64(seed)), "prand_batch_plan_create")
    return p.value


def prand_batch_plan_launch(plan: int, stream: int = 0) -> None:
    _check(load().prand_batch_plan_launch(plan, stream), "prand_batch_plan_launch")


def prand_batch_plan_destroy(plan: int) -> None:
    if plan:
        _check(load().prand_batch_plan_destroy(plan), "prand_batch_plan_destroy")


def prand_batch_autotune(requests, seed: int, stream: int = 0):
    """Returns (seclen_mrg_lfsr, seclen_gm, block, row_bytes, best_ms) and keeps
    them for later batches."""
    arr, n = requests_array(requests)
    a, b, c, d, t = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_float()
    _check(load().prand_batch_autotune(arr, n, ctypes.c_uint64(seed), stream, ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c), ctypes.byref(d), ctypes.byref(t)), "prand_batch_autotune")
    return a.value, b.value, c.value, d.value, t.value


def prand_batch_set_params(seclen_mrg_lfsr: int, seclen_gm: int, block: int = 64, row_bytes: int = 128) -> None:
    _check(load().prand_batch_set_params(seclen_mrg_lfsr, seclen_gm, block, row_bytes), "prand_batch_set_params")


def prand_mrg32k3a_generate_u32_noalloc(dev_state: int, n_streams: int, dev_out: int, n_per_stream: int,
                                        stream: int = 0) -> None:
    """MRG32K3A u32 fill on caller-held states without any device allocation."""
    _check(load().prand_mrg32k3a_generate_u32_noalloc(dev_state, n_streams, dev_out, n_per_stream, stream),
           "prand_mrg32k3a_generate_u32_noalloc")


def prand_host_generate(gen, dtype: int, host_states: int, n_streams: int, host_out: int, n_per_stream: int,
                        n_threads: int = 0) -> None:
    """MT19937 / MRG32K3A / LFSR113 outputs computed on the host's vector units
    from states in the prand_device.h layouts (advanced in place)."""
    _check(load().prand_host_generate(_gid(gen), dtype, host_states, n_streams, host_out, n_per_stream, n_threads),
           "prand_host_generate")


MAP_MRG_F64 = 3


def prand_init_streams_spaced(h: int, log2_spacing: int, first: int, n: int) -> None:
    """Streams first..first+n-1 spaced 2^log2_spacing outputs apart (Table 3's layout)."""
    _check(load().prand_init_streams_spaced(h, log2_spacing, first, n), "prand_init_streams_spaced")


def make_test(kind: int, bits: int = 0, lo: int = 0, hi: int = 0, t: int = 0) -> Test:
    return Test(kind, bits, t, 0, lo, hi)


def prand_test_cells(test: Test) -> int:
    return int(load().prand_test_cells(ctypes.byref(test)))


def prand_test_counts(test: Test, dev_words: int, n: int, dev_counts: int, stream: int = 0) -> None:
    """Cell counts of `test` over n device words into dev_counts (uint64, prand_test_cells entries)."""
    _check(load().prand_test_counts(ctypes.byref(test), dev_words, n, dev_counts, stream), "prand_test_counts")


def prand_test_evaluate(test: Test, n: int, counts) -> tuple:
    """(chi2, degrees of freedom, p-value) of host counts (a sequence of ints) of `test` over n words."""
    cells = prand_test_cells(test)
    arr = (ctypes.c_uint64 * cells)(*[int(c) for c in counts])
    chi2, dof, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().prand_test_evaluate(ctypes.byref(test), n, arr, ctypes.byref(chi2), ctypes.byref(dof),
                                      ctypes.byref(p)), "prand_test_evaluate")
    return chi2.value, dof.value, p.value


def prand_chi2_sf(x: float, dof: float) -> float:
    return float(load().prand_chi2_sf(x, dof))


def prand_convert(dev_in: int, n: int, map_: int, dev_out: int, stream: int = 0) -> None:
    """Float map of n device u32 words: map_ = DTYPE_F32, DTYPE_F64 or MAP_MRG_F64."""
    _check(load().prand_convert(dev_in, n, map_, dev_out, stream), "prand_convert")


def prand_server_create(seed: int, output_bytes: int, slots_per_generator: int) -> int:
    h = ctypes.c_void_p()
    _check(load().prand_server_create(ctypes.byref(h), ctypes.c_uint64(seed), output_bytes, slots_per_generator),
           "prand_server_create")
    return h.value


def prand_server_submit(srv: int, gen, stream: int, length: int, dtype: int) -> int:
    i = ctypes.c_uint64()
    _check(load().prand_server_submit(srv, _gid(gen), stream, length, dtype, ctypes.byref(i)), "prand_server_submit")
    return i.value


def prand_server_query(srv: int, rid: int):
    """(done, device pointer or None, latency seconds)."""
    d, p, lat = ctypes.c_int32(), ctypes.c_void_p(), ctypes.c_double()
    _check(load().prand_server_query(srv, rid, ctypes.byref(d), ctypes.byref(p), ctypes.byref(lat)),
           "prand_server_query")
    return bool(d.value), p.value, lat.value


def prand_server_completed(srv: int, cap: int = 4096):
    arr = (ctypes.c_uint64 * cap)()
    n = ctypes.c_size_t()
    _check(load().prand_server_completed(srv, arr, cap, ctypes.byref(n)), "prand_server_completed")
    return [arr[i] for i in range(n.value)]


def prand_server_read(srv: int, rid: int, out) -> None:
    """Copy a completed request's output into the numpy array `out`."""
    _check(load().prand_server_read(srv, rid, out.ctypes.data, out.nbytes), "prand_server_read")


def prand_server_release(srv: int, rid: int) -> None:
    _check(load().prand_server_release(srv, rid), "prand_server_release")


def prand_server_stats(srv: int) -> dict:
    st = ServerStats()
    _check(load().prand_server_stats(srv, ctypes.byref(st)), "prand_server_stats")
    return {nm: getattr(st, nm) for nm, _ in ServerStats._fields_}


def prand_server_destroy(srv: int) -> None:
    if srv:
        _check(load().prand_server_destroy(srv), "prand_server_destroy")


def prand_server_replay(srv: int, requests, arrivals):
    """requests: (gen, dtype, stream, length) tuples; arrivals: seconds.  Returns (latencies, wall_s)."""
    reqs = list(requests)
    n = len(reqs)
    arr = (Request * max(1, n))()
    for i, (g, dt, k, L) in enumerate(reqs):
        arr[i] = Request(_gid(g), dt, k, L, None)
    at = (ctypes.c_double * max(1, n))(*arrivals)
    lat = (ctypes.c_double * max(1, n))()
    wall = ctypes.c_double()
    _check(load().prand_server_replay(srv, arr, at, n, lat, ctypes.byref(wall)), "prand_server_replay")
    return [lat[i] for i in range(n)], wall.value


# ----------------------------------------------------------------- wrapper

class Generator:
    """One handle: ``n_streams`` block-split streams of one generator."""

    def __init__(self, gen, seed: int = SEED_DEFAULT, first_stream: int = 0, n_streams: int = 1):
        self.gen = gen
        self.h = prand_create(gen, seed)
        self.status = prand_init_streams(self.h, first_stream, n_streams)
        self.n_streams = n_streams

    def close(self):
        if self.h:
            prand_destroy(self.h)
            self.h = 0

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def generate(self, n_per_stream: int, dtype: str = "u32", out=None, stream=None):
        import torch
        tdt = {"u32": torch.int32, "f32": torch.float32, "f64": torch.float64}[dtype]
        if out is None:
            out = torch.empty((self.n_streams, n_per_stream), dtype=tdt, device="cuda")
        st = torch.cuda.current_stream().cuda_stream if stream is None else stream
        fn = {"u32": prand_generate_u32, "f32": prand_generate_f32, "f64": prand_generate_f64}[dtype]
        fn(self.h, out.data_ptr(), n_per_stream, st)
        return out

    def skipahead(self, offset: int):
        prand_skipahead(self.h, offset)

    def get_state(self) -> bytes:
        return prand_get_state(self.h)

    def set_state(self, blob: bytes):
        prand_set_state(self.h, blob)
        self.n_streams = prand_query(self.h)[1]
