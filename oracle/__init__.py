"""CPU oracle for the PRAND generators (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The library under
``paper_1307_5869_gb300`` never imports it, and the two share no code.

The arithmetic lives in ``prand_oracle.c`` (plain C, one recurrence step at a
time); this module only compiles it with gcc and marshals arguments through
ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prand_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

GENS = ["MT19937", "MRG32K3A", "LFSR113", "GM19", "GM29", "GM31", "GM55",
        "GM61", "GQ58_1", "GQ58_3", "GQ58_4"]
GEN_ID = {name: i for i, name in enumerate(GENS)}
SEED_DEFAULT = 2**64 - 1
NBIG = 8  # 512-bit jump offsets

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            vp = ctypes.c_void_p
            L.orc_state_bytes.argtypes = [ctypes.c_int]
            L.orc_seed.argtypes = [ctypes.c_int, ctypes.c_uint64, vp]
            L.orc_next_u32.argtypes = [ctypes.c_int, vp]
            L.orc_next_u32.restype = ctypes.c_uint32
            L.orc_jump.argtypes = [ctypes.c_int, vp, u64p]
            L.orc_block_length.argtypes = [ctypes.c_int, u64p]
            L.orc_stream.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, vp]
            L.orc_stream_range.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, vp]
            L.orc_stream_v.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, vp]
            L.orc_stream_range_v.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_uint64, vp]
            L.orc_variant.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), u64p]
            L.orc_stream_spaced.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, vp]
            L.orc_freq_counts.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, vp]
            L.orc_serial_counts.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, vp]
            L.orc_gap_counts.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, vp]
            for nm in ("orc_freq_counts", "orc_serial_counts", "orc_gap_counts"):
                getattr(L, nm).restype = None
            for nm in ("orc_gen_u32", "orc_gen_f32", "orc_gen_f64"):
                getattr(L, nm).argtypes = [ctypes.c_int, vp, vp, ctypes.c_uint64]
            for nm in ("orc_gen_many_u32", "orc_gen_many_f32", "orc_gen_many_f64"):
                getattr(L, nm).argtypes = [ctypes.c_int, vp, ctypes.c_uint64, vp, ctypes.c_uint64]
            L.orc_u32_to_f32.argtypes = [ctypes.c_uint32]
            L.orc_u32_to_f32.restype = ctypes.c_float
            L.orc_u32_to_f64.argtypes = [ctypes.c_uint32]
            L.orc_u32_to_f64.restype = ctypes.c_double
            L.orc_mrg_to_f64.argtypes = [ctypes.c_uint32]
            L.orc_mrg_to_f64.restype = ctypes.c_double
            L.orc_convert.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, vp]
            L.orc_mt_charpoly.argtypes = [u64p]
            L.orc_mt_jump_poly.argtypes = [u64p, u64p]
            L.orc_mt_x_pow2k.argtypes = [ctypes.c_int, u64p]
            L.orc_mt_apply_poly.argtypes = [vp, u64p]
            L.orc_lfsr_bits.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int]
            L.orc_lfsr_comp_step.argtypes = [ctypes.c_uint32, ctypes.c_int]
            L.orc_lfsr_comp_step.restype = ctypes.c_uint32
            L.orc_lfsr_comp_jump.argtypes = [ctypes.c_uint32, ctypes.c_int, u64p]
            L.orc_lfsr_comp_jump.restype = ctypes.c_uint32
            L.orc_lfsr_param.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_gm_param.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
            L.orc_gm_matpow.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p, u64p]
            L.orc_gm_point_step.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p, u64p]
            L.orc_splitmix64.argtypes = [u64p]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_gm_point_jump.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p, u64p, u64p]
            _lib = L
    return _lib


def convert(u: np.ndarray, kind: str) -> np.ndarray:
    """The float maps applied to an array of u32 words: kind "f32", "f64" or
    "mrg_f64" (the MRG32K3A double map)."""
    u = np.ascontiguousarray(u, dtype=np.uint32)
    k = {"f32": 0, "f64": 1, "mrg_f64": 2}[kind]
    out = np.empty(u.size, dtype=np.float32 if k == 0 else np.float64)
    lib().orc_convert(u.ctypes.data, u.size, k, out.ctypes.data)
    return out


def big(n: int, words: int = NBIG):
    """A non-negative Python int as a little-endian uint64 ctypes array."""
    if n < 0 or n >= 1 << (64 * words):
        raise ValueError("offset out of range")
    arr = (ctypes.c_uint64 * words)()
    for i in range(words):
        arr[i] = (n >> (64 * i)) & 0xFFFFFFFFFFFFFFFF
    return arr


def gid(gen) -> int:
    return GEN_ID[gen] if isinstance(gen, str) else int(gen)


class State:
    """An oracle generator state (opaque bytes, layout fixed by the C file)."""

    def __init__(self, gen, seed: int = SEED_DEFAULT, raw: bytes | None = None):
        self.gen = gid(gen)
        self.nbytes = lib().orc_state_bytes(self.gen)
        self.buf = ctypes.create_string_buffer(self.nbytes)
        if raw is not None:
            ctypes.memmove(self.buf, raw, self.nbytes)
        else:
            lib().orc_seed(self.gen, ctypes.c_uint64(seed), self.buf)

    @classmethod
    def stream(cls, gen, seed: int, k: int, variant: int = 0) -> "State":
        st = cls(gen, seed)
        if lib().orc_stream_v(st.gen, ctypes.c_uint64(seed), variant, ctypes.c_uint64(k), st.buf):
            raise ValueError("no such stream variant")
        return st

    @classmethod
    def spaced(cls, gen, seed: int, spacing_log2: int, k: int) -> "State":
        """Stream k of the spaced layout: the base advanced by k * 2^spacing_log2."""
        st = cls(gen, seed)
        if lib().orc_stream_spaced(st.gen, ctypes.c_uint64(seed), spacing_log2, ctypes.c_uint64(k), st.buf):
            raise ValueError("spacing out of range")
        return st

    def copy(self) -> "State":
        return State(self.gen, raw=self.buf.raw)

    def raw(self) -> bytes:
        return self.buf.raw

    def jump(self, n: int) -> "State":
        lib().orc_jump(self.gen, self.buf, big(n))
        return self

    def next(self) -> int:
        return lib().orc_next_u32(self.gen, self.buf)

    def u32(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint32)
        lib().orc_gen_u32(self.gen, self.buf, out.ctypes.data, n)
        return out

    def f32(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.float32)
        lib().orc_gen_f32(self.gen, self.buf, out.ctypes.data, n)
        return out

    def f64(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.float64)
        lib().orc_gen_f64(self.gen, self.buf, out.ctypes.data, n)
        return out


def block_length(gen, variant: int = 0) -> int:
    return variant_info(gen, variant)[1]


def variant_info(gen, variant: int):
    """(number of sequences, block length) of a Table 4 variant, or None."""
    arr = (ctypes.c_uint64 * NBIG)()
    nmax = ctypes.c_uint64()
    if lib().orc_variant(gid(gen), variant, ctypes.byref(nmax), arr):
        return None
    return nmax.value, sum(int(arr[i]) << (64 * i) for i in range(NBIG))


def splitmix64(seed: int, n: int) -> list:
    """The first n outputs of SplitMix64 from the 64-bit state `seed` (the
    generator that expands seeds into MRG32K3A, LFSR113 and GM/GQ states)."""
    st = ctypes.c_uint64(seed)
    return [int(lib().orc_splitmix64(ctypes.byref(st))) for _ in range(n)]


def gm_state_raw(gen, x_prev, x) -> "State":
    """An oracle GM/GQ state from explicit (x^(n-1), x^(n)) of each point (the
    first s entries; the remaining slots are zero)."""
    s = gm_param(gen, "s")
    if len(x_prev) != s or len(x) != s:
        raise ValueError("need one (x_prev, x) pair per point")
    words = np.zeros(64, dtype=np.uint64)
    words[:s] = np.array(x_prev, dtype=np.uint64)
    words[32:32 + s] = np.array(x, dtype=np.uint64)
    st = State(gen)
    raw = words.tobytes()
    assert len(raw) == st.nbytes
    return State(gen, raw=raw)


def gm_state_points(st: "State"):
    """(x_prev, x) of each point of an oracle GM/GQ state."""
    s = gm_param(st.gen, "s")
    words = np.frombuffer(st.raw(), dtype=np.uint64)
    return [int(v) for v in words[:s]], [int(v) for v in words[32:32 + s]]


def gm_param(gen, name: str) -> int:
    which = ["k", "q", "g", "v", "s", "t", "p", "L", "nmax"].index(name)
    out = ctypes.c_uint64()
    if lib().orc_gm_param(gid(gen), which, ctypes.byref(out)):
        raise ValueError(gen)
    return out.value


class Streams:
    """States of streams first..first+n-1 (back to back) for bulk generation."""

    def __init__(self, gen, seed: int, first: int, n: int, variant: int = 0):
        self.gen = gid(gen)
        self.n = n
        self.sb = lib().orc_state_bytes(self.gen)
        self.buf = ctypes.create_string_buffer(self.sb * n)
        rc = lib().orc_stream_range_v(self.gen, ctypes.c_uint64(seed), variant, ctypes.c_uint64(first),
                                      ctypes.c_uint64(n), self.buf)
        if rc:
            raise RuntimeError("oracle stream range failed")

    def state(self, j: int) -> State:
        return State(self.gen, raw=self.buf.raw[j * self.sb:(j + 1) * self.sb])

    def generate(self, dtype: str, n_per: int) -> np.ndarray:
        npdt = {"u32": np.uint32, "f32": np.float32, "f64": np.float64}[dtype]
        out = np.empty(self.n * n_per, dtype=npdt)
        fn = {"u32": lib().orc_gen_many_u32, "f32": lib().orc_gen_many_f32,
              "f64": lib().orc_gen_many_f64}[dtype]
        fn(self.gen, self.buf, ctypes.c_uint64(self.n), out.ctypes.data, ctypes.c_uint64(n_per))
        return out.reshape(self.n, n_per)


def stream_digest(gen, seed: int, first: int, count: int, n_per: int, dtypes=("u32", "f32")) -> str:
    """BLAKE2b digest of streams first..first+count-1, each dtype's block of
    count x n_per outputs in turn (the later dtypes continue the streams), as
    raw little-endian bytes.  A caller holding the same outputs from elsewhere
    hashes them the same way to compare whole blocks at once."""
    import hashlib
    st = Streams(gen, seed, first, count)
    h = hashlib.blake2b(digest_size=32)
    for dt in dtypes:
        h.update(np.ascontiguousarray(st.generate(dt, n_per)).tobytes())
    return h.hexdigest()


def _digest_job(args):
    return stream_digest(*args)


def stream_digests(gen, seed: int, n_streams: int, n_per: int, chunk: int, dtypes=("u32", "f32"), procs=None):
    """stream_digest of every chunk of `chunk` streams, computed by a pool of
    processes started with spawn (safe after the parent has used a GPU)."""
    import multiprocessing as mp
    jobs = [(gen, seed, a, min(chunk, n_streams - a), n_per, tuple(dtypes)) for a in range(0, n_streams, chunk)]
    with mp.get_context("spawn").Pool(procs or os.cpu_count() or 1) as pool:
        return pool.map(_digest_job, jobs, chunksize=1)


def mt_charpoly() -> int:
    """The MT19937 characteristic polynomial as a Python int (bit i = x^i)."""
    arr = (ctypes.c_uint64 * 313)()
    deg = lib().orc_mt_charpoly(arr)
    if deg != 19937:
        raise RuntimeError(f"Berlekamp-Massey gave degree {deg}")
    return sum(int(arr[i]) << (64 * i) for i in range(313))


def mt_poly_words_to_int(arr) -> int:
    return sum(int(arr[i]) << (64 * i) for i in range(313))


def mt_x_pow2k(k: int) -> int:
    arr = (ctypes.c_uint64 * 313)()
    lib().orc_mt_x_pow2k(k, arr)
    return mt_poly_words_to_int(arr)


def mt_jump_poly(e: int) -> int:
    arr = (ctypes.c_uint64 * 313)()
    lib().orc_mt_jump_poly(big(e), arr)
    return mt_poly_words_to_int(arr)


def mt_apply_poly(st: State, poly: int) -> State:
    arr = (ctypes.c_uint64 * 313)()
    for i in range(313):
        arr[i] = (poly >> (64 * i)) & 0xFFFFFFFFFFFFFFFF
    lib().orc_mt_apply_poly(st.buf, arr)
    return st


# ---------------------------------------------------------------- tests
# Spaced streams and the classical tests of the skip-ahead study (Table 3):
# the oracle computes cell counts plainly; the chi-square tail comes from
# scipy (a library routine).

def spaced_outputs(gen, seed: int, spacing_log2: int, first: int, n: int, n_per: int = 1) -> np.ndarray:
    """Outputs 0..n_per-1 of streams first..first+n-1 of the spaced layout
    (stream k = base advanced by k * 2^spacing_log2), stream-major; with
    n_per = 1 this is the subsequence u[(first + j) * 2^spacing_log2]."""
    base = State.spaced(gen, seed, spacing_log2, first)
    out = np.empty((n, n_per), dtype=np.uint32)
    for j in range(n):
        if j:
            base.jump(1 << spacing_log2)  # stream first + j
        out[j] = base.copy().u32(n_per)
    return out


def freq_counts(u: np.ndarray, bits: int) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    c = np.zeros(1 << bits, dtype=np.uint64)
    lib().orc_freq_counts(u.ctypes.data, ctypes.c_uint64(u.size), bits, c.ctypes.data)
    return c


def serial_counts(u: np.ndarray, bits: int) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    c = np.zeros(1 << (2 * bits), dtype=np.uint64)
    lib().orc_serial_counts(u.ctypes.data, ctypes.c_uint64(u.size), bits, c.ctypes.data)
    return c


def gap_counts(u: np.ndarray, lo: int, hi: int, t: int) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.uint32)
    c = np.zeros(t + 1, dtype=np.uint64)
    lib().orc_gap_counts(u.ctypes.data, ctypes.c_uint64(u.size), ctypes.c_uint64(lo), ctypes.c_uint64(hi), t,
                         c.ctypes.data)
    return c


def expected_counts(kind: str, n: int, counts: np.ndarray, bits: int = 0, lo: int = 0, hi: int = 0,
                    t: int = 0) -> np.ndarray:
    """Cell expectations under the uniform hypothesis (Knuth, Sec. 3.3.2):
    frequency n / 2^b; serial floor(n / 2) / 4^b; gap G p (1-p)^r for r < t
    and G (1-p)^t for the last cell, G = the number of gaps, p = (hi-lo)/2^32."""
    if kind == "frequency":
        return np.full(1 << bits, n / (1 << bits))
    if kind == "serial":
        return np.full(1 << (2 * bits), (n // 2) / (1 << (2 * bits)))
    p = (hi - lo) / 2.0**32
    G = float(counts.sum())
    e = np.array([G * p * (1 - p) ** r for r in range(t)] + [G * (1 - p) ** t])
    return e


def chi2_test(kind: str, n: int, counts: np.ndarray, **kw):
    """Pearson's statistic sum (O - E)^2 / E over the cells and its upper tail
    probability with (cells - 1) degrees of freedom."""
    from scipy.stats import chi2 as _chi2
    e = expected_counts(kind, n, counts, **kw)
    o = counts.astype(np.float64)
    stat = float(((o - e) ** 2 / e).sum())
    return stat, float(_chi2.sf(stat, len(e) - 1))
