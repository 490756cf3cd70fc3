"""GPU parity of the batched forms (one persistent launch, CUDA-graph plans,
per-request launches) against the oracle: every request's output must equal
the oracle's stream k from its start, bit for bit, alone and in the mix."""
import numpy as np
import pytest

import oracle as O
import paper_1307_5869_gb300 as P
from paper_1307_5869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TDT = {"u32": "int32", "f32": "float32", "f64": "float64"}
DTI = {"u32": 0, "f32": 1, "f64": 2}
BITS = {"u32": np.uint32, "f32": np.uint32, "f64": np.uint64}


def _mk(reqspec, offset_elems=0):
    import torch
    bufs, reqs = [], []
    for gen, dt, k, n in reqspec:
        t = torch.empty(n + offset_elems, dtype=getattr(torch, TDT[dt]), device="cuda")
        v = t[offset_elems:]
        bufs.append(v)
        reqs.append((gen, DTI[dt], k, n, v.data_ptr()))
    return bufs, reqs


def _check(bufs, reqspec, seed, what):
    for v, (gen, dt, k, n) in zip(bufs, reqspec):
        got = v.cpu().numpy().view(BITS[dt])
        want = getattr(O.State.stream(gen, seed, k), dt)(n).view(BITS[dt])
        if not np.array_equal(got, want):
            bad = np.flatnonzero(got != want)
            raise AssertionError(f"{what}: {gen} {dt} stream {k} n={n}: {len(bad)} mismatches from {bad[0]}")


def _spec(seed, count, maxlen, dts=("u32", "f32", "f64")):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        gen = P.GENERATORS[i % len(P.GENERATORS)]
        dt = dts[i % len(dts)]
        k = int(rng.integers(0, 10**19, dtype=np.uint64))
        n = int(np.floor(2 ** (np.log2(maxlen) * rng.random()))) + 1
        out.append((gen, dt, k, n))
    return out


def test_batch_long_requests_all_gens_dtypes():
    # lengths up to ~2^17: requests span many tiles, sections and store paths
    spec = _spec(3, 66, 1 << 17) + [("GM61", "u32", 5, 300000), ("MRG32K3A", "f64", 7, 250001),
                                    ("LFSR113", "f32", 9, 1 << 18), ("GQ58_3", "u32", 11, 100003)]
    bufs, reqs = _mk(spec)
    P.prand_batch_run(reqs, 12345)
    import torch
    torch.cuda.synchronize()
    _check(bufs, spec, 12345, "batch")


def test_batch_misaligned_outputs_scalar_paths():
    spec = _spec(4, 22, 5000, dts=("u32", "f32"))
    bufs, reqs = _mk(spec, offset_elems=1)
    P.prand_batch_run(reqs, 99)
    import torch
    torch.cuda.synchronize()
    _check(bufs, spec, 99, "batch misaligned")


def test_batch_alone_equals_in_the_mix():
    import torch
    spec = _spec(5, 33, 20000)
    bufs, reqs = _mk(spec)
    P.prand_batch_run(reqs, 7)
    torch.cuda.synchronize()
    for i in (0, 7, 19):
        b1, r1 = _mk([spec[i]])
        P.prand_batch_run(r1, 7)
        torch.cuda.synchronize()
        assert torch.equal(b1[0], bufs[i])


def test_plan_graph_replay_and_per_request_form():
    import torch
    spec = _spec(6, 44, 30000)
    bufs, reqs = _mk(spec)
    plan = P.prand_batch_plan_create(reqs, 2024)
    for _ in range(2):
        for b in bufs:
            b.zero_()
        P.prand_batch_plan_launch(plan, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        _check(bufs, spec, 2024, "plan replay")
    P.prand_batch_plan_destroy(plan)
    for b in bufs:
        b.zero_()
    P.prand_batch_run_per_request(reqs, 2024)
    torch.cuda.synchronize()
    _check(bufs, spec, 2024, "per request")


def test_autotune_keeps_outputs_exact():
    import torch
    spec = _spec(8, 22, 1 << 16, dts=("u32",))
    bufs, reqs = _mk(spec)
    a, b, bs, rb, ms = P.prand_batch_autotune(reqs, 31)
    assert a in (2048, 8192, 32768) and b in (2048, 8192, 32768) and bs in (64, 128) and rb in (128, 256) and ms > 0
    for x in bufs:
        x.zero_()
    P.prand_batch_run(reqs, 31)
    torch.cuda.synchronize()
    _check(bufs, spec, 31, "after autotune")


@pytest.mark.parametrize("block,row_bytes", [(64, 128), (64, 256), (128, 128), (128, 256)])
def test_every_rest_build_exact(block, row_bytes):
    # each build of the rest-of-generators kernel the tuner can pick (threads
    # per block, staged row size), with short sections so requests span many
    # tiles, on mixed generators and dtypes
    import torch
    spec = _spec(11, 23, 40_000)
    bufs, reqs = _mk(spec)
    P.prand_batch_set_params(2048, 2048, block, row_bytes)
    try:
        P.prand_batch_run(reqs, 77)
        torch.cuda.synchronize()
        _check(bufs, spec, 77, f"block {block}, rows {row_bytes}")
    finally:
        P.prand_batch_set_params(8192, 8192, 64, 128)
    with pytest.raises(P.PrandError):
        P.prand_batch_set_params(2048, 2048, 96, 128)


def test_batched_workload_sampled():
    # the 10^4-request batched workload (generator uniform over 11, stream uniform in
    # [0, 1e19), length floor(2^(20 U))), checked on a sample of requests
    import torch
    spec = [(g, "u32", k, n) for g, k, n, _ in W.batched_requests(10_000, seed=7)]
    total = sum(n for _, _, _, n in spec)
    buf = torch.empty(total, dtype=torch.int32, device="cuda")
    reqs, offs, o = [], [], 0
    for gen, dt, k, n in spec:
        reqs.append((gen, 0, k, n, buf.data_ptr() + 4 * o))
        offs.append(o)
        o += n
    P.prand_batch_run(reqs, 7)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    pick = set(int(i) for i in rng.integers(0, len(spec), 40))
    pick |= {i for i, s in enumerate(spec) if s[0] == "MT19937"}.intersection(range(0, 400))
    for i in sorted(pick):
        gen, dt, k, n = spec[i]
        n_chk = min(n, 20000)
        got = buf[offs[i]:offs[i] + n_chk].cpu().numpy().view(np.uint32)
        st = O.State.stream(gen, 7, k)
        assert np.array_equal(got, st.u32(n_chk)), (i, gen, k, n)
