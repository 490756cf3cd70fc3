#!/usr/bin/env python3
"""Benchmark of the multi-stream generation hot path on GB300.

Workload (bulk fill): MT19937, LFSR113 and GM61, 2^20 block-split streams each,
2^10 u32 outputs per stream followed by 2^10 f32 outputs per stream (2^30 + 2^30
outputs per generator), seed from a 64-bit counter.  One step = both fills for
all three generators (6 kernel launches, 6 * 2^30 outputs).  Stream states are
initialised (jump-ahead) once before timing and stay resident; their init time
is reported separately.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead
(on the host cores, a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving leg keeps up to 32 batches in flight, each on its own stream; with
# the default 8 hardware queues, streams would share queues and a long batch
# would hold up unrelated ones.  Takes effect only before CUDA starts.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_1307_5869_gb300 import workloads as W  # noqa: E402

METRIC = "GSamples/s (uint32) per generator, 2^30 outputs; % of HBM-write/int-pipe roofline"
UNIT = "GSamples/s"
WORKLOAD = ("bulk fill: MT19937, LFSR113, GM61; 2^20 block-split streams x (2^10 u32 + 2^10 f32) "
            "outputs per generator per GPU per step; seed 0x9E3779B97F4A7C15; rank r takes streams "
            "[r 2^20, (r+1) 2^20)")

# Algorithmic work per output: bytes of generator state per stream (loaded and stored once per fill).
STATE_BYTES = {"MT19937": 624 * 4, "MRG32K3A": 24, "LFSR113": 16, "GM19": 32 * 16, "GM29": 32 * 16,
               "GM31": 32 * 16, "GM55": 8 * 16, "GM61": 32 * 16, "GQ58_1": 32 * 16, "GQ58_3": 12 * 16,
               "GQ58_4": 8 * 16}
# Algorithmic int32 operations per output word of the integer-bound generators,
# counted from each kernel's arithmetic on 32-bit lanes (a 32x32->64 product or
# multiply-add counts as two operations): GM/GQ = the points' steps (the
# recurrence and its fold), strips and word assembly; MRG32K3A = its two
# component steps and the combination.  Per point step: GM19, GM29 7; GM31,
# GQ58.1 10; GM61 16; GM55 20; GQ58.3 12, GQ58.4 13 (a 7-operation step and a
# 32-bit strip of 5 or 6; GQ58.3's point 11 steps without a strip: 7).
OPS_PER_WORD = {"GM19": 32 * 7, "GM29": 32 * 7, "GM31": 32 * 10, "GM55": 8 * 20, "GM61": 32 * 16,
                "GQ58_1": 32 * 10, "GQ58_3": 11 * 12 + 7, "GQ58_4": 8 * 13, "MRG32K3A": 28}
# int32 lanes per SM: four schedulers, each issuing one 32-lane warp instruction per
# cycle (the issue-slot bound of an integer kernel; the SM count and clock are
# queried at run time)
LANES_PER_SM = 128
# DRAM bytes (read + write) per stream of one fill of 1024 outputs, from ncu
# captures (dram__bytes_read.sum + dram__bytes_write.sum) of the current kernels
# at 2^18 streams x 2^10 outputs, scaled per stream; None for other shapes.
TRAFFIC_PER_STREAM_1024 = {"MT19937.u32": 2.322e9 / 2**18, "MT19937.f32": 2.319e9 / 2**18,
                           "LFSR113.u32": 1.025e9 / 2**18, "LFSR113.f32": 1.022e9 / 2**18,
                           "GM61.u32": 1.396e9 / 2**18, "GM61.f32": 1.395e9 / 2**18}
# Output arena of the serving leg: 32 GiB of the GPU's HBM holds every request's
# output until it is read (at 1.9e10 samples/s of 4-8 byte samples, about a
# third of a second of demand).
SERVE_OUTPUT_BYTES = 32 << 30


def int_issue_peak(torch, device: int, sm_max_mhz):
    """Integer issue-slot bound (T int32 ops/s): SMs of the device (queried) x
    128 lanes x the maximum SM clock (from nvidia-smi during the run, else the
    measured figure, else the nominal 2070 MHz)."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    src = "nvidia-smi clocks.max.sm"
    if not sm_max_mhz:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                sm_max_mhz, src = float(json.load(f)["sm_max_mhz"]), "measured sm_max_mhz"
        except Exception:
            sm_max_mhz, src = 2070.0, "nominal 2070 MHz"
    peak = sms * LANES_PER_SM * sm_max_mhz * 1e6 / 1e12
    return peak, f"unit counts: {sms} SMs (queried) x {LANES_PER_SM} int32 lanes x {sm_max_mhz:g} MHz ({src})"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- oracle (CPU) legs

def oracle_rates(budget_s: float = 6.0, streams: int = 4):
    """Time the oracle (single thread, as it stands) generating u32 then f32
    rounds of 2^10 outputs per stream on the first streams of the bulk fill.
    Stream initialisation is not timed (as on the GPU)."""
    import oracle as O
    rates, detail = {}, {}
    share = {"MT19937": 0.2, "LFSR113": 0.2, "GM61": 0.6}
    for gen in W.BULK_GENERATORS:
        st = O.Streams(gen, W.bulk_seed(0), 0, streams)
        t0 = time.perf_counter()
        n = 0
        while True:
            st.generate("u32", W.BULK_PER_STREAM)
            st.generate("f32", W.BULK_PER_STREAM)
            n += 2 * streams * W.BULK_PER_STREAM
            if time.perf_counter() - t0 >= budget_s * share[gen]:
                break
        dt = time.perf_counter() - t0
        rates[gen] = n / dt
        detail[gen] = {"samples": n, "seconds": round(dt, 3)}
    return rates, detail


def _oracle_worker(job):
    """One process of the all-cores timing: the oracle on its own streams."""
    gen, first, streams, budget_s = job
    import oracle as O
    st = O.Streams(gen, W.bulk_seed(0), first, streams)
    t0 = time.perf_counter()
    n = 0
    while True:
        st.generate("u32", W.BULK_PER_STREAM)
        st.generate("f32", W.BULK_PER_STREAM)
        n += 2 * streams * W.BULK_PER_STREAM
        if time.perf_counter() - t0 >= budget_s:
            break
    return n, time.perf_counter() - t0


def oracle_rates_all_cores(budget_s: float = 6.0, streams: int = 4):
    """The same timing with one oracle process per host core (a spawn pool,
    as the process already uses CUDA), each on its own streams; the rate is
    the sum over the processes."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    share = {"MT19937": 0.2, "LFSR113": 0.2, "GM61": 0.6}
    rates = {}
    with mp.get_context("spawn").Pool(cores) as pool:
        for gen in W.BULK_GENERATORS:
            jobs = [(gen, k * streams, streams, budget_s * share[gen]) for k in range(cores)]
            rates[gen] = sum(n / dt for n, dt in pool.map(_oracle_worker, jobs))
    return rates, cores


def mix_throughput(rates: dict) -> float:
    """Whole-workload samples/s for equal sample counts per generator."""
    per = 2 * W.BULK_STREAMS * W.BULK_PER_STREAM
    total_t = sum(per / rates[g] for g in W.BULK_GENERATORS)
    return len(W.BULK_GENERATORS) * per / total_t


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, step_s = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rates, detail = oracle_rates(budget_s=args.ref_budget)
        if i >= args.warmup:
            steps.append((rates, detail))
            step_s.append(time.perf_counter() - t0)
    rates = {g: statistics.median(s[0][g] for s in steps) for g in W.BULK_GENERATORS}
    value = mix_throughput(rates) / 1e9
    # ms_per_step is the wall time of one measured reference step (the bounded
    # sample); the time the oracle would need for the whole workload step is
    # reported apart, as an extrapolation from the measured rates
    full_step_ms = 1e3 * 3 * 2 * W.BULK_STREAMS * W.BULK_PER_STREAM / (value * 1e9)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(step_s),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: first 4 streams of each generator, u32+f32 rounds of 2^10, "
                                   f"~{args.ref_budget:.0f} s of oracle time; the rate is the sample's",
                         "per_generator_samples_per_s": {g: rates[g] for g in rates}},
        "sample_step_ms": [round(1e3 * x, 1) for x in step_s],
        "full_step_ms_extrapolated": full_step_ms,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- GPU leg

def run_gpu(args):
    import torch
    import paper_1307_5869_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.load(build_if_missing=True)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    nS = args.streams or W.BULK_STREAMS
    nP = args.per_stream or W.BULK_PER_STREAM
    gens = args.gens.split(",") if args.gens else W.BULK_GENERATORS
    handles, init_ms = {}, {}
    for g in gens:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = P.prand_create(g, W.bulk_seed(0))
        P.prand_init_streams(h, *W.shard_range(rank, world, nS))
        init_ms[g] = 1e3 * (time.perf_counter() - t0)
        handles[g] = h
    U = torch.empty(nS * nP, dtype=torch.int32, device="cuda")
    F = torch.empty(nS * nP, dtype=torch.float32, device="cuda")

    def step(ev=None):
        for g in gens:
            if ev is not None:
                ev[g][0].record(stream)
            P.prand_generate_u32(handles[g], U.data_ptr(), nP, sp)
            if ev is not None:
                ev[g][1].record(stream)
            P.prand_generate_f32(handles[g], F.data_ptr(), nP, sp)
            if ev is not None:
                ev[g][2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [{g: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for g in gens} for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = P.prand_kernel_launches()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for k in range(args.steps):
            step(evs[k])
        e1.record(stream)
        torch.cuda.synchronize()
    launches = P.prand_kernel_launches() - l0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_u = {g: statistics.mean(e[g][0].elapsed_time(e[g][1]) for e in evs) for g in gens}
    ms_f = {g: statistics.mean(e[g][1].elapsed_time(e[g][2]) for e in evs) for g in gens}
    samples_step = len(gens) * 2 * nS * nP
    value = world * samples_step * args.steps / (total_ms * 1e-3) / 1e9

    # ----- context: a plain write-only fill of the same u32 buffer (torch's fill_),
    # the rate a kernel that only writes can reach on this GPU; reported beside
    # the rooflines, whose peak stays the measured copy bandwidth
    for _ in range(3):
        U.fill_(0)
    fill_ms = []
    for _ in range(10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        U.fill_(0)
        b.record(stream)
        b.synchronize()
        fill_ms.append(a.elapsed_time(b))
    write_fill_bytes = U.numel() * 4
    write_fill_gbs = write_fill_bytes / (statistics.median(fill_ms) * 1e-3) / 1e9

    # ----- rooflines (per launch, live CUDA-event durations)
    hbm_peak, peak_src = _peaks()
    clocks = clk.summary()
    int_peak, int_src = int_issue_peak(torch, local, clocks.get("sm_max_mhz"))
    args.int_peak = (int_peak, int_src)
    rooflines = {}
    for g in gens:
        for dt, ms in (("u32", ms_u[g]), ("f32", ms_f[g])):
            key = f"{g}.{dt}"
            if g.startswith("GM") or g.startswith("GQ"):
                ops = nS * nP * OPS_PER_WORD[g]
                rooflines[key] = {"bound": "alu", "achieved": ops / (ms * 1e-3) / 1e12,
                                  "peak": int_peak, "unit": "Tops/s",
                                  "ms": ms, "gsamples_per_s": nS * nP / (ms * 1e-3) / 1e9}
            else:
                byts = nS * nP * 4 + 2 * nS * STATE_BYTES[g]
                rooflines[key] = {"bound": "hbm", "achieved": byts / (ms * 1e-3) / 1e9, "peak": hbm_peak,
                                  "unit": "GB/s", "ms": ms, "gsamples_per_s": nS * nP / (ms * 1e-3) / 1e9,
                                  "traffic": None}
            ach = rooflines[key]["achieved"]
            rooflines[key]["frac"] = ach / rooflines[key]["peak"] if ach is not None else None
            tr = TRAFFIC_PER_STREAM_1024.get(key) if nP == 1024 else None
            rooflines[key]["traffic"] = tr * nS if tr else None
            if rooflines[key]["bound"] == "hbm":
                rooflines[key]["frac_of_write_fill"] = rooflines[key]["achieved"] / write_fill_gbs
    # dominant kernel = the launch with the largest share of the step
    dom = max(rooflines, key=lambda k: rooflines[k]["ms"])
    R = rooflines[dom]
    roofline = {"bound": R["bound"], "achieved": R["achieved"], "peak": R["peak"], "unit": R["unit"],
                "frac": R["frac"], "traffic": R.get("traffic"), "kernel": dom,
                "peak_source": int_src if R["bound"] == "alu" else f"{peak_src} HBM copy GB/s"}
    per_gen = {g: 2 * nS * nP / ((ms_u[g] + ms_f[g]) * 1e-3) / 1e9 for g in gens}

    # ----- end to end: same step through host buffers (device -> pinned host copies inside)
    e2e = None
    if not args.no_e2e:
        hu = torch.empty(nS * nP, dtype=torch.int32, pin_memory=True)
        hf = torch.empty(nS * nP, dtype=torch.float32, pin_memory=True)

        call_ms = {}

        def e2e_step():
            # the library's host-array fill: generation in blocks on the device,
            # each block's copy into the page-locked arrays overlapping the next
            for g in gens:
                for dt, fn, buf in (("u32", P.prand_generate_host_u32, hu), ("f32", P.prand_generate_host_f32, hf)):
                    t = time.perf_counter()
                    fn(handles[g], buf.data_ptr(), nP, sp)
                    call_ms.setdefault(f"{g}.{dt}", []).append(1e3 * (time.perf_counter() - t))
            return int(hu[0]) + int(hf[0] > 2)  # read back a result on the host

        for _ in range(2):  # warm-up: staging allocation, first touch of the host arrays
            e2e_step()
        call_ms.clear()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        # the host link's rate for context: a plain device-to-host copy of the
        # u32 output buffer into the same page-locked array (median of 3)
        cp = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hu.copy_(U, non_blocking=True)
            b.record(stream)
            b.synchronize()
            cp.append(a.elapsed_time(b))
        d2h_gbs = U.numel() * 4 / (statistics.median(cp) * 1e-3) / 1e9
        # the host link's rate: the faster of that copy and the fastest host
        # fill (an HBM-bound fill into host memory runs at the link's rate);
        # the step can be no faster than, per fill, the slower of its bytes at
        # that rate and its device time
        fill_bytes = nS * nP * 4
        link_gbs = max([d2h_gbs] + [fill_bytes / (min(v) * 1e-3) / 1e9 for v in call_ms.values()])
        bound_ms = sum(max(fill_bytes / (link_gbs * 1e9) * 1e3, ms_u[g]) + max(fill_bytes / (link_gbs * 1e9) * 1e3,
                                                                              ms_f[g]) for g in gens)
        e2e = {"value": world * samples_step * args.e2e_steps / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": len(gens) * nS * nP * 8,
               "steps": args.e2e_steps,
               "api": "prand_generate_host_u32 / _f32 into page-locked host arrays (written by the kernels directly)",
               "call_ms": {k: round(statistics.median(v), 2) for k, v in call_ms.items()},
               "slow": {k: [round(x, 1) for x in v if x > 1.5 * statistics.median(v)] for k, v in call_ms.items()},
               "d2h_copy_gb_per_s": round(d2h_gbs, 1), "link_gb_per_s": round(link_gbs, 1),
               "bound_gsamples_per_s": round(world * samples_step / (bound_ms * 1e-3) / 1e9, 2)}
        del hu, hf

    for h in handles.values():
        P.prand_destroy(h)
    del U, F
    torch.cuda.empty_cache()

    table = single = study = host_simd = None
    if not args.no_table and rank == 0:
        table = run_table(P, torch, sp, args)
        single = run_single(P, torch, sp, args)
        host_simd = run_host_simd(P, torch, sp, args)
    if not args.no_study and rank == 0:
        study = run_skipahead(P, torch, sp, args)
    batched = None
    if not args.no_batched and rank == 0:
        batched = run_batched(P, torch, sp, args)
    serving = None
    if not args.no_serving and rank == 0:
        serving = run_serving(P, args)

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "generators": gens, "n_streams_per_gpu": nS,
                       "n_per_stream": [nP, nP], "outputs": ["u32", "f32"],
                       "l2": "no flush: every step writes 8 GiB of outputs per generator (>> 129 MB L2)",
                       "parallelism": f"{world} GPU(s), disjoint stream ranges, no collective"},
            "roofline": roofline,
            "rooflines": rooflines,
            "write_fill": {"gb_per_s": write_fill_gbs, "bytes": write_fill_bytes,
                           "what": "torch fill_ of the u32 output buffer, write only, median of 10 (context)"},
            "per_generator_gsamples_per_s": per_gen,
            "init_ms": init_ms,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": e2e,
            "table": table,
            "single_stream": single,
            "host_simd": host_simd,
            "skipahead_study": study,
            "batched": batched,
            "serving": serving,
        }
        if args.gens or args.streams or args.per_stream:
            line["config"]["workload"] = f"custom: {','.join(gens)}; {nS} streams x ({nP} u32 + {nP} f32)"
        if world == 1 and not args.no_cpu_baseline and not (args.gens or args.streams or args.per_stream):
            rates, detail = oracle_rates(budget_s=args.cpu_budget)
            line["cpu_baseline"] = {
                "value": mix_throughput(rates) / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"first 4 streams of each generator, u32+f32 rounds of 2^10 outputs, "
                          f"~{args.cpu_budget:.0f} s of single-thread oracle time, extrapolated to the mix",
                "per_generator_samples_per_s": rates, "detail": detail}
            all_rates, cores = oracle_rates_all_cores(budget_s=args.cpu_budget)
            line["cpu_baseline"]["all_cores"] = {
                "value": mix_throughput(all_rates) / 1e9, "unit": UNIT, "cores": cores,
                "sample": f"one oracle process per core, each on 4 streams of its own, "
                          f"~{args.cpu_budget:.0f} s, extrapolated to the mix",
                "per_generator_samples_per_s": all_rates}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))
    return 0


def _time_calls(torch, stream, fn, warmup=3, reps=5):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_table(P, torch, sp, args):
    """All eleven generators, 2^16 block-split streams x 2^12 outputs (u32, then
    f32 on the continued streams), seed 12345: device time per fill (CUDA
    events, 5 timed fills after 3 warm-up fills; 1 GiB per fill >> L2).  HBM
    bytes = outputs + state read and written; the GM/GQ fills are integer-pipe
    bound, so their HBM fraction is small by nature."""
    hbm_peak, _ = _peaks()
    int_peak, int_src = getattr(args, "int_peak", None) or int_issue_peak(torch, torch.cuda.current_device(), None)
    stream = torch.cuda.current_stream()
    nS, nP = W.TABLE_STREAMS, W.TABLE_PER_STREAM
    U = torch.empty(nS * nP, dtype=torch.int32, device="cuda")
    out = {}
    for g in W.GENERATORS:
        h = P.prand_create(g, W.TABLE_SEED)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.prand_init_streams(h, 0, nS)
        torch.cuda.synchronize()
        init_ms = 1e3 * (time.perf_counter() - t0)
        res = {"init_ms": init_ms}
        for dt, fn in (("u32", P.prand_generate_u32), ("f32", P.prand_generate_f32)):
            ms = _time_calls(torch, stream, lambda: fn(h, U.data_ptr(), nP, sp))
            byts = nS * nP * 4 + 2 * nS * STATE_BYTES[g]
            res[dt] = {"ms": ms, "gsamples_per_s": nS * nP / (ms * 1e-3) / 1e9,
                       "hbm_frac": byts / (ms * 1e-3) / 1e9 / hbm_peak}
            if g in OPS_PER_WORD:
                tops = nS * nP * OPS_PER_WORD[g] / (ms * 1e-3) / 1e12
                res[dt]["int_tops"] = tops
                res[dt]["int_frac"] = tops / int_peak
        P.prand_destroy(h)
        out[g] = res
    del U
    torch.cuda.empty_cache()
    return {"workload": "11 generators x 2^16 streams x 2^12 outputs (u32, then f32), seed 12345",
            "int_peak_tops": int_peak, "int_peak_source": int_src,
            "ops_per_word": {g: OPS_PER_WORD[g] for g in W.GENERATORS if g in OPS_PER_WORD},
            "generators": out}


def run_skipahead(P, torch, sp, args):
    """The skip-ahead study of Table 3 on the GPU: for each generator the
    subsequence skipping 2^n values per step (n = the largest of the paper's
    rows) is output 0 of streams spaced 2^n apart; the frequency, serial and gap
    tests give p-values (the paper counts p outside [1e-3, 1 - 1e-3] as
    suspicious).  Times: spaced initialisation (the jumps) and generation,
    wall clock with a synchronize; the three count launches, CUDA events.  Then
    the count kernels alone over 2^30 words (4 GiB >> L2), against the HBM
    roofline: 4 bytes read per word."""
    hbm_peak, _ = _peaks()
    stream = torch.cuda.current_stream()
    kinds = {"frequency": P.TEST_FREQUENCY, "serial": P.TEST_SERIAL, "gap": P.TEST_GAP}
    tests = [(name, P.make_test(kinds[name], **kw)) for name, kw in W.STUDY_TESTS]
    cnt = torch.empty(4096, dtype=torch.int64, device="cuda")
    res, suspicious = {}, 0
    for g, n_skip in W.STUDY_SKIPS.items():
        N = W.STUDY_WORDS_MT if g == "MT19937" else W.STUDY_WORDS
        w = torch.empty(N, dtype=torch.int32, device="cuda")
        h = P.prand_create(g, W.STUDY_SEED)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.prand_init_streams_spaced(h, n_skip, 0, N)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        P.prand_generate_u32(h, w.data_ptr(), 1, sp)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        P.prand_destroy(h)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pv, counts = {}, []
        a.record(stream)
        for name, t in tests:
            c = cnt[:P.prand_test_cells(t)]
            P.prand_test_counts(t, w.data_ptr(), N, c.data_ptr(), sp)
            counts.append(c.clone())
        b.record(stream)
        torch.cuda.synchronize()
        for (name, t), c in zip(tests, counts):
            _, _, p = P.prand_test_evaluate(t, N, c.cpu().numpy().view("uint64").tolist())
            pv[name] = p
            suspicious += not (1e-3 <= p <= 1 - 1e-3)
        res[g] = {"skip_log2": n_skip, "words": N, "p": pv, "init_ms": 1e3 * (t1 - t0),
                  "generate_ms": 1e3 * (t2 - t1), "tests_ms": a.elapsed_time(b)}
        del w
    # count kernels alone on 2^30 words
    n = 1 << 30
    big = torch.empty(n, dtype=torch.int32, device="cuda")
    h = P.prand_create("LFSR113", 5)
    P.prand_init_streams(h, 0, 1 << 20)
    P.prand_generate_u32(h, big.data_ptr(), n >> 20, sp)
    P.prand_destroy(h)
    kern = {}
    for name, t in tests:
        c = cnt[:P.prand_test_cells(t)]
        ms = _time_calls(torch, stream, lambda: P.prand_test_counts(t, big.data_ptr(), n, c.data_ptr(), sp),
                         warmup=3, reps=5)
        gbs = 4.0 * n / (ms * 1e-3) / 1e9
        kern[name] = {"ms": ms, "gb_per_s": gbs, "hbm_frac": gbs / hbm_peak}
    del big, cnt
    torch.cuda.empty_cache()
    return {"workload": "Table 3 skip-ahead study: output 0 of 2^22 streams spaced 2^n apart (MT19937 2^20), "
                        "frequency 2^10 cells, serial 2^5 x 2^5, gap [0, 2^29) t = 48; seed 20140401",
            "generators": res, "p_outside_1e-3": suspicious, "tests_run": 3 * len(res),
            "count_kernels_2^30_words": kern}


def run_host_simd(P, torch, sp, args):
    """The host SIMD generators (no GPU): MT19937, LFSR113 and MRG32K3A, u32,
    2^16 streams x 2^10 outputs from states exported from a handle, on one
    host thread and on all of them; wall time of the call, best of 3 (the
    paper's SSE realisations ran one core of a Xeon X5670: MT19937 2.5e8,
    MRG32K3A 1.5e8, LFSR113 1.6e8 outputs/s, Table 6)."""
    import numpy as np
    n, nper = 1 << 16, 1 << 10
    out = np.empty(n * nper, dtype=np.uint32)
    res = {"workload": "2^16 streams x 2^10 u32 outputs per call, states exported from a handle (seed 5)",
           "host_threads": os.cpu_count()}
    for g in ("MT19937", "LFSR113", "MRG32K3A"):
        h = P.prand_create(g, 5)
        P.prand_init_streams(h, 0, n)
        sb = P.prand_device_state_bytes(g)
        dev = torch.empty(n * sb // 4, dtype=torch.int32, device="cuda")
        P.prand_export_states(h, dev.data_ptr(), sp)
        torch.cuda.synchronize()
        P.prand_destroy(h)
        st = dev.cpu().numpy().copy()
        del dev
        r = {}
        for label, threads in (("one_thread", 1), ("all_threads", 0)):
            best = None
            for _ in range(3):
                t0 = time.perf_counter()
                P.prand_host_generate(g, P.DTYPE_U32, st.ctypes.data, n, out.ctypes.data, nper, threads)
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            r[label] = {"gsamples_per_s": n * nper / best / 1e9, "ms": 1e3 * best}
        res[g] = r
    return res


def run_single(P, torch, sp, args):
    """One MRG32K3A stream from the default state, 2^20 outputs (u32 and f64):
    the launch- and latency-bound case (the library splits the stream into
    sections).  Device time per call, CUDA events over 50 calls (the 4-8 MiB
    output stays in L2)."""
    stream = torch.cuda.current_stream()
    n = W.SINGLE_LENGTH
    buf = torch.empty(n, dtype=torch.float64, device="cuda")
    h = P.prand_create("MRG32K3A", P.SEED_DEFAULT)
    P.prand_init_streams(h, 0, 1)
    res = {}
    for dt, fn in (("u32", P.prand_generate_u32), ("f64", P.prand_generate_f64)):
        ms = _time_calls(torch, stream, lambda: fn(h, buf.data_ptr(), n, sp), warmup=5, reps=50)
        res[dt] = {"us": 1e3 * ms, "gsamples_per_s": n / (ms * 1e-3) / 1e9}
    P.prand_destroy(h)
    del buf
    return {"workload": "MRG32K3A, default state, 1 stream x 2^20 outputs", **res}


def _batched_pair(P, torch, sp, reqspec, args):
    """One request list as a graph-replayed persistent launch (after the tile
    tuner) and as per-request launches: device times and whether the outputs
    agree bit for bit."""
    total = sum(n for _, _, n, _ in reqspec)
    buf = torch.empty(total, dtype=torch.int32, device="cuda")
    reqs, o = [], 0
    for gen, k, n, _ in reqspec:
        reqs.append((gen, P.DTYPE_U32, k, n, buf.data_ptr() + 4 * o))
        o += n
    t0 = time.perf_counter()
    tuned = P.prand_batch_autotune(reqs, 7, sp)
    tune_s = time.perf_counter() - t0
    plan = P.prand_batch_plan_create(reqs, 7)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        P.prand_batch_plan_launch(plan, sp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        P.prand_batch_plan_launch(plan, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    fused_ms = e0.elapsed_time(e1) / reps
    P.prand_batch_plan_destroy(plan)
    fused_copy = buf.clone()
    buf.zero_()
    torch.cuda.synchronize()
    per_ms = identical = None
    if not args.no_per_request:
        t0 = time.perf_counter()
        P.prand_batch_run_per_request(reqs, 7, sp)
        torch.cuda.synchronize()
        per_ms = 1e3 * (time.perf_counter() - t0)
        identical = bool(torch.equal(buf, fused_copy))
    del buf, fused_copy
    torch.cuda.empty_cache()
    return {"requests": len(reqspec), "outputs": total, "fused_graph_ms": fused_ms,
            "fused_gsamples_per_s": total / (fused_ms * 1e-3) / 1e9, "per_request_ms": per_ms,
            "speedup_vs_per_request": (per_ms / fused_ms) if per_ms else None, "outputs_identical": identical,
            "tuned": {"seclen_mrg_lfsr": tuned[0], "seclen_gm": tuned[1], "block": tuned[2], "row_bytes": tuned[3],
                      "best_ms": tuned[4], "tune_s": tune_s}}


def run_batched(P, torch, sp, args):
    """The batched workload: 10^4 requests (generator uniform over the eleven,
    stream uniform in [0, 1e19), length floor(2^(20 U)) u32 outputs), run as one
    persistent launch replayed from a CUDA graph, after the tile tuner; compared
    with the same requests as per-request plain launches (bit-identical output;
    both reach each stream by the same jump method).  The same comparison is
    repeated without the MT19937 requests, whose jump chains dominate both."""
    reqspec = W.batched_requests(10_000, seed=7)
    res = _batched_pair(P, torch, sp, reqspec, args)
    res["workload"] = "10^4 requests, gen uniform over 11, stream uniform [0,1e19), length floor(2^(20U)) u32, seed 7"
    res["mt_requests"] = sum(1 for g, _, _, _ in reqspec if g == "MT19937")
    res["without_mt19937"] = _batched_pair(P, torch, sp, [r for r in reqspec if r[0] != "MT19937"], args)
    return res


def run_serving(P, args):
    """The serving workload: Poisson arrivals at 5e4 req/s for 10 s, each request
    (generator uniform over the eleven, stream uniform in [0, 1e19), length
    floor(2^(6 + 16 U)), dtype u32/f32/f64 equiprobable), replayed open-loop by
    the library's native driver against the continuous-batching server."""
    arr = W.serving_arrivals(rate=args.serve_rate, seconds=args.serve_seconds, seed=11)
    reqs = [(g, d, k, n) for _, g, k, n, d in arr]
    times = [t for t, _, _, _, _ in arr]
    srv = P.prand_server_create(11, SERVE_OUTPUT_BYTES, 65536)
    try:
        lat, wall = P.prand_server_replay(srv, reqs, times)
        st = P.prand_server_stats(srv)
    finally:
        P.prand_server_destroy(srv)
    lat_ms = sorted(1e3 * x for x in lat)
    samples = sum(n for _, _, _, n in reqs)
    pct = lambda q: lat_ms[min(len(lat_ms) - 1, int(q * len(lat_ms)))]

    def pcts(v):
        v = sorted(v)
        at = lambda q: round(v[min(len(v) - 1, int(q * len(v)))], 3)
        return {"n": len(v), "p50_ms": at(0.5), "p99_ms": at(0.99), "max_ms": round(v[-1], 3)}

    # where the tail comes from: latency by generator and by length (2^6-2^10,
    # 2^10-2^14, 2^14-2^18, 2^18-2^22 outputs)
    by_gen, by_len = {}, {}
    for (g, _, _, n), x in zip(reqs, lat):
        by_gen.setdefault(g, []).append(1e3 * x)
        b = min(3, max(0, (int(n).bit_length() - 1 - 6) // 4))
        by_len.setdefault(f"2^{6 + 4 * b}-2^{10 + 4 * b}", []).append(1e3 * x)
    return {"workload": f"Poisson {args.serve_rate:g} req/s for {args.serve_seconds:g} s; gen uniform over 11, "
                        "stream uniform [0,1e19), length floor(2^(6+16U)), dtype u32/f32/f64 equiprobable",
            "requests": len(reqs), "samples": samples, "wall_s": wall,
            "gsamples_per_s": samples / wall / 1e9, "demanded_gsamples_per_s": samples / args.serve_seconds / 1e9,
            "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": lat_ms[-1],
            "by_generator": {g: pcts(v) for g, v in sorted(by_gen.items())},
            "by_length": {k: pcts(v) for k, v in sorted(by_len.items())},
            "resident_hit_rate": st["hits"] / max(1, st["hits"] + st["misses"] + st["restores"]),
            "batches": st["batches"], "spills": st["spills"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-per-request", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-table", action="store_true")
    ap.add_argument("--no-study", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=5e4)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=10.0)
    # smaller cases of single kernels (profiling); the default is the bulk-fill workload
    ap.add_argument("--gens", default="", help="comma list of generators (default MT19937,LFSR113,GM61)")
    ap.add_argument("--streams", type=int, default=0)
    ap.add_argument("--per-stream", type=int, default=0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
