#!/usr/bin/env python
"""Benchmark of the GB300 SquareSort.

Default workload (one step = one SquareSort of n = 2^28 uint32 keys with a
uint32 index payload, a 16384 x 16384 view): the steps cycle through four
seeded distributions -- uniform over [0, 2^32), that draw ascending, that
draw descending, and 16 distinct values.  Every step sorts its own copy of
the input, staged in HBM before the timed region (2 GiB per step, larger
than L2, so no flush is needed between steps).

Prints one JSON line (rank 0): throughput in Gkeys/s, the dominant kernel's
HBM roofline, the end-to-end figure through the C ABI with host buffers, the
CPU oracle's throughput on a bounded sample, and the SM clocks seen.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload plain|batch|serve]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gkeys/s & % HBM roofline, batched/served vs plain SquareSort; serve p50/p99"
UNIT = "Gkeys/s"
DISTS = ["uniform", "sorted", "reverse", "distinct16"]
DIST_SEED = {"uniform": 2, "sorted": 3, "reverse": 4, "distinct16": 5}
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["sq_kernels.cuh", "sq_sorter.cuh", "sq_types.cuh", "sq_radix.cuh"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2407_14801_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(family: str, workload: str):
    """DRAM bytes per launch of a kernel family from the committed ncu
    summary, or None when absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash()
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == family and parts[1] == workload:
                return float(parts[2]) if parts[3] == src else None
    return None


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"sq_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}



def make_clocks(local: int) -> "ClockSampler":
    vis = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    return ClockSampler(int(vis[local]) if local < len(vis) and vis[local].strip().isdigit() else local)


def profiled(sq, run):
    """Runs run() once more with per-launch CUDA events on (outside every
    timed region) and returns the library's statistics of that pass."""
    import torch

    torch.cuda.synchronize()
    sq.reset_stats()
    sq.set_profiling(True)
    try:
        run()
        torch.cuda.synchronize()
    finally:
        sq.set_profiling(False)
    return sq.stats()


def roofline_of(st, workload_name: str, note: str):
    """The dominant kernel family's achieved HBM bandwidth: its algorithmic
    bytes per launch (counted on the device) over its average launch time."""
    fams = [f for f in st["ms"] if st["launches"][f] > 0 and st["bytes"][f] > 0]
    dom = max(fams, key=lambda f: st["ms"][f])
    L = st["launches"][dom]
    bytes_per_launch = st["bytes"][dom] / L
    avg_ms = st["ms"][dom] / L
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    return {"bound": "hbm", "kernel": f"k_{dom}", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": profiled_traffic(dom, workload_name),
            "peak_source": f"{peak_src} (copy bandwidth)", "algorithmic_bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": avg_ms, "launches": L, "measured_in": note,
            "family_ms": {f: round(st["ms"][f], 3) for f in st["ms"] if st["launches"][f]}}


# ------------------------------------------------------------- workloads --

def make_inputs_u32(n: int, device, dists=DISTS):
    """The distributions as device tensors (int32 views of uint32)."""
    import numpy as np
    import torch

    import workloads as W

    out = {}
    if "uniform" in dists:
        uni = W.uniform_u32(n, DIST_SEED["uniform"])
        out["uniform"] = torch.from_numpy(uni.view(np.int32)).to(device)
    # "sorted" / "reverse" are a uniform draw ordered; sorting the draw on the
    # GPU gives the same bytes as workloads.sorted_u32 / reverse_u32, faster.
    for d in ("sorted", "reverse"):
        if d in dists:
            draw = torch.from_numpy(W.uniform_u32(n, DIST_SEED[d]).astype(np.int64)).to(device)
            srt = torch.sort(draw).values
            if d == "reverse":
                srt = torch.flip(srt, [0])
            out[d] = srt.to(torch.int32)  # values < 2^32 wrap to the int32 view of the uint32 bits
            del draw, srt
    if "distinct16" in dists:
        out["distinct16"] = torch.from_numpy(W.distinct16_u32(n, DIST_SEED["distinct16"]).view(np.int32)).to(device)
    return out


def check_sorted_u32(keys, vals, orig_keys):
    """Full-size check on the device: non-decreasing (key, val) order, vals a
    permutation, every key equal to the original key at its payload index."""
    import torch

    k = keys.to(torch.int64) & 0xFFFFFFFF
    v = vals.to(torch.int64) & 0xFFFFFFFF
    comp = (k - (1 << 31)) * (1 << 32) + v  # order-preserving and inside int64
    ok = bool((comp[1:] > comp[:-1]).all())
    n = keys.numel()
    seen = torch.zeros(n, dtype=torch.bool, device=keys.device)
    seen[v] = True
    ok = ok and bool(seen.all())
    ok = ok and bool((orig_keys[v] == keys).all())
    return ok


def np_sorted_ok(k0, v0, k, v, dt) -> bool:
    """Host check of one served request: the output is the input ordered by
    (ordinal(key), val), float32 by IEEE order with NaNs last and tied."""
    import numpy as np

    if dt == "f32":
        b = k0.view(np.uint32).astype(np.uint64)
        nan = (b & 0x7FFFFFFF) > 0x7F800000
        ords = np.where(nan, 0xFFFFFFFF, np.where(b & 0x80000000, b ^ 0xFFFFFFFF, b | 0x80000000))
        bits0, bits = k0.view(np.uint32), k.view(np.uint32)
    else:
        ords, bits0, bits = k0, k0, k
    order = np.lexsort((v0, ords))
    return bool((v == v0[order]).all() and (bits == bits0[order]).all())


# ----------------------------------------------------------- our impl -----

def bench_plain(args, sq, dist, rank, world, local):
    import numpy as np
    import torch

    import workloads as W

    dev = torch.device("cuda", local)
    n = args.n
    dists = args.dists.split(",")
    inputs = make_inputs_u32(n, dev, dists)
    iota = torch.arange(n, dtype=torch.int32, device=dev)
    total = args.warmup + args.steps
    seq = [dists[i % len(dists)] for i in range(total)]
    keys = [inputs[d].clone() for d in seq]
    vals = [iota.clone() for _ in seq]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    cutoff = args.cutoff
    for i in range(args.warmup):
        sq.sort(keys[i], vals[i], seed=i, dtype="u32", cutoff=cutoff, variant=args.variant)
    torch.cuda.synchronize()
    sq.reset_stats()
    clocks = make_clocks(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist_mod = dist
    from paper_2407_14801_gb300 import dist as D

    D.barrier(dist_mod)
    torch.cuda.synchronize()
    ev0.record(stream)
    t_wall0 = time.perf_counter()
    for i in range(args.warmup, total):
        sq.sort(keys[i], vals[i], seed=i, dtype="u32", cutoff=cutoff, variant=args.variant)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    D.barrier(dist_mod)
    clk = clocks.stop()
    st_timed = sq.stats()
    ms = ev0.elapsed_time(ev1)
    ms_max = D.max_over_ranks(ms, dist_mod, dev)
    value = world * args.steps * n / (ms_max / 1e3) / 1e9

    # correctness of every timed step (outside the timed region)
    ok = all(check_sorted_u32(keys[i], vals[i], inputs[seq[i]]) for i in range(args.warmup, total))

    # kernel-family split: the same sorts again on the same inputs, with
    # per-launch CUDA events on (a pass of its own, not the timed one)
    def again():
        for i in range(args.warmup, total):
            keys[i].copy_(inputs[seq[i]])
            vals[i].copy_(iota)
        torch.cuda.synchronize()
        for i in range(args.warmup, total):
            sq.sort(keys[i], vals[i], seed=i, dtype="u32", cutoff=cutoff, variant=args.variant)

    st = profiled(sq, again)
    del keys, vals
    torch.cuda.empty_cache()
    workload_name = f"plain_u32_n{n}" + ("" if args.variant == "algorithm1" else f"_{args.variant}")
    roofline = roofline_of(st, workload_name, "a profiling pass over the same sorts after the timed region")
    peak = roofline["peak"]
    # whole-step roofline against the ideal one-level traffic 6 w n (w = 8 bytes)
    step_frac = (6 * 8 * n) / (ms_max / args.steps / 1e3) / 1e9 / peak

    # end to end through the C ABI with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        e2e = bench_e2e(sq, n, min(args.steps, 4), dev, inputs, args.variant)
    del inputs
    torch.cuda.empty_cache()

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name, "n": n, "view": f"{int(n ** 0.5)}x{int(n ** 0.5)}",
                   "key": "uint32", "payload": "uint32 original index", "distributions": dists,
                   "distribution_seeds": {d: DIST_SEED[d] for d in dists},
                   "step_cycle": f"step i sorts distribution i mod {len(dists)}",
                   "cutoff": sq.get_cutoff("u32") if not cutoff else cutoff,
                   "variant": args.variant,
                   "l2": "inputs larger than L2 (each step sorts its own 2 GiB copy)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "step_hbm_frac_ideal_6wn": round(step_frac, 4),
        "e2e": e2e,
        "gpu_launches": int(sum(st_timed["launches"].values())),
        "rounds_per_step": st_timed["rounds"] / max(1, args.steps),
        "recursing_nodes_per_step": st_timed["nodes"] / max(1, args.steps),
        "wall_s": round(t_wall, 4),
        "clocks": clk,
        "verified": ok,
    }
    return out


def check_sorted_any(src_bits, keys_bits, vals, dtype) -> bool:
    """Device check for any key type: non-decreasing (ordinal(key), val), vals a
    permutation, every key's bits equal to the original key at its payload
    index -- together these pin the unique sorted result."""
    import torch

    n = keys_bits.numel()
    v = vals.to(torch.int64) & 0xFFFFFFFF
    if dtype == "u64":
        o = keys_bits ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=keys_bits.device)
    else:
        b = keys_bits.to(torch.int64) & 0xFFFFFFFF
        if dtype == "f32":
            nan = (b & 0x7FFFFFFF) > 0x7F800000
            neg = (b & 0x80000000) != 0
            b = torch.where(nan, torch.full_like(b, 0xFFFFFFFF), torch.where(neg, b ^ 0xFFFFFFFF, b | 0x80000000))
        o = b
    ok = bool(((o[1:] > o[:-1]) | ((o[1:] == o[:-1]) & (v[1:] > v[:-1]))).all())
    seen = torch.zeros(n, dtype=torch.bool, device=vals.device)
    seen[v] = True
    return ok and bool(seen.all()) and bool((src_bits[v] == keys_bits).all())


def bench_wide(args, sq, dist, rank, world, local):
    """Wide keys: n uint64 keys, Zipf(1.1) ranks over [1, 2^40] through a seeded
    bijection, and n float32 keys N(0,1) with 0.1% +-inf, 0.1% -0.0 and 0.01%
    NaN, index payload; one step sorts one array of each."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2407_14801_gb300 import dist as D

    dev = torch.device("cuda", local)
    n = args.wide_n
    src = {"u64": torch.from_numpy(W.zipf_u64(n, 31).view(np.int64)).to(dev),
           "f32": torch.from_numpy(W.normal_f32(n, 32)).to(dev)}
    iota = torch.arange(n, dtype=torch.int32, device=dev)
    total = args.warmup + args.steps
    bufs = [{d: (src[d].clone(), iota.clone()) for d in src} for _ in range(total)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def step(i):
        for d in ("u64", "f32"):
            k, v = bufs[i][d]
            sq.sort(k, v, seed=i, dtype=d, cutoff=args.cutoff)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    sq.reset_stats()
    clocks = make_clocks(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    D.barrier(dist)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.warmup, total):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    D.barrier(dist)
    clk = clocks.stop()
    st_timed = sq.stats()
    ms_max = D.max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    value = world * args.steps * 2 * n / (ms_max / 1e3) / 1e9
    bits = {"u64": lambda t: t, "f32": lambda t: t.view(torch.int32)}
    ok = all(check_sorted_any(bits[d](src[d]), bits[d](bufs[i][d][0]), bufs[i][d][1], d)
             for i in range(args.warmup, total) for d in src)

    def again():
        for i in range(args.warmup, total):
            for d in src:
                bufs[i][d][0].copy_(src[d])
                bufs[i][d][1].copy_(iota)
        torch.cuda.synchronize()
        for i in range(args.warmup, total):
            step(i)

    st = profiled(sq, again)
    del bufs
    torch.cuda.empty_cache()
    workload_name = f"wide_u64_f32_n{n}"
    roofline = roofline_of(st, workload_name, "a profiling pass over the same sorts after the timed region")
    peak = roofline["peak"]
    step_frac = (6 * (12 + 8) * n) / (ms_max / args.steps / 1e3) / 1e9 / peak
    e2e = None
    if not args.no_e2e:
        hosts = {d: src[d].cpu() for d in src}
        pins = {d: torch.empty_like(hosts[d]).pin_memory() for d in src}
        hv = torch.empty(n, dtype=torch.int32).pin_memory()
        iota_h = torch.arange(n, dtype=torch.int32)
        tot, reps = 0.0, min(args.steps, 2)
        for i in range(-1, reps):  # (the first round untimed: it grows the device memory pool)
            for d in src:
                pins[d].copy_(hosts[d])
                hv.copy_(iota_h)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sq.sort(pins[d], hv, seed=100 + i, dtype=d)
                if i >= 0:
                    tot += time.perf_counter() - t0
        e2e = {"value": round(reps * 2 * n / tot / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": (12 + 8) * n, "d2h_bytes_per_step": (12 + 8) * n, "steps": reps, "warmup": 1,
               "buffers": "pinned host, read by the first pass and written by the last through the device mapping"}
    return {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64+f32", "data": "synthetic",
        "config": {"workload": workload_name, "n_per_array": n, "keys": ["uint64 Zipf(1.1) over 2^40 ranks, bijection",
                                                                            "float32 N(0,1) + 0.1% inf, 0.1% -0, 0.01% NaN"],
                   "payload": "uint32 original index", "seeds": {"u64": 31, "f32": 32},
                   "step": "one uint64 sort and one float32 sort", "cutoff": args.cutoff or "tuned table",
                   "l2": "inputs larger than L2 (each step sorts its own copies)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "step_hbm_frac_ideal_6wn": round(step_frac, 4), "e2e": e2e,
        "gpu_launches": int(sum(st_timed["launches"].values())),
        "rounds_per_step": st_timed["rounds"] / max(1, args.steps), "clocks": clk, "verified": ok,
    }


def bench_e2e(sq, n, steps, dev, inputs, variant="algorithm1", threads=2):
    """End to end through sq_sort on page-locked host buffers (the first pass
    reads the input there, the last writes the result there).  Every step has
    its own buffers, filled before the timed region.  Measured twice: one call
    after the other, and from `threads` host threads, each calling sq_sort on
    its own stream, so that one sort's host traffic can overlap another's
    device work; the second is the reported value (at 2^28 it gains only a
    few percent: the passes over host memory take most of a call)."""
    import threading

    import torch

    names = list(inputs)
    src = {d: inputs[d].cpu() for d in names}
    iota = torch.arange(n, dtype=torch.int32)
    bufs = [(torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory())
            for _ in range(steps)]

    def fill():
        for i, (hk, hv) in enumerate(bufs):
            hk.copy_(src[names[i % len(names)]])
            hv.copy_(iota)

    streams = [torch.cuda.Stream(device=dev) for _ in range(threads)]
    fill()
    for w in range(threads):  # untimed: the first calls grow the device memory pool
        sq.sort(bufs[w % steps][0], bufs[w % steps][1], seed=90 + w, dtype="u32", variant=variant, stream=streams[w])
    fill()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (hk, hv) in enumerate(bufs):
        sq.sort(hk, hv, seed=100 + i, dtype="u32", variant=variant)  # H2D, sort, D2H inside the call
    single = steps * n / (time.perf_counter() - t0) / 1e9
    fill()
    torch.cuda.synchronize()
    errors = []

    def worker(w):
        try:
            torch.cuda.set_device(dev)
            for i in range(w, steps, threads):
                sq.sort(bufs[i][0], bufs[i][1], seed=200 + i, dtype="u32", variant=variant, stream=streams[w])
        except Exception as e:  # reported after the join
            errors.append(e)

    ths = [threading.Thread(target=worker, args=(w,)) for w in range(threads)]
    t0 = time.perf_counter()
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    conc = steps * n / (time.perf_counter() - t0) / 1e9
    if errors:
        raise errors[0]
    ok = all(check_sorted_any(inputs[names[i % len(names)]], bufs[i][0].to(dev), bufs[i][1].to(dev), "u32")
             for i in range(steps))
    return {"value": round(conc, 3), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
            "d2h_bytes_per_step": 8 * n, "steps": steps, "warmup": threads, "threads": threads,
            "single_stream_value": round(single, 3), "verified": ok,
            "buffers": "pinned host, one pair per step, read by the first pass and written by the last through the "
                       "device mapping"}


def cpu_baseline(sample_log2: int = 23, budget_s: float = 25.0, variant: str = "algorithm1", min_s: float = 12.0):
    """The CPU oracle, single-threaded, on a bounded sample of the workload:
    the first 2^sample_log2 keys of each distribution's generator, the four
    in turn until at least min_s seconds of sorting (at most budget_s)."""
    import numpy as np

    import oracle
    import workloads as W

    n = 1 << sample_log2
    done, t = 0, 0.0
    gens = {"uniform": W.uniform_u32, "sorted": W.sorted_u32, "reverse": W.reverse_u32,
            "distinct16": W.distinct16_u32}
    samples = {d: gens[d](n, DIST_SEED[d]) for d in DISTS}
    v = W.iota(n)
    i = 0
    while t < min_s and t < budget_s:
        d = DISTS[i % len(DISTS)]
        t0 = time.perf_counter()
        oracle.sort(samples[d], v, seed=1 + i, cutoff=16384, variant=variant)
        t += time.perf_counter() - t0
        done += n
        i += 1
    return {"value": round(done / t / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done // n} x 2^{sample_log2} uint32 keys (first keys of each distribution's generator), "
                      f"cutoff 16384, {variant}, single thread", "seconds": round(t, 2)}


def cpu_baseline_wide(sample_log2: int = 21, budget_s: float = 20.0, min_s: float = 12.0):
    """The CPU oracle, single-threaded, on the first 2^sample_log2 keys of the
    wide workload's two generators, in turn until at least min_s seconds of
    sorting (at most budget_s)."""
    import oracle
    import workloads as W

    n = 1 << sample_log2
    done, t, i = 0, 0.0, 0
    samples = (("u64", W.zipf_u64(n, 31)), ("f32", W.normal_f32(n, 32)))
    while t < min_s and t < budget_s:
        dt, k = samples[i % 2]
        t0 = time.perf_counter()
        oracle.sort(k, W.iota(n), seed=1 + i, cutoff=16384, dtype=dt)
        t += time.perf_counter() - t0
        done += n
        i += 1
    return {"value": round(done / t / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{i} sorts of 2^{sample_log2} keys, uint64 Zipf and float32 in turn (first keys of the "
                      f"workload's generators), cutoff 16384, single thread", "seconds": round(t, 2)}


def bench_huge(args, sq, dist, rank, world, local):
    """2^31 uint32 keys (uniform, drawn on the device from a seeded generator)
    with an index payload: a root of 46341 columns whose 46340 pivots a
    cluster of 8 CTAs sorts and the bucket count reads from global memory.
    One input copy is sorted per step (restored outside the timed sorts, each
    sort timed by CUDA events on the launch stream); end to end through
    sq_sort on page-locked host buffers."""
    import torch

    from paper_2407_14801_gb300 import dist as D

    dev = torch.device("cuda", local)
    n = args.huge_n
    g = torch.Generator(device=dev)
    g.manual_seed(31 + rank)
    src = torch.randint(-(1 << 31), 1 << 31, (n,), dtype=torch.int32, device=dev, generator=g)
    iota = torch.arange(n, dtype=torch.int32, device=dev)
    keys, vals = src.clone(), iota.clone()
    stream = torch.cuda.current_stream()

    def restore():
        keys.copy_(src)
        vals.copy_(iota)
        torch.cuda.synchronize()

    for i in range(args.warmup):
        restore()
        sq.sort(keys, vals, seed=i, dtype="u32", cutoff=args.cutoff)
    sq.reset_stats()
    clocks = make_clocks(local)
    clocks.start()
    ms, ok = 0.0, True
    D.barrier(dist)
    for i in range(args.steps):
        restore()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sq.sort(keys, vals, seed=100 + i, dtype="u32", cutoff=args.cutoff)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms += ev0.elapsed_time(ev1)
        if i == 0:
            ok = check_sorted_any(src, keys, vals, "u32")
    D.barrier(dist)
    clk = clocks.stop()
    st_timed = sq.stats()
    ms_max = D.max_over_ranks(ms, dist, dev)
    value = world * args.steps * n / (ms_max / 1e3) / 1e9

    def again():
        for i in range(min(args.steps, 2)):
            restore()
            sq.sort(keys, vals, seed=200 + i, dtype="u32", cutoff=args.cutoff)

    st = profiled(sq, again)
    del keys, vals
    torch.cuda.empty_cache()
    workload_name = f"huge_u32_n{n}"
    roofline = roofline_of(st, workload_name, "a profiling pass over two more sorts after the timed ones")
    step_frac = (6 * 8 * n) / (ms_max / args.steps / 1e3) / 1e9 / roofline["peak"]
    e2e = None
    if not args.no_e2e:
        hk = torch.empty(n, dtype=torch.int32).pin_memory()
        hv = torch.empty(n, dtype=torch.int32).pin_memory()
        tot, reps = 0.0, min(args.steps, 3)
        for i in range(-1, reps):  # (the first untimed: it grows the device memory pool)
            hk.copy_(src)
            hv.copy_(iota)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sq.sort(hk, hv, seed=300 + i, dtype="u32")  # reads and writes the host buffers
            if i >= 0:
                tot += time.perf_counter() - t0
        ok = ok and check_sorted_any(src, hk.to(dev), hv.to(dev), "u32")
        e2e = {"value": round(reps * n / tot / 1e9, 3), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 8 * n, "steps": reps, "warmup": 1,
               "buffers": "pinned host, read by the first pass and written by the last through the device mapping"}
        del hk, hv
    return {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name, "n": n, "key": "uint32 uniform (torch generator, seed 31 + rank)",
                   "payload": "uint32 original index", "cutoff": args.cutoff or sq.get_cutoff("u32"),
                   "root": f"{int(n ** 0.5) + 1} columns, pivots sorted by a cluster of 8 CTAs",
                   "l2": "inputs larger than L2 (restored before each timed sort)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "step_hbm_frac_ideal_6wn": round(step_frac, 4), "e2e": e2e,
        "gpu_launches": int(sum(st_timed["launches"].values())),
        "rounds_per_step": st_timed["rounds"] / max(1, args.steps), "clocks": clk, "verified": ok,
    }


def cpu_baseline_huge(sample_log2: int = 23, budget_s: float = 25.0, min_s: float = 12.0):
    """The CPU oracle, single-threaded, on 2^sample_log2-key uniform uint32
    samples until at least min_s seconds of sorting."""
    import oracle
    import workloads as W

    n = 1 << sample_log2
    k = W.uniform_u32(n, 31)
    v = W.iota(n)
    done, t, i = 0, 0.0, 0
    while t < min_s and t < budget_s:
        t0 = time.perf_counter()
        oracle.sort(k, v, seed=1 + i, cutoff=16384)
        t += time.perf_counter() - t0
        done += n
        i += 1
    return {"value": round(done / t / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{i} sorts of 2^{sample_log2} uniform uint32 keys, cutoff 16384, single thread",
            "seconds": round(t, 2)}


def run_ours(args):
    import torch

    from paper_2407_14801_gb300 import dist as D

    rank, world, local = D.rank_world()
    torch.cuda.set_device(local)
    dist = D.init()
    import paper_2407_14801_gb300 as sq

    sq.lib()
    sq.set_launch_mode(args.launch_mode)
    if args.workload == "plain":
        out = bench_plain(args, sq, dist, rank, world, local)
        if rank == 0 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(variant=args.variant)
    elif args.workload == "wide":
        out = bench_wide(args, sq, dist, rank, world, local)
        if rank == 0 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_wide()
    elif args.workload == "batch":
        out = bench_batch(args, sq, dist, rank, world, local)
        if rank == 0 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_batch(args)
    elif args.workload == "huge":
        out = bench_huge(args, sq, dist, rank, world, local)
        if rank == 0 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_huge()
    elif args.workload == "serve":
        out = bench_serve(args, sq, dist, rank, world, local)
        if rank == 0 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_serve(args)
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------- batched and served ----

def bench_batch(args, sq, dist, rank, world, local):
    """4096 independent uint32 instances, sizes log-uniform in [2^8, 2^20],
    uniform keys, index payload, seed 7: one sq_sort_batch call per step
    against one sq_sort call per instance.  Ranks take disjoint shares.
    The instances lie end to end in one device buffer (each a view)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2407_14801_gb300 import dist as D

    dev = torch.device("cuda", local)
    count = args.batch_count
    sizes = W.batch_sizes(count, 7, args.batch_lo, args.batch_hi)
    mine = list(D.shard(count, rank, world))
    my_sizes = [int(sizes[i]) for i in mine]
    offs = np.concatenate([[0], np.cumsum(my_sizes)]).astype(np.int64)
    total_keys = int(offs[-1])
    flat = np.empty(total_keys, dtype=np.uint32)
    for j, i in enumerate(mine):
        flat[offs[j]:offs[j + 1]] = W.uniform_u32(my_sizes[j], (7 << 20) + i + 1)
    src = torch.from_numpy(flat.view(np.int32)).to(dev)
    iota = torch.cat([torch.arange(m, dtype=torch.int32, device=dev) for m in my_sizes]) if my_sizes else \
        torch.empty(0, dtype=torch.int32, device=dev)
    keys, vals = src.clone(), iota.clone()
    views = [(keys[offs[j]:offs[j + 1]], vals[offs[j]:offs[j + 1]], 7 + i) for j, i in enumerate(mine)]
    stream = torch.cuda.current_stream()

    def restore():
        keys.copy_(src)
        vals.copy_(iota)
        torch.cuda.synchronize()

    def run_batched():
        sq.sort_batch(views)

    def run_single():
        for k, v, seed in views:
            sq.sort(k, v, seed=seed, dtype="u32")

    def timed(fn, steps, warm, clocks=None):
        for _ in range(warm):
            restore()
            fn()
        if clocks is not None:
            clocks.start()
        tot = 0.0
        for _ in range(steps):
            restore()
            D.barrier(dist)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        clk = clocks.stop() if clocks is not None else None
        return D.max_over_ranks(tot, dist, dev) / steps, clk

    clocks = make_clocks(local)
    sq.reset_stats()
    ms_b, clk = timed(run_batched, args.steps, args.warmup, clocks)
    st_timed = sq.stats()
    launches = sum(st_timed["launches"].values()) / max(1, args.steps + args.warmup)
    ms_s = None if args.batch_no_single else timed(run_single, max(1, args.steps // 4), 1)[0]
    # correctness of one batched step, every instance, on the device
    restore()
    run_batched()
    torch.cuda.synchronize()
    ok = all(check_sorted_u32(k, v, src[offs[j]:offs[j + 1]]) for j, (k, v, _) in enumerate(views))

    def again():
        restore()
        run_batched()

    st = profiled(sq, again)
    workload_name = f"batch_u32_{count}_instances_2^{args.batch_lo}..2^{args.batch_hi}"
    roofline = roofline_of(st, workload_name, "a profiling pass over one batched step after the timed region")

    # end to end: the instances from pinned host memory, the batched call, and
    # the results back, every step
    e2e = None
    if not args.no_e2e and total_keys:
        hk = torch.from_numpy(flat.view(np.int32)).pin_memory()
        hv = iota.cpu().pin_memory()
        ok_h = torch.empty_like(hk).pin_memory()
        ov_h = torch.empty_like(hv).pin_memory()
        reps, tot = min(args.steps, 4), 0.0
        for r in range(-1, reps):  # (the first untimed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            keys.copy_(hk, non_blocking=True)
            vals.copy_(hv, non_blocking=True)
            run_batched()
            ok_h.copy_(keys, non_blocking=True)
            ov_h.copy_(vals, non_blocking=True)
            torch.cuda.synchronize()
            if r >= 0:
                tot += time.perf_counter() - t0
        e2e = {"value": round(world * reps * total_keys / tot / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": 8 * total_keys, "d2h_bytes_per_step": 8 * total_keys, "steps": reps,
               "warmup": 1, "buffers": "pinned host; copies to and from device buffers around sq_sort_batch"}
    all_keys = int(sizes.sum())
    gk_b = world * total_keys / (ms_b / 1e3) / 1e9
    gk_s = world * total_keys / (ms_s / 1e3) / 1e9 if ms_s else None
    return {"metric": METRIC, "value": round(gk_b, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_b, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_name, "instances": count,
                       "total_keys": all_keys, "seed": 7, "cutoff": "tuned table",
                       "l2": "inputs larger than L2 (2 x 4 bytes x total_keys, restored before every step)",
                       "parallelism": f"instances sharded over {world} rank(s)"},
            "roofline": roofline, "e2e": e2e,
            "per_instance_launches": ({"value": round(gk_s, 3), "unit": UNIT, "ms_per_step": round(ms_s, 3)}
                                      if ms_s else None),
            "batched_over_per_instance": round(ms_s / ms_b, 2) if ms_s else None,
            "gpu_launches": int(round(launches)), "gpu_launches_per_step": launches,
            "rounds_per_step": st_timed["rounds"] / max(1, args.steps + args.warmup), "clocks": clk,
            "verified": ok}


def cpu_baseline_batch(args, budget_s: float = 20.0):
    """The CPU oracle, single-threaded, on the batch's first instances (same
    sizes and keys) until about budget_s seconds of sorting."""
    import oracle
    import workloads as W

    sizes = W.batch_sizes(args.batch_count, 7, args.batch_lo, args.batch_hi)
    done, t, i = 0, 0.0, 0
    while i < len(sizes) and t < budget_s:
        k = W.uniform_u32(int(sizes[i]), (7 << 20) + i + 1)
        t0 = time.perf_counter()
        oracle.sort(k, W.iota(k.size), seed=7 + i, cutoff=16384)
        t += time.perf_counter() - t0
        done += k.size
        i += 1
    return {"value": round(done / t / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the first {i} instances of the batch ({done} keys), cutoff 16384, single thread",
            "seconds": round(t, 2)}


class RingArena:
    """Request buffers in one page-locked host allocation, handed out in
    request order and returned in any order (a ring whose tail advances over
    the returned prefix)."""

    def __init__(self, nbytes: int):
        import collections
        import threading

        import torch

        self.size = nbytes
        self.buf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        self.np = self.buf.numpy()
        self.recs = collections.deque()
        self.lock = threading.Lock()

    def alloc(self, nbytes: int):
        with self.lock:
            if nbytes > self.size:
                raise ValueError("request larger than the arena")
            if not self.recs:
                start = 0
            else:
                head, tail = self.recs[-1][1], self.recs[0][0]
                if self.recs[-1][0] >= tail:  # live bytes [tail, head): free at the end, then the start
                    if head + nbytes <= self.size:
                        start = head
                    elif nbytes <= tail:
                        start = 0
                    else:
                        return None
                elif head + nbytes <= tail:  # wrapped: live [tail, end) and [0, head), free [head, tail)
                    start = head
                else:
                    return None
            rec = [start, start + nbytes, False]
            self.recs.append(rec)
            return rec

    def free(self, rec):
        with self.lock:
            rec[2] = True
            while self.recs and self.recs[0][2]:
                self.recs.popleft()


def bench_serve(args, sq, dist, rank, world, local):
    """A Poisson stream of sort requests (sizes log-uniform in [2^10, 2^24],
    key type uniform over uint32 / uint64 / float32 with the workload
    generators, index payload) served under a 16 GiB budget at 80% of the
    saturation rate of a closed-loop run; keys/s, p50/p99 submit-to-done
    latency, and the same requests through one sq_sort call each.

    Request i holds n_i keys cut at a seeded offset from a 2^25-key draw of
    its key type's generator (payload: its own index 0..n_i-1).  Its buffers
    are page-locked host memory (as a serving process keeps them), filled
    from the draws by a producer thread ahead of the request's arrival and
    returned once the request is done, so only the requests in flight hold
    memory."""
    import threading

    import numpy as np
    import torch

    import workloads as W

    nreq = args.serve_requests
    reqs = W.serve_requests(nreq, 11, rate_per_s=1.0)  # arrival times rescaled below
    src_n = 1 << 25
    srcs = {"u32": torch.from_numpy(W.uniform_u32(src_n, 1101).view(np.int32)),
            "u64": torch.from_numpy(W.zipf_u64(src_n, 1102).view(np.int64)),
            "f32": torch.from_numpy(W.normal_f32(src_n, 1103))}
    iota = torch.arange(1 << 24, dtype=torch.int32)
    wbytes = {"u32": 4, "u64": 8, "f32": 4}
    tdt = {"u32": torch.int32, "u64": torch.int64, "f32": torch.float32}
    npdt = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32}
    g = np.random.default_rng(1104)
    offs = [int(g.integers(0, src_n - n + 1)) for (_, n, _, _) in reqs]
    keys_total = sum(n for (_, n, _, _) in reqs)
    budget = 16 << 30
    arena = RingArena(args.serve_arena_gb << 30)
    verify_every = max(1, nreq // 2000)

    def producer(ready, stop, count):
        for i in range(count):
            _, n, dt, _ = reqs[i]
            kb = (n * wbytes[dt] + 255) & ~255
            need = kb + ((n * 4 + 255) & ~255)
            rec = arena.alloc(need)
            while rec is None:
                if stop[0]:
                    return
                time.sleep(0.0005)
                rec = arena.alloc(need)
            if stop[0]:
                return
            k = arena.np[rec[0]:rec[0] + n * wbytes[dt]].view(npdt[dt])
            v = arena.np[rec[0] + kb:rec[0] + kb + n * 4].view(np.uint32)
            torch.from_numpy(k.view(np.uint8)).view(tdt[dt]).copy_(srcs[dt][offs[i]:offs[i] + n])
            torch.from_numpy(v.view(np.int32)).copy_(iota[:n])
            ready.append((i, rec, k, v))

    def start_producer(count):
        ready, stop = [], [False]
        th = threading.Thread(target=producer, args=(ready, stop, count), daemon=True)
        th.start()
        return ready, stop, th

    def end_producer(stop, th):
        stop[0] = True
        th.join()
        arena.recs.clear()  # (requests filled but not run are dropped)

    def check(i, k, v):
        _, n, dt, _ = reqs[i]
        s0 = srcs[dt][offs[i]:offs[i] + n].to(local)
        kk = torch.from_numpy(k.view(np.int64 if dt == "u64" else np.int32)).to(local)  # key bits
        vv = torch.from_numpy(v.view(np.int32)).to(local)
        if dt == "f32":
            s0 = s0.view(torch.int32)
        return check_sorted_any(s0, kk, vv, dt)

    def run_served(rate, clocks=None, limit=None):
        """Closed loop (rate 0: every request submitted as soon as its
        buffers are filled) or Poisson arrivals at `rate` requests/s."""
        count = limit or nreq
        ready, stop, th = start_producer(count)
        srv = sq.Server(budget, device=local)
        lat, pending, nready, i_next, ok, nchk = [], {}, 0, 0, True, 0
        if clocks is not None:
            clocks.start()
        t0 = time.perf_counter()
        try:
            while i_next < count or pending:
                now = time.perf_counter() - t0
                while i_next < count and nready < len(ready) and (not rate or reqs[i_next][0] / rate <= now):
                    i, rec, k, v = ready[nready]
                    nready += 1
                    pending[srv.submit(k, v, seed=i, dtype=reqs[i][2])] = (i, rec, k, v)
                    i_next += 1
                for t in list(pending):
                    r = srv.poll(t)
                    if r is not None:
                        i, rec, k, v = pending.pop(t)
                        if r[0] != 0:
                            raise RuntimeError(f"request {i} failed with status {r[0]}")
                        lat.append(r[1])
                        if i % verify_every == 0:
                            ok = ok and check(i, k, v)
                            nchk += 1
                        arena.free(rec)
                time.sleep(0.0002)
            wall = time.perf_counter() - t0
        finally:
            srv.close()
            end_producer(stop, th)
        clk = clocks.stop() if clocks is not None else None
        keys = sum(reqs[i][1] for i in range(count))
        return wall, keys, np.array(lat), ok, nchk, clk

    def run_per_request(limit=None):
        """The same requests, closed loop, through one synchronous sq_sort
        call each (host buffers: the call stages them itself)."""
        count = limit or nreq
        ready, stop, th = start_producer(count)
        t0 = time.perf_counter()
        ok, nchk = True, 0
        try:
            for j in range(count):
                while j >= len(ready):
                    time.sleep(0.0002)
                i, rec, k, v = ready[j]
                sq.sort(k, v, seed=i, dtype=reqs[i][2])
                if i % verify_every == 0:
                    ok = ok and check(i, k, v)
                    nchk += 1
                arena.free(rec)
            wall = time.perf_counter() - t0
        finally:
            end_producer(stop, th)
        return wall, sum(reqs[i][1] for i in range(count)), ok, nchk

    # the producer's own rate (host copies into page-locked memory), alone:
    # every filled request is returned at once
    probe = min(nreq, 2000)
    t0 = time.perf_counter()
    ready, stop, th = start_producer(probe)
    j = 0
    while j < probe:
        if j < len(ready):
            arena.free(ready[j][1])
            j += 1
        else:
            time.sleep(0.0002)
    fill_s = time.perf_counter() - t0
    end_producer(stop, th)
    fill_keys = sum(reqs[i][1] for i in range(probe))

    warm = min(nreq, 200)
    run_served(0.0, limit=warm)  # warm-up: engines, pools, graphs
    wall_sat, kk, _, ok_sat, chk_sat, _ = run_served(0.0)
    sat_rps = nreq / wall_sat
    clocks = make_clocks(local)
    wall, kk, lat, ok_run, chk_run, clk = run_served(0.8 * sat_rps, clocks=clocks)
    per = None
    if not args.serve_no_single:
        wall_one, kk1, ok_one, chk_one = run_per_request()
        per = {"value": round(kk1 / wall_one / 1e9, 3), "unit": UNIT, "seconds": round(wall_one, 2),
               "verified": ok_one, "verified_requests": chk_one}
    st = profiled(sq, lambda: run_served(0.0, limit=min(nreq, 3000)))
    workload = f"serve_{nreq}_poisson_requests_2^10..2^24"
    roofline = roofline_of(st, workload, "a profiling pass over the first 3000 requests, closed loop")
    value = keys_total / wall / 1e9
    sat = keys_total / wall_sat / 1e9
    h2d = sum(n * (wbytes[dt] + 4) for (_, n, dt, _) in reqs)
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": nreq, "warmup": warm, "ms_per_step": round(wall / nreq * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64/f32", "data": "synthetic",
            "config": {"workload": workload, "requests": nreq, "mean_keys": keys_total / nreq,
                       "budget_bytes": budget, "arrival_rate_rps": round(0.8 * sat_rps, 2),
                       "saturation_rps": round(sat_rps, 2), "request_buffers": "pinned host ring arena",
                       "request_keys": "slices of a 2^25-key draw per key type at seeded offsets",
                       "l2": "inputs larger than L2 (requests stream from host memory)"},
            "saturation_keys_per_s": round(sat, 3),
            "per_request_sq_sort": per,
            "served_over_per_request": round(sat / per["value"], 2) if per else None,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean())},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d // nreq,
                    "d2h_bytes_per_step": h2d // nreq,
                    "note": "the served rate itself: requests arrive and leave in host memory"},
            "host_fill_keys_per_s": round(fill_keys / fill_s / 1e9, 3),
            "roofline": roofline, "gpu_launches": int(sum(st["launches"].values())),
            "clocks": clk, "verified": bool(ok_sat and ok_run),
            "verified_requests": {"saturation": chk_sat, "poisson": chk_run, "every": verify_every}}


def cpu_baseline_serve(args, budget_s: float = 20.0):
    """The CPU oracle, single-threaded, on the first requests of the stream
    (same sizes and key types) until about budget_s seconds of sorting."""
    import oracle
    import workloads as W

    reqs = W.serve_requests(args.serve_requests, 11, rate_per_s=1.0)
    done, t, i = 0, 0.0, 0
    while i < len(reqs) and t < budget_s:
        _, n, dt, ks = reqs[i]
        k = W.keys_for(dt, n, ks)
        t0 = time.perf_counter()
        oracle.sort(k, W.iota(n), seed=i, cutoff=16384, dtype=dt)
        t += time.perf_counter() - t0
        done += n
        i += 1
    return {"value": round(done / t / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the first {i} requests of the stream ({done} keys), cutoff 16384, single thread",
            "seconds": round(t, 2)}


# ----------------------------------------------------- the reference arm --

def run_reference(args):
    """The CPU oracle timed on the host cores: each step one bounded sample
    (2^20 keys) of the workload, cycling through the four distributions."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    import workloads as W

    n = 1 << 20
    gens = {"uniform": W.uniform_u32, "sorted": W.sorted_u32, "reverse": W.reverse_u32,
            "distinct16": W.distinct16_u32}
    samples = [(gens[d](n, DIST_SEED[d]), W.iota(n)) for d in DISTS]
    for i in range(args.warmup):
        k, v = samples[i % 4]
        oracle.sort(k, v, seed=i, cutoff=16384)
    t0 = time.perf_counter()
    for i in range(args.steps):
        k, v = samples[i % 4]
        oracle.sort(k, v, seed=i, cutoff=16384)
    t = time.perf_counter() - t0
    value = args.steps * n / t / 1e9
    sample = f"2^20 uint32 keys per step (first keys of each distribution's generator), cutoff 16384"
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"plain_u32_n{1 << 28}", "sample_n": n, "distributions": DISTS},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain", choices=["plain", "wide", "batch", "serve", "huge"])
    ap.add_argument("--n", type=int, default=1 << 28)
    ap.add_argument("--cutoff", type=int, default=0)
    ap.add_argument("--variant", default="algorithm1", choices=["algorithm1", "appendix"],
                    help="plain workload: Algorithm 1, or the variant of the paper's appendix code")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-lo", type=int, default=8, help="log2 of the smallest batch instance")
    ap.add_argument("--batch-hi", type=int, default=20, help="log2 of the largest batch instance")
    ap.add_argument("--batch-no-single", action="store_true",
                    help="skip the per-instance comparison (profiling runs)")
    ap.add_argument("--wide-n", type=int, default=1 << 26, help="keys per array of the wide workload")
    ap.add_argument("--huge-n", type=int, default=1 << 31, help="keys of the huge workload (uint32)")
    ap.add_argument("--launch-mode", default="auto", choices=["auto", "host", "graph"],
                    help="how recursion rounds are launched (profilers cannot see kernels inside graph loops)")
    ap.add_argument("--dists", default=",".join(DISTS), help="comma-separated subset (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=100000)
    ap.add_argument("--serve-arena-gb", type=int, default=8, help="page-locked host memory for requests in flight")
    ap.add_argument("--serve-no-single", action="store_true", help="skip the one-sq_sort-per-request comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
