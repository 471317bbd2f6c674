"""Leaf-cutoff autotuner.

Algorithm 1 stops recursing once a subproblem has at most `cutoff` elements
and sorts it directly; Section 4.2 sweeps that threshold and finds the best
value depends on the machine and the input size.  This module does the same
sweep on the local GPU: for each key type and each size 2^lg it times
``sq_sort_ex`` with every candidate cutoff on uniform random keys and keeps
the fastest, then writes ``tuning.json`` beside the package, which the binding
applies (``sq_set_cutoff_table``) when it loads the library.  The cutoff only
changes the shape of the recursion, never the sorted result.

    python -m paper_2407_14801_gb300.autotune [--lg 16:28] [--dtypes u32,u64,f32]

The same timing loop also runs the paper's cutoff experiment (Section 4.2:
normalised time against n for several cutoffs, where each extra recursion
level shows as a step): ``--sweep`` times every (n, cutoff) pair, records
nanoseconds per element per log2 n and the recursion depth the sort took,
and writes ``cutoff_sweep.json``; ``--report`` renders it as a table.

    python -m paper_2407_14801_gb300.autotune --sweep [--lg 10:28:2] [--cutoffs 64,256,1024,4096,16384,65536]
    python -m paper_2407_14801_gb300.autotune --report cutoff_sweep.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

CANDIDATES = (2048, 8192, 16384, 32768, 65536)


TIE = 0.02  # a smaller cutoff must beat the largest one by this fraction


def choose(ms: dict, tie: float = TIE) -> int:
    """The cutoff to use given {cutoff: median ms}: the fastest, except that
    a cutoff within `tie` of the fastest time wins if it is larger (fewer
    recursion levels; small differences are timing noise)."""
    best = min(ms.values())
    return max(int(c) for c, t in ms.items() if t <= best * (1.0 + tie))


def fill(best: dict) -> dict:
    """Extends {log2 n: cutoff} measured at some sizes to every log2 n in
    [0, 64): each size takes the nearest measured one (the smaller on a tie)."""
    got = sorted(int(k) for k in best)
    if not got:
        return {}
    out = {}
    for lg in range(64):
        near = min(got, key=lambda g: (abs(g - lg), g))
        out[str(lg)] = int(best[str(near)] if str(near) in best else best[near])
    return out


def retable(median_ms: dict) -> dict:
    """{dtype: {log2 n: {cutoff: ms}}} -> {dtype: {log2 n: cutoff}} for all log2 n."""
    return {dt: fill({lg: choose(ms) for lg, ms in per.items()}) for dt, per in median_ms.items()}


def _device_keys(torch, dtype: str, n: int, gen):
    if dtype == "u32":
        return torch.randint(-(2**31), 2**31, (n,), dtype=torch.int32, device="cuda", generator=gen)
    if dtype == "u64":
        return torch.randint(-(2**63), 2**63 - 1, (n,), dtype=torch.int64, device="cuda", generator=gen)
    return torch.randn(n, dtype=torch.float32, device="cuda", generator=gen)


def time_cutoff(sq, torch, src, vals0, dtype: str, cutoff: int, reps: int) -> float:
    """Median milliseconds of one sort of `src` (copied afresh every rep)."""
    keys, vals = torch.empty_like(src), torch.empty_like(vals0)
    stream = torch.cuda.current_stream()
    times = []
    for r in range(reps + 1):
        keys.copy_(src)
        vals.copy_(vals0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sq.sort(keys, vals, seed=r + 1, dtype=dtype, cutoff=cutoff)
        b.record(stream)
        b.synchronize()
        if r:  # the first run warms caches and the allocator
            times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


RADIX_CLASSES = tuple(range(2, 11))  # leaf classes with a radix kernel (32-bit key ordinals)


def class_size(c: int) -> int:
    """The largest leaf of size class c: 64, 512, 2048, then (c - 2) * 8192."""
    return 64 if c == 0 else 512 if c == 1 else 2048 if c == 2 else (c - 2) * 8192


def choose_radix(ms_radix: float, ms_merge: float, tie: float = TIE) -> bool:
    """Radix for a class unless the merge sort is faster by more than `tie`
    (the radix kernels are the default)."""
    return ms_radix <= ms_merge * (1.0 + tie)


def time_leaves(sq, torch, dtype: str, n: int, key_bits: int, reps: int) -> float:
    """Median ms of one sq_sort_batch of 2^25 / n independent n-key instances
    (each a single leaf: the cutoff is the largest leaf), keys uniform over
    [0, 2^key_bits) (float32: normal deviates scaled into that many ranks)."""
    count = max(1, (1 << 25) // n)
    g = torch.Generator(device="cuda")
    g.manual_seed(n + key_bits)
    if dtype == "u32":
        k = torch.randint(0, 1 << key_bits, (count * n,), dtype=torch.int64, device="cuda", generator=g)
        src = (k - (1 << 31) * (key_bits == 32)).to(torch.int32)
    else:
        src = torch.randn(count * n, dtype=torch.float32, device="cuda", generator=g)
        if key_bits < 32:
            src = (src * 1e-3).to(torch.float32)
    iota = torch.arange(n, dtype=torch.int32, device="cuda").repeat(count)
    keys, vals = src.clone(), iota.clone()
    items = [(keys[i * n:(i + 1) * n], vals[i * n:(i + 1) * n], i) for i in range(count)]
    times = []
    for r in range(reps + 1):
        keys.copy_(src)
        vals.copy_(iota)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sq.sort_batch(items)
        b.record()
        b.synchronize()
        if r:
            times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def tune_radix(dtypes, reps: int = 3, log=print):
    """Per key type with 32-bit ordinals: for every radix-capable leaf class,
    the batch of its largest leaves sorted with the class on the radix base
    case and on the merge sort, on full-range keys (a root column) and on a
    20-bit key range (a bucket of a 2^28 sort); keeps radix where it is not
    slower in total.  Returns ({dtype: mask}, {dtype: {class: timings}})."""
    import torch

    import paper_2407_14801_gb300 as sq

    masks, measured = {}, {}
    for dtype in dtypes:
        if dtype == "u64":
            continue
        saved = sq.get_radix_classes(dtype)
        sq.set_cutoff(dtype, sq.max_leaf(dtype))
        mask, measured[dtype] = 0, {}
        try:
            for c in RADIX_CLASSES:
                n = class_size(c)
                t = {}
                for mode, m in (("radix", 1 << c), ("merge", 0)):
                    sq.set_radix_classes(dtype, m)
                    t[mode] = sum(time_leaves(sq, torch, dtype, n, bits, reps) for bits in (32, 20))
                if choose_radix(t["radix"], t["merge"]):
                    mask |= 1 << c
                measured[dtype][str(c)] = {k: round(v, 4) for k, v in t.items()}
                log(f"{dtype} class {c} ({n} keys): radix {t['radix']:.3f} ms, merge {t['merge']:.3f} ms")
        finally:
            sq.set_cutoff(dtype, 0)
            sq.set_radix_classes(dtype, saved)
        masks[dtype] = mask
    return masks, measured


def tune(dtypes, lgs, reps: int = 3, candidates=CANDIDATES, log=print) -> dict:
    import torch

    import paper_2407_14801_gb300 as sq

    gen = torch.Generator(device="cuda")
    table, measured = {}, {}
    masks, radix_ms = tune_radix(dtypes, reps, log)  # the cutoffs are timed with the chosen leaf kernels
    for dt, m in masks.items():
        sq.set_radix_classes(dt, m)
    for dtype in dtypes:
        table[dtype], measured[dtype] = {}, {}
        limit = sq.max_n(dtype)
        for lg in lgs:
            n = 1 << lg
            if n > limit:
                continue
            gen.manual_seed(1000 * lg + len(dtype))
            src = _device_keys(torch, dtype, n, gen)
            vals0 = torch.arange(n, dtype=torch.int32, device="cuda")
            ms = {}
            for c in candidates:
                if c > sq.max_leaf(dtype):
                    continue
                # a reps-scaled budget: tiny sizes get more repetitions
                r = max(reps, min(50, (1 << 22) // n))
                ms[c] = time_cutoff(sq, torch, src, vals0, dtype, c, r)
            best = choose(ms)
            table[dtype][str(lg)] = best
            measured[dtype][str(lg)] = {str(c): round(t, 4) for c, t in ms.items()}
            log(f"{dtype} 2^{lg}: " + " ".join(f"{c}:{t:.3f}ms" for c, t in ms.items()) + f" -> {best}")
            del src, vals0
            torch.cuda.empty_cache()
        table[dtype] = fill(table[dtype])
    return {"device": torch.cuda.get_device_name(), "candidates": list(candidates), "reps": reps, "tie": TIE,
            "cutoff_by_log2n": table, "median_ms": measured, "radix_classes": masks,
            "radix_ms_by_class": radix_ms, "written": time.strftime("%Y-%m-%d %H:%M:%S")}


SWEEP_CUTOFFS = (64, 256, 1024, 4096, 16384, 65536)
SWEEP_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cutoff_sweep.json")


def normalised_ns(ms: float, n: int) -> float:
    """Nanoseconds per element per log2 n: the paper's t / (n log n)."""
    import math

    return ms * 1e6 / (n * max(1.0, math.log2(n)))


def sweep(dtypes, lgs, cutoffs=SWEEP_CUTOFFS, reps: int = 3, log=print) -> dict:
    """Times sq_sort_ex for every (dtype, n = 2^lg, cutoff) on uniform keys.
    Per point: median ms, normalised ns, and the sort's recursion rounds and
    recursing nodes (from the library's counters on one more, untimed run)."""
    import torch

    import paper_2407_14801_gb300 as sq

    gen = torch.Generator(device="cuda")
    out = {}
    for dtype in dtypes:
        out[dtype] = {}
        for lg in lgs:
            n = 1 << lg
            if n > sq.max_n(dtype):
                continue
            gen.manual_seed(7000 + lg)
            src = _device_keys(torch, dtype, n, gen)
            vals0 = torch.arange(n, dtype=torch.int32, device="cuda")
            row = {}
            for c in cutoffs:
                if c > sq.max_leaf(dtype):
                    continue
                r = max(reps, min(50, (1 << 22) // n))
                ms = time_cutoff(sq, torch, src, vals0, dtype, c, r)
                keys, vals = src.clone(), vals0.clone()
                sq.reset_stats()
                sq.sort(keys, vals, seed=1, dtype=dtype, cutoff=c)
                torch.cuda.synchronize()
                st = sq.stats()
                row[str(c)] = {"ms": round(ms, 4), "ns_per_n_log2n": round(normalised_ns(ms, n), 5),
                               "rounds": st["rounds"], "nodes": st["nodes"]}
                del keys, vals
            out[dtype][str(lg)] = row
            log(f"{dtype} 2^{lg}: " + " ".join(f"c{c}:{v['ns_per_n_log2n']:.4f}ns/{v['rounds']}r"
                                              for c, v in row.items()))
            del src, vals0
            torch.cuda.empty_cache()
    return {"device": torch.cuda.get_device_name(), "cutoffs": list(cutoffs), "reps": reps, "keys": "uniform",
            "points": out, "written": time.strftime("%Y-%m-%d %H:%M:%S")}


def report(doc: dict) -> str:
    """Markdown tables of a sweep: per key type, one row per n, one column
    per cutoff, each cell 'normalised ns (recursion rounds)'."""
    lines = []
    cut = [str(c) for c in doc["cutoffs"]]
    for dtype, pts in doc["points"].items():
        lines.append(f"**{dtype}** (ns per element per log2 n; recursion rounds in parentheses)\n")
        lines.append("| n | " + " | ".join(f"cutoff {c}" for c in cut) + " |")
        lines.append("|---|" + "---:|" * len(cut))
        for lg in sorted(pts, key=int):
            cells = []
            for c in cut:
                v = pts[lg].get(c)
                cells.append(f"{v['ns_per_n_log2n']:.4f} ({v['rounds']})" if v else "-")
            lines.append(f"| 2^{lg} | " + " | ".join(cells) + " |")
        lines.append("")
    return "\n".join(lines)


def level_steps(doc: dict, dtype: str, cutoff) -> list:
    """The sizes at which a sort with this cutoff took more recursion rounds
    than at the next smaller measured size (an extra level appeared)."""
    pts = doc["points"][dtype]
    out, prev = [], None
    for lg in sorted(pts, key=int):
        v = pts[lg].get(str(cutoff))
        if v is None:
            continue
        if prev is not None and v["rounds"] > prev:
            out.append(int(lg))
        prev = v["rounds"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--lg", default="16:28", help="log2 n range lo:hi (inclusive)")
    ap.add_argument("--dtypes", default="u32,u64,f32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None, help="output path (default: tuning.json in the package)")
    ap.add_argument("--dry-run", action="store_true", help="print the table, write nothing")
    ap.add_argument("--from", dest="src", default=None,
                    help="re-derive the table from the timings of an earlier tuning file (no GPU)")
    ap.add_argument("--sweep", action="store_true", help="the cutoff experiment instead of the tuning table")
    ap.add_argument("--cutoffs", default=",".join(str(c) for c in SWEEP_CUTOFFS))
    ap.add_argument("--report", default=None, help="print a sweep file as tables (no GPU)")
    a = ap.parse_args(argv)
    if a.report:
        with open(a.report) as f:
            doc = json.load(f)
        print(report(doc))
        for dt in doc["points"]:
            for c in doc["cutoffs"]:
                print(f"{dt} cutoff {c}: extra rounds from n = " + ", ".join(f"2^{g}" for g in level_steps(doc, dt, c)))
        return doc
    if a.sweep:
        parts = [int(x) for x in a.lg.split(":")] if a.lg != "16:28" else [10, 28, 2]
        lo, hi = parts[0], parts[1]
        stride = parts[2] if len(parts) > 2 else 1
        os.environ["SQ_NO_TUNING"] = "1"
        doc = sweep(a.dtypes.split(","), range(lo, hi + 1, stride), [int(c) for c in a.cutoffs.split(",")], a.reps)
        if not a.dry_run:
            path = a.out or SWEEP_PATH
            with open(path, "w") as f:
                json.dump(doc, f, indent=1)
            print(f"wrote {path}")
        print(report(doc))
        return doc
    if a.src:
        with open(a.src) as f:
            doc = json.load(f)
        doc["cutoff_by_log2n"] = retable(doc["median_ms"])
        doc["tie"] = TIE
        path = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
        if not a.dry_run:
            with open(path, "w") as f:
                json.dump(doc, f, indent=1)
            print(f"wrote {path}")
        return doc
    lo, hi = (int(x) for x in a.lg.split(":"))
    os.environ["SQ_NO_TUNING"] = "1"  # time the candidates themselves, not a previous table
    import paper_2407_14801_gb300 as sq

    doc = tune(a.dtypes.split(","), range(lo, hi + 1), a.reps)
    if not a.dry_run:
        path = a.out or sq.TUNING_PATH
        with open(path, "w") as f:
            json.dump(doc, f, indent=1)
        print(f"wrote {path}")
    return doc


if __name__ == "__main__":
    main()
