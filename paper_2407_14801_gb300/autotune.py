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


def tune(dtypes, lgs, reps: int = 3, candidates=CANDIDATES, log=print) -> dict:
    import torch

    import paper_2407_14801_gb300 as sq

    gen = torch.Generator(device="cuda")
    table, measured = {}, {}
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
            "cutoff_by_log2n": table, "median_ms": measured, "written": time.strftime("%Y-%m-%d %H:%M:%S")}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--lg", default="16:28", help="log2 n range lo:hi (inclusive)")
    ap.add_argument("--dtypes", default="u32,u64,f32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None, help="output path (default: tuning.json in the package)")
    ap.add_argument("--dry-run", action="store_true", help="print the table, write nothing")
    ap.add_argument("--from", dest="src", default=None,
                    help="re-derive the table from the timings of an earlier tuning file (no GPU)")
    a = ap.parse_args(argv)
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
