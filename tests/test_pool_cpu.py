"""Host logic of the serving pool (sq_pool.h): a best-fit range allocator.
Compiled into a small C++ driver with g++ and exercised against a Python model
of the free space: no overlaps, exact accounting, full coalescing."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2407_14801_gb300", "csrc", "sq_pool.h")

DRIVER = r'''
#include <cstdio>
#include "sq_pool.h"
// stdin: "C cap" | "A bytes" | "F off" ; stdout: one line per op
int main() {
  sq::RangePool p;
  setvbuf(stdout, nullptr, _IOLBF, 0);  // one answer per line, unbuffered for the pipe
  char op; unsigned long long x;
  while (scanf(" %c %llu", &op, &x) == 2) {
    if (op == 'C') { p.reset(x); printf("ok %llu\n", (unsigned long long)p.capacity()); }
    else if (op == 'A') { uint64_t off; bool ok = p.alloc(x, &off);
      printf("%s %llu %llu %llu %zu\n", ok ? "a" : "n", (unsigned long long)off,
             (unsigned long long)p.used(), (unsigned long long)p.largest_free(), p.free_ranges()); }
    else if (op == 'F') { bool ok = p.release(x);
      printf("%s %llu %llu %zu\n", ok ? "f" : "x", (unsigned long long)p.used(),
             (unsigned long long)p.largest_free(), p.free_ranges()); }
  }
}
'''


@pytest.fixture(scope="module")
def driver():
    d = tempfile.mkdtemp(prefix="sqpool_")
    src = os.path.join(d, "drv.cc")
    open(src, "w").write(DRIVER)
    exe = os.path.join(d, "drv")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.dirname(HDR), src, "-o", exe], check=True)
    return exe


def run(exe, ops):
    out = subprocess.run([exe], input="\n".join(ops) + "\n", capture_output=True, text=True, check=True).stdout
    return out.strip().splitlines()


def rnd(b):
    return (b + 255) // 256 * 256


def test_random_alloc_free_against_model(driver):
    """3000 random allocations and releases through one driver process:
    every live range stays inside the capacity and disjoint from the others,
    and the driver's byte accounting matches the model's."""
    rng = np.random.default_rng(0)
    cap = 1 << 20
    proc = subprocess.Popen([driver], stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True, bufsize=1)

    def ask(line):
        proc.stdin.write(line + "\n")
        proc.stdin.flush()
        return proc.stdout.readline().split()

    try:
        assert ask(f"C {cap}") == ["ok", str(cap)]
        live, used = {}, 0
        for _ in range(3000):
            if live and rng.random() < 0.45:
                off = sorted(live)[int(rng.integers(len(live)))]
                r = ask(f"F {off}")
                assert r[0] == "f"
                used -= live.pop(off)
                assert int(r[1]) == used
            else:
                b = int(rng.integers(1, 40000))
                r = ask(f"A {b}")
                if r[0] == "n":  # refused: no free range is large enough
                    assert int(r[3]) < rnd(b)
                    continue
                off, size = int(r[1]), rnd(b)
                assert off % 256 == 0 and off + size <= cap
                for o, s in live.items():
                    assert off + size <= o or o + s <= off
                live[off] = size
                used += size
                assert int(r[2]) == used
        for off in list(live):  # releasing everything leaves one free range
            r = ask(f"F {off}")
            used -= live.pop(off)
        assert int(r[1]) == 0 and int(r[2]) == cap and int(r[3]) == 1
    finally:
        proc.stdin.close()
        proc.wait()


def test_full_coalescing_and_errors(driver):
    cap = 1 << 16
    seq = [f"C {cap}"] + ["A 1000"] * 8
    res = run(driver, seq)
    offs = [int(l.split()[1]) for l in res[1:]]
    assert len(set(offs)) == 8
    frees = [f"F {o}" for o in offs[1::2]] + [f"F {o}" for o in offs[0::2]]
    res = run(driver, seq + frees + ["F 12345", f"A {cap}", f"A {cap}"])
    last_free = res[len(seq) + len(frees) - 1].split()
    assert last_free[0] == "f" and int(last_free[1]) == 0 and int(last_free[2]) == cap and int(last_free[3]) == 1
    assert res[-3].split()[0] == "x"          # unknown offset
    assert res[-2].split()[0] == "a"          # whole capacity again
    assert res[-1].split()[0] == "n"          # nothing left
