"""GPU parity of sorts whose root has more pivots than one CTA sorts
(uint32 keys, n above (16384 + 1)^2): the pivot sample sorted by a cluster
of 8 CTAs, the bucket count reading its pivots from global memory.

- n = 17000^2 = 289 000 000 (k - 1 = 16999 pivots) with cutoff 8192: every
  bucket of the root is a traced node, so the trace carries the root's
  pivot-sample count and every bucket size, compared with the oracle's
  node step (column sorts, pivot draws with redraws, bucket sizes) on the
  same packed (key, index) input; the output by the properties that pin the
  unique sorted result (non-decreasing (key, val), the payloads a
  permutation, every key with its payload).
- n = 2^31 from page-locked host buffers (the first pass reads them, the last
  writes them): the output by the same properties.
- n = 2^31 with every round in one CUDA-graph launch (the graph sized for
  k up to 2^16).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_ROOT = 17000 * 17000


@pytest.fixture(scope="module")
def sq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_14801_gb300 as sq

    sq.lib()
    return sq


def check_unique_result(src_bits, out_bits, out_vals):
    """src_bits, out_bits: int32 key bits; out_vals: int32 payloads (the
    original indices)."""
    n = out_bits.numel()
    o = out_bits.to(torch.int64) & 0xFFFFFFFF
    v = out_vals.to(torch.int64) & 0xFFFFFFFF
    ok = bool(((o[1:] > o[:-1]) | ((o[1:] == o[:-1]) & (v[1:] > v[:-1]))).all())
    assert ok, "not sorted by (key, val)"
    del o
    seen = torch.zeros(n, dtype=torch.bool, device=out_vals.device)
    seen[v] = True
    assert bool(seen.all()), "payloads are not a permutation"
    del seen
    assert bool((src_bits[v] == out_bits).all()), "a key left its payload"


def test_root_with_cluster_sorted_pivots_matches_oracle(sq):
    assert sq.max_n("u32") > N_ROOT
    keys_np = W.uniform_u32(N_ROOT, 6)
    src = torch.from_numpy(keys_np.view(np.int32)).cuda()
    keys = src.clone()
    vals = torch.arange(N_ROOT, dtype=torch.int32, device="cuda")
    seed = 23
    tr = sq.sort(keys, vals, seed=seed, dtype="u32", cutoff=8192, trace_cap=1 << 16)
    torch.cuda.synchronize()
    check_unique_result(src, keys, vals)
    del keys, vals, src
    torch.cuda.empty_cache()
    root = [r for r in tr if r["kind"] == 0]
    assert len(root) == 1 and root[0]["m"] == 17000 and root[0]["hash"] == oracle.root_hash(seed)
    packed = (keys_np.astype(np.uint64) << np.uint64(32)) | np.arange(N_ROOT, dtype=np.uint64)
    sizes, attempts = oracle.node_buckets(packed, oracle.root_hash(seed))
    del packed
    assert attempts > 0 and root[0]["attempts"] == attempts
    got = {r["index"]: r["n"] for r in tr if r["kind"] == 2 and r["depth"] == 1}
    want = {j: int(s) for j, s in enumerate(sizes) if s > 8192}
    assert got == want
    assert sum(int(s) for s in sizes) == N_ROOT


def test_u32_2e31_from_pinned_host_memory(sq):
    n = 1 << 31
    g = torch.Generator(device="cuda")
    g.manual_seed(31)
    src = torch.randint(-(1 << 31), 1 << 31, (n,), dtype=torch.int32, device="cuda", generator=g)
    hk = torch.empty(n, dtype=torch.int32).pin_memory()
    hv = torch.empty(n, dtype=torch.int32).pin_memory()
    hk.copy_(src)
    hv.copy_(torch.arange(n, dtype=torch.int32))
    sq.sort(hk, hv, seed=5, dtype="u32")
    out_k = hk.cuda()
    out_v = hv.cuda()
    del hk, hv
    check_unique_result(src, out_k, out_v)


def test_u32_2e31_graph_launch_mode(sq):
    n = 1 << 31
    g = torch.Generator(device="cuda")
    g.manual_seed(32)
    src = torch.randint(-(1 << 31), 1 << 31, (n,), dtype=torch.int32, device="cuda", generator=g)
    keys = src.clone()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    sq.set_launch_mode("graph")
    try:
        sq.sort(keys, vals, seed=6, dtype="u32")
        sq.sync()
    finally:
        sq.set_launch_mode("auto")
    check_unique_result(src, keys, vals)
