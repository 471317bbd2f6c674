// In-register / shared-memory merge sort of one group of threads (a warp or
// a whole CTA).  Used for SquareSort's base case (simple_sort of Algorithm 1)
// and for sorting a node's pivot sample.
//
// Each thread holds R elements.  They are first sorted in registers by a
// bitonic network, then runs of width R, 2R, ... are merged pairwise with
// merge-path partitioning: every thread finds the split of its R outputs in
// the pair of sorted runs by a binary search on its diagonal and merges them
// sequentially from shared memory.  Shared memory is padded by one slot per
// R elements so that the blocked (thread-contiguous) stores and loads hit
// distinct banks.
#pragma once
#include <cooperative_groups.h>

#include "sq_types.cuh"

namespace sq {

__device__ __forceinline__ u64 shfl_xor_e(u64 v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ E3 shfl_xor_e(E3 v, int m) {
  E3 r;
  r.k = __shfl_xor_sync(0xffffffffu, v.k, m);
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.pad = 0;
  return r;
}
__device__ __forceinline__ u64 shfl_e(u64 v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ E3 shfl_e(E3 v, int src) {
  E3 r;
  r.k = __shfl_sync(0xffffffffu, v.k, src);
  r.x = __shfl_sync(0xffffffffu, v.x, src);
  r.pad = 0;
  return r;
}

template <class K>
__device__ __forceinline__ typename K::elem_t warp_min(typename K::elem_t v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    typename K::elem_t o = shfl_xor_e(v, m);
    v = K::lt(o, v) ? o : v;
  }
  return v;
}

// T threads (T == 32 and WARP: one warp of a larger CTA), R elements each.
template <class K, int T, int R, bool WARP>
struct Sorter {
  typedef typename K::elem_t E;
  static constexpr int N = T * R;
  static constexpr int SMEM = N + N / R;  // padded element slots
  static_assert(!WARP || T == 32, "warp groups have 32 threads");

  __device__ __forceinline__ static int px(int p) { return p + p / R; }
  __device__ __forceinline__ static void sync() {
    if (WARP)
      __syncwarp();
    else
      __syncthreads();
  }

  // Bitonic sorting network on the R register-resident elements.
  __device__ __forceinline__ static void network(E (&x)[R]) {
#pragma unroll
    for (int k = 2; k <= R; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int i = 0; i < R; i++) {
          const int l = i ^ j;
          if (l > i) {
            const bool up = (i & k) == 0;
            E a = x[i], b = x[l];
            const bool sw = up ? K::lt(b, a) : K::lt(a, b);
            x[i] = sw ? b : a;
            x[l] = sw ? a : b;
          }
        }
      }
    }
  }

  // Sorts the group's N elements; on return thread tid holds sorted
  // positions [tid*R, tid*R + R).  Ends with a barrier, so s is free.
  // Merge rounds whose run pairs lie inside one warp's 32*R elements need
  // only a warp barrier.
  __device__ static void sort(E (&x)[R], E *s, int tid) {
    network(x);
#pragma unroll 1
    for (int w = R; w < N; w <<= 1) {
      const bool warp_local = WARP || 2 * w <= 32 * R;
#pragma unroll
      for (int k = 0; k < R; k++) s[px(tid * R + k)] = x[k];
      if (warp_local)
        __syncwarp();
      else
        __syncthreads();
      const int p0 = tid * R;
      const int base = p0 & ~(2 * w - 1);
      const int diag = p0 - base;
      const int bb = base + w;
      int lo = diag > w ? diag - w : 0, hi = diag < w ? diag : w;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (K::lt(s[px(bb + diag - 1 - mid)], s[px(base + mid)]))
          hi = mid;
        else
          lo = mid + 1;
      }
      int ai = lo, bi = diag - lo;
      E av = ai < w ? s[px(base + ai)] : K::top();
      E bv = bi < w ? s[px(bb + bi)] : K::top();
#pragma unroll
      for (int k = 0; k < R; k++) {
        const bool tb = (bi < w) && (ai >= w || K::lt(bv, av));
        x[k] = tb ? bv : av;
        if (k + 1 < R) {  // advance the consumed run; one unconditional load
          const int ni = (tb ? bi : ai) + 1;
          const bool in = ni < w;
          const int addr = (tb ? bb : base) + (in ? ni : 0);
          E nv = s[px(addr)];
          nv = in ? nv : K::top();
          ai = tb ? ai : ni;
          bi = tb ? ni : bi;
          av = tb ? av : nv;
          bv = tb ? nv : bv;
        }
      }
      if (warp_local)
        __syncwarp();
      else
        __syncthreads();
    }
  }

  // Loads n <= N elements (coalesced, through shared memory) into the
  // blocked register layout; positions >= n become top().
  __device__ static void load(E (&x)[R], E *s, int tid, const typename K::key_t *keys, const u32 *vals,
                              u32 n) {
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int p = k * T + tid;
      s[px(p)] = (u32)p < n ? K::make(keys[p], vals[p]) : K::top();
    }
    sync();
#pragma unroll
    for (int k = 0; k < R; k++) x[k] = s[px(tid * R + k)];
    sync();
  }

  // Stores the first n sorted elements (coalesced, through shared memory).
  __device__ static void store(E (&x)[R], E *s, int tid, typename K::key_t *keys, u32 *vals, u32 n) {
#pragma unroll
    for (int k = 0; k < R; k++) s[px(tid * R + k)] = x[k];
    sync();
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int p = k * T + tid;
      if ((u32)p < n) {
        const E e = s[px(p)];
        keys[p] = K::key(e);
        vals[p] = K::val(e);
      }
    }
    sync();
  }
};

// A leaf of up to G*T*R elements sorted by a cluster of G CTAs: each CTA
// sorts its T*R elements with Sorter, then log2(G) merge rounds run across
// the cluster, every thread reading the two runs it merges from whichever
// CTAs' shared memory holds them (distributed shared memory).  Outputs go
// through registers between rounds, as in the in-CTA rounds.
template <class K, int T, int R, int G>
struct ClusterSorter {
  typedef Sorter<K, T, R, false> S;
  typedef typename K::elem_t E;
  static constexpr int NC = T * R;  // elements per CTA
  static constexpr int N = NC * G;

  __device__ static void sort(E (&x)[R], E *s, int tid) {
    S::sort(x, s, tid);
    merge_rounds(x, s, tid);
  }

  // The cross-CTA rounds only: x holds this CTA's sorted run, blocked.
  __device__ static void merge_rounds(E (&x)[R], E *s, int tid) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    auto at = [&](int gi) -> E { return *cl.map_shared_rank(s + S::px(gi % NC), gi / NC); };
#pragma unroll 1
    for (int w = NC; w < N; w <<= 1) {
#pragma unroll
      for (int k = 0; k < R; k++) s[S::px(tid * R + k)] = x[k];
      cl.sync();
      const int p0 = rank * NC + tid * R;
      const int base = p0 & ~(2 * w - 1);
      const int diag = p0 - base;
      const int bb = base + w;
      int lo = diag > w ? diag - w : 0, hi = diag < w ? diag : w;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (K::lt(at(bb + diag - 1 - mid), at(base + mid)))
          hi = mid;
        else
          lo = mid + 1;
      }
      int ai = lo, bi = diag - lo;
      E av = ai < w ? at(base + ai) : K::top();
      E bv = bi < w ? at(bb + bi) : K::top();
#pragma unroll
      for (int k = 0; k < R; k++) {
        const bool tb = (bi < w) && (ai >= w || K::lt(bv, av));
        x[k] = tb ? bv : av;
        if (k + 1 < R) {
          const int ni = (tb ? bi : ai) + 1;
          const bool in = ni < w;
          E nv = at((tb ? bb : base) + (in ? ni : 0));
          nv = in ? nv : K::top();
          ai = tb ? ai : ni;
          bi = tb ? ni : bi;
          av = tb ? av : nv;
          bv = tb ? nv : bv;
        }
      }
      cl.sync();  // every CTA has read its runs before they are overwritten
    }
  }
};

}  // namespace sq
