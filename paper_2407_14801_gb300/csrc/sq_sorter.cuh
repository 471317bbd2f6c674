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

#include <type_traits>

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

#ifndef SQ_MERGE_LOOKAHEAD
#define SQ_MERGE_LOOKAHEAD 0  // elements of each run held ahead of its head (shared memory)
#endif
#ifndef SQ_CLUSTER_LOOKAHEAD
#define SQ_CLUSTER_LOOKAHEAD 0  // the same for runs read from other CTAs' shared memory
#endif
constexpr int kLookahead = SQ_MERGE_LOOKAHEAD;
constexpr int kClusterLookahead = SQ_CLUSTER_LOOKAHEAD;

// One thread's part of a merge round: R outputs of the merge of runs A and
// B (wa and wb elements) starting at A[ai], B[bi] (its merge-path split).
// Besides its head, each run keeps the next D elements in registers, so the
// load issued when a run advances is needed only D steps later and the
// merge's compare-select chain does not wait on load latency.  get(run, i)
// reads element i of run 0 (A) or 1 (B).
template <class K, int R, int D, class Get>
__device__ __forceinline__ void serial_merge(typename K::elem_t (&x)[R], int ai, int bi, int wa, int wb, Get get) {
  typedef typename K::elem_t E;
  E a[D + 1], b[D + 1];
#pragma unroll
  for (int j = 0; j <= D; j++) {
    a[j] = ai + j < wa ? get(0, ai + j) : K::top();
    b[j] = bi + j < wb ? get(1, bi + j) : K::top();
  }
#pragma unroll
  for (int k = 0; k < R; k++) {
    // An exhausted run's head is top().  Where top() is bit-identical to any
    // element equal to it, taking it in place of such an element outputs the
    // same bits, and everything after it is top() as well: no bound checks.
    const bool tb = K::top_is_value ? K::lt(b[0], a[0]) : (bi < wb) && (ai >= wa || K::lt(b[0], a[0]));
    x[k] = tb ? b[0] : a[0];
    if (k + 1 < R) {
      E nv = K::top();
      if (k + D + 1 < R) {  // a value loaded now is used D+1 steps later at the earliest
        const int ni = (tb ? bi : ai) + D + 1;
        const bool in = ni < (tb ? wb : wa);
        nv = get(tb ? 1 : 0, in ? ni : 0);
        nv = in ? nv : K::top();
      }
#pragma unroll
      for (int j = 0; j < D; j++) {
        a[j] = tb ? a[j] : a[j + 1];
        b[j] = tb ? b[j + 1] : b[j];
      }
      a[D] = tb ? a[D] : nv;
      b[D] = tb ? nv : b[D];
      ai += tb ? 0 : 1;
      bi += tb ? 1 : 0;
    }
  }
}

// T threads (T == 32 and WARP: one warp of a larger CTA), R elements each.
template <class K_, int T, int R_, bool WARP>
struct Sorter {
  typedef K_ K;
  static constexpr int R = R_;
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
      serial_merge<K, R, kLookahead>(x, lo, diag - lo, w, w,
                                     [&](int run, int i) { return s[px((run ? bb : base) + i)]; });
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
    load(x, s, tid, keys, vals, n, [](typename K::key_t, u32) {});
  }
  // The same, calling obs(key, val) for every element loaded.
  template <class Obs>
  __device__ static void load(E (&x)[R], E *s, int tid, const typename K::key_t *keys, const u32 *vals, u32 n,
                              Obs obs) {
    if constexpr (K::async_load) {
      // asynchronous copies put the key's and the val's bytes straight into
      // the element's slot in shared memory, every copy of the thread in
      // flight at once and no register held for them; then each thread
      // completes its own slots (K::raw) and observes them
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int p = k * T + tid;
        E *slot = s + px(p);
        if ((u32)p < n) {
          const unsigned sa = (unsigned)__cvta_generic_to_shared(slot);
          if constexpr (sizeof(typename K::key_t) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa + K::key_off), "l"(keys + p) : "memory");
          else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + K::key_off), "l"(keys + p) : "memory");
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa + K::val_off), "l"(vals + p) : "memory");
        } else {
          *slot = K::top();
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      sync();
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int p = tid * R + k;
        E e = s[px(p)];
        if ((u32)p < n) {
          obs(*reinterpret_cast<const typename K::key_t *>(reinterpret_cast<const char *>(&e) + K::key_off),
              *reinterpret_cast<const u32 *>(reinterpret_cast<const char *>(&e) + K::val_off));
          e = K::raw(e);
          s[px(p)] = e;
        }
        x[k] = e;
      }
      sync();
      return;
    }
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int p = k * T + tid;
      if ((u32)p < n) {
        const typename K::key_t kk = keys[p];
        const u32 vv = vals[p];
        obs(kk, vv);
        s[px(p)] = K::make(kk, vv);
      } else {
        s[px(p)] = K::top();
      }
    }
    sync();
#pragma unroll
    for (int k = 0; k < R; k++) x[k] = s[px(tid * R + k)];
    sync();
  }

  // Stores the first n sorted elements (coalesced, through shared memory).
  __device__ static void store(E (&x)[R], E *s, int tid, typename K::key_t *keys, u32 *vals, u32 n) {
    store_mapped(x, s, tid, keys, vals, n, [](int i) { return i; });
  }

  // The same, position i of x's blocked order going to position to(i).
  template <class Map>
  __device__ static void store_mapped(E (&x)[R], E *s, int tid, typename K::key_t *keys, u32 *vals, u32 n, Map to) {
#pragma unroll
    for (int k = 0; k < R; k++) {
      const int i = tid * R + k;
      s[px((u32)i < n ? to(i) : i)] = x[k];
    }
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

  // Presorted input (what an insertion-sort base case finds cheaply): x
  // holds positions [tid*R, tid*R + R) as loaded, s all N.  Counts the
  // descents x[i] > x[i+1] among the first n; returns 1 if there are none
  // (sorted), 2 if every step descends (reversed), 3 if there is exactly
  // one, at p - 1, and x[n-1] <= x[0] (two sorted runs in swapped order),
  // 4 if there are few (at most kFewRuns) or almost n (at least n - n/8):
  // worth the runs test below; else 0.  w: kPreWords of shared memory (one
  // pair per warp; free again once any later barrier of the group has
  // passed).
  static constexpr int kPreWords = WARP ? 1 : 2 * (T / 32);
  static constexpr u32 kFewRuns = 32;
  static_assert(R <= 64, "a thread's descents fit one mask word");
  // A thread's descents as a bit mask (bit k: a descent after its element k).
  typedef typename std::conditional<(R < 32), u32, u64>::type mask_t;
  static constexpr u32 kMaskBits = 8 * sizeof(mask_t);
  __device__ __forceinline__ static u32 mclz(mask_t m) {
    if constexpr (sizeof(mask_t) == 8) return (u32)__clzll((long long)m); else return (u32)__clz((int)m);
  }
  __device__ __forceinline__ static u32 mffs(mask_t m) {
    if constexpr (sizeof(mask_t) == 8) return (u32)__ffsll((long long)m); else return (u32)__ffs((int)m);
  }
  __device__ __forceinline__ static mask_t below(int k) { return (mask_t(1) << k) - mask_t(1); }  // bits [0, k)
  __device__ __forceinline__ static int classify(u32 n, u32 d, bool wrap) {
    if (n < 2 || d == 0) return 1;
    if (d == n - 1) return 2;
    if (d == 1 && wrap) return 3;
    if (d <= kFewRuns || d >= n - n / 8) return 4;
    return 0;
  }
  __device__ static void descents(const E (&x)[R], const E *s, int tid, u32 n, u32 &d, u32 &first) {
    d = 0;
    first = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < R; k++) {  // x holds positions tid*R + k; the next thread's first is in s
      const u32 i = (u32)(tid * R + k);
      if (i + 1 < n) {
        const E nx = k + 1 < R ? x[k + 1] : s[px(tid * R + R)];
        if (K::lt(nx, x[k])) {
          first = d ? first : i;
          ++d;
        }
      }
    }
    d = __reduce_add_sync(0xffffffffu, d);
    first = __reduce_min_sync(0xffffffffu, first);
  }
  __device__ static int presorted(E (&x)[R], E *s, int tid, u32 n, u32 *w, u32 &p) {
    u32 d, first;
    descents(x, s, tid, n, d, first);
    return presorted_tail(s, tid, n, w, p, d, first);
  }
  // The same, the thread's elements read from s (x need not be live).
  __device__ static int presorted_s(const E *s, int tid, u32 n, u32 *w, u32 &p) {
    const mask_t m = desc_mask(s, tid, n);
    u32 d = (u32)__popcll((unsigned long long)m);
    u32 first = m ? (u32)(tid * R) + mffs(m) - 1u : 0xffffffffu;
    d = __reduce_add_sync(0xffffffffu, d);
    first = __reduce_min_sync(0xffffffffu, first);
    return presorted_tail(s, tid, n, w, p, d, first);
  }
  // d, first: the warp's descents and first descent.
  __device__ static int presorted_tail(const E *s, int tid, u32 n, u32 *w, u32 &p, u32 d, u32 first) {
    // (s is read only before the barrier: once past it, other threads may
    // already be writing the sorted or moved leaf into s)
    const bool wrap = n >= 2 && !K::lt(s[px(0)], s[px((int)n - 1)]);
    if (!WARP) {
      if ((tid & 31) == 0) {
        w[2 * (tid >> 5)] = d;
        w[2 * (tid >> 5) + 1] = first;
      }
      __syncthreads();
      const int l = tid & 31;  // lane l adds warp l's pair
      d = __reduce_add_sync(0xffffffffu, l < T / 32 ? w[2 * l] : 0u);
      first = __reduce_min_sync(0xffffffffu, l < T / 32 ? w[2 * l + 1] : 0xffffffffu);
    }
    p = first + 1;
    return classify(n, d, wrap);
  }

  // Runs.  A leaf's ascending runs are the stretches between its descents.
  // When each run lies entirely below the run before it (a reversed input
  // with ties, a few sorted runs swapped), the leaf is sorted by putting the
  // runs in reverse order: the run [b, e) holding element i sends it to
  // n - e + (i - b).  A thread describes its runs by the mask of its
  // descents (bit k: one at base + k) and the bounds of the runs that cross
  // its ends (pre: the start of the run holding its first element; suf: the
  // end of the run holding its last).
  // (The runs test reads the loaded leaf from s only, so that x is free
  // meanwhile.)
  __device__ static mask_t desc_mask(const E *s, int tid, u32 n) {
    mask_t m = 0;
    E cur = s[px(tid * R)];
#pragma unroll
    for (int k = 0; k < R; k++) {
      const u32 i = (u32)(tid * R + k);
      if (i + 1 < n) {
        const E nx = s[px(tid * R + k + 1)];
        if (K::lt(nx, cur)) m |= mask_t(1) << k;
        cur = nx;
      }
    }
    return m;
  }
  // b and e of the element at base + k
  __device__ __forceinline__ static u32 run_b(mask_t m, int k, u32 base, u32 pre) {
    const mask_t lb = m & below(k);  // the descents before it
    return lb ? base + kMaskBits - mclz(lb) : pre;
  }
  __device__ __forceinline__ static u32 run_e(mask_t m, int k, u32 base, u32 suf) {
    const mask_t hb = m & ~below(k);  // the descents at or after it (k <= R < kMaskBits)
    return hb ? base + mffs(hb) : suf;
  }
  // pre and suf for every thread of the group from the masks: the largest
  // run start of the earlier threads (lo if none) and the smallest run end
  // of the later ones (hi if none); tmax and tmin: the group's own largest
  // run start and smallest run end.  w: kRunWords of shared memory.
  static constexpr int kRunWords = WARP ? 1 : 2 * (T / 32);
  __device__ static void run_scan(mask_t m, u32 base, int tid, u32 lo, u32 hi, u32 *w, u32 &pre, u32 &suf, u32 &tmax,
                                  u32 &tmin) {
    const int lane = tid & 31;
    u32 a = m ? base + kMaskBits - mclz(m) : lo;  // the start of the thread's last run
    u32 z = m ? base + mffs(m) : hi;              // the end of its first run
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 ta = __shfl_up_sync(0xffffffffu, a, o);
      const u32 tz = __shfl_down_sync(0xffffffffu, z, o);
      if (lane >= o) a = max(a, ta);
      if (lane + o < 32) z = min(z, tz);
    }
    pre = __shfl_up_sync(0xffffffffu, a, 1);
    suf = __shfl_down_sync(0xffffffffu, z, 1);
    if (lane == 0) pre = lo;
    if (lane == 31) suf = hi;
    tmax = __shfl_sync(0xffffffffu, a, 31);
    tmin = __shfl_sync(0xffffffffu, z, 0);
    if (!WARP) {
      const int wid = tid >> 5;
      if (lane == 0) {
        w[wid] = tmax;
        w[T / 32 + wid] = tmin;
      }
      __syncthreads();
      tmax = lo;
      tmin = hi;
#pragma unroll
      for (int j = 0; j < T / 32; j++) {
        const u32 wa = w[j], wz = w[T / 32 + j];
        if (j < wid) pre = max(pre, wa);
        if (j > wid) suf = min(suf, wz);
        tmax = max(tmax, wa);
        tmin = min(tmin, wz);
      }
    }
  }
  // This thread's share of the test that the runs in reverse order are
  // sorted: at each of its descents d, the run after it, [d+1, e), must end
  // no higher than the run before it, [b, d+1), starts (x[e-1] <= x[b]).
  // at(p): the element at leaf position p.
  template <class At>
  __device__ static bool runs_descend(mask_t m, u32 base, u32 pre, u32 suf, At at) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < R; k++)
      if (m >> k & mask_t(1)) {
        const u32 b = run_b(m, k, base, pre), e = run_e(m, k + 1, base, suf);
        if (K::lt(at(b), at(e - 1))) ok = false;
      }
    return ok;
  }
  // A thread's runs, kept for the move.
  struct RunInfo {
    mask_t m;
    u32 pre, suf;
  };
  // The runs test for a group holding the whole leaf; ri[tid] gets this
  // thread's runs (read by the others after the test's closing barrier).
  __device__ static bool runs(const E *s, int tid, u32 n, u32 *w, RunInfo *ri) {
    const mask_t m = desc_mask(s, tid, n);
    const u32 base = (u32)(tid * R);
    u32 pre, suf, tmax, tmin;
    run_scan(m, base, tid, 0u, n, w, pre, suf, tmax, tmin);
    ri[tid] = RunInfo{m, pre, suf};
    const bool ok = runs_descend(m, base, pre, suf, [&](u32 p) { return s[px((int)p)]; });
    return WARP ? __all_sync(0xffffffffu, ok) : __syncthreads_and(ok);
  }
  // Where the element at output position o comes from when the runs are
  // put in reverse order: the input run [b, e) fills the outputs
  // [n - e, n - b), so with j = n - 1 - o (which lies in that run)
  // the source is b + e - 1 - j.  r: the runs of the thread holding j,
  // kj: j's index within that thread.
  __device__ __forceinline__ static u32 run_source(u32 j, const RunInfo &r, int kj) {
    const u32 base = j - (u32)kj;
    return run_b(r.m, kj, base, r.pre) + run_e(r.m, kj, base, r.suf) - 1u - j;
  }
};

// A leaf of up to G*T*R elements sorted by a cluster of G CTAs (any G up
// to 8): each CTA sorts its T*R elements with Sorter, then ceil(log2 G)
// merge rounds run across the cluster on runs held in the CTAs' shared
// memories (distributed shared memory).  Outputs go through registers
// between rounds, as in the in-CTA rounds.
template <class K, int T, int R, int G>
struct ClusterSorter {
  typedef Sorter<K, T, R, false> S;
  typedef typename K::elem_t E;
  static constexpr int NC = T * R;  // elements per CTA
  static constexpr int N = NC * G;

  // Sorter::presorted over the whole leaf of n elements held by the
  // cluster (this CTA's part as loaded in s).  Each CTA counts the descents
  // inside its part and publishes them with its first and last element in
  // w; after one cluster barrier every CTA adds the descents between parts
  // and returns the same answer.  w is read by the other CTAs until the
  // cluster's next barrier.
  struct PreW {
    E head, tail;
    u32 wd[S::kPreWords];
    u32 d, first;
    u32 wr[S::kRunWords];  // the runs test (written after the count has been read everywhere)
    u32 rmax, rmin, rok;
    typename S::RunInfo ri[T];
  };
  __device__ static int presorted(E (&x)[R], E *s, int tid, u32 n, PreW *w, u32 &p) {
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    const u32 q0 = (u32)rank * NC;
    const u32 nr = n > q0 ? min((u32)NC, n - q0) : 0u;
    u32 d, first;
    S::descents(x, s, tid, nr, d, first);
    return presorted_tail(s, tid, n, w, p, d, first);
  }
  // The same, the thread's elements read from s (x need not be live).
  __device__ static int presorted_s(const E *s, int tid, u32 n, PreW *w, u32 &p) {
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    const u32 q0 = (u32)rank * NC;
    const u32 nr = n > q0 ? min((u32)NC, n - q0) : 0u;
    const typename S::mask_t m = S::desc_mask(s, tid, nr);
    u32 d = (u32)__popcll((unsigned long long)m);
    u32 first = m ? (u32)(tid * R) + S::mffs(m) - 1u : 0xffffffffu;
    d = __reduce_add_sync(0xffffffffu, d);
    first = __reduce_min_sync(0xffffffffu, first);
    return presorted_tail(s, tid, n, w, p, d, first);
  }
  // d, first: the warp's descents and first descent within this CTA's part.
  __device__ static int presorted_tail(const E *s, int tid, u32 n, PreW *w, u32 &p, u32 d, u32 first) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const u32 q0 = (u32)rank * NC;
    const u32 nr = n > q0 ? min((u32)NC, n - q0) : 0u;
    if ((tid & 31) == 0) {
      w->wd[2 * (tid >> 5)] = d;
      w->wd[2 * (tid >> 5) + 1] = first;
    }
    __syncthreads();
    if (tid < 32) {  // lane l adds warp l's pair
      d = __reduce_add_sync(0xffffffffu, tid < T / 32 ? w->wd[2 * tid] : 0u);
      first = __reduce_min_sync(0xffffffffu, tid < T / 32 ? w->wd[2 * tid + 1] : 0xffffffffu);
    }
    if (tid == 0) {
      w->d = d;
      w->first = first == 0xffffffffu ? first : q0 + first;
      if (nr) {
        w->head = s[S::px(0)];
        w->tail = s[S::px((int)nr - 1)];
      }
    }
    cl.sync();
    u32 tot = 0, fst = 0xffffffffu;
    E head = E(), tail = E();
    for (int r = 0; r < G && (u32)r * NC < n; r++) {
      const PreW *pw = cl.map_shared_rank(w, r);
      const E h = pw->head;
      tot += pw->d;
      fst = min(fst, pw->first);
      if (r == 0)
        head = h;
      else if (K::lt(h, tail)) {  // the descent between part r-1 and part r
        ++tot;
        fst = min(fst, (u32)r * NC - 1);
      }
      tail = pw->tail;
    }
    p = fst + 1;
    return S::classify(n, tot, !K::lt(head, tail));
  }

  // Sorter::runs over the whole leaf held by the cluster, after presorted
  // (whose w it extends, w->ri included); every CTA returns the same answer.
  __device__ static bool runs(const E *s, int tid, u32 n, PreW *w) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const u32 q0 = (u32)rank * NC;
    const u32 nr = n > q0 ? min((u32)NC, n - q0) : 0u;
    typename S::mask_t m = S::desc_mask(s, tid, nr);
    if (tid == T - 1 && q0 + NC < n && K::lt(cl.map_shared_rank(w, rank + 1)->head, s[S::px(NC - 1)]))
      m |= typename S::mask_t(1) << (R - 1);  // the descent into the next part
    const u32 base = q0 + (u32)(tid * R);
    u32 pre, suf, tmax, tmin;
    S::run_scan(m, base, tid, 0u, n, w->wr, pre, suf, tmax, tmin);
    if (tid == 0) {
      w->rmax = tmax;
      w->rmin = tmin;
    }
    cl.sync();
    for (int r = 0; r < G && (u32)r * NC < n; r++) {
      const PreW *pw = cl.map_shared_rank(w, r);
      if (r < rank) pre = max(pre, pw->rmax);
      if (r > rank) suf = min(suf, pw->rmin);
    }
    w->ri[tid] = typename S::RunInfo{m, pre, suf};
    bool ok = S::runs_descend(m, base, pre, suf, [&](u32 p) {
      return *cl.map_shared_rank(s + S::px((int)(p % NC)), (int)(p / NC));
    });
    ok = __syncthreads_and(ok);
    if (tid == 0) w->rok = ok;
    cl.sync();  // (also: every read of a part is done before any part changes)
    for (int r = 0; r < G && (u32)r * NC < n; r++) ok = ok && cl.map_shared_rank(w, r)->rok;
    return ok;
  }

  // n: valid elements of the whole leaf (the rest top(), as left by
  // S::load).
  __device__ static void sort(E (&x)[R], E *s, int tid, int n = N) {
    S::sort(x, s, tid);
    merge_rounds(x, s, tid, n);
  }

  // The cross-CTA rounds only: x holds this CTA's sorted run, blocked.
  // In a round merging runs of w elements, this CTA produces outputs
  // [rank*NC, rank*NC + NC) of its pair of runs A, B.  Two warps find the
  // merge-path splits of that window's ends by 32-way searches over the
  // other CTAs' shared memory; every thread then copies window elements
  // (coalesced distributed-shared-memory loads, no dependent chains) into
  // registers; after a cluster barrier the window goes to this CTA's own
  // shared memory (the A part, then the B part) and is merged locally like
  // an in-CTA round.
  // A CTA whose outputs all lie at positions >= n (top() only) keeps its
  // shared memory (top() since load) and only takes part in the barriers.
  __device__ static void merge_rounds(E (&x)[R], E *s, int tid, int n = N) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ int split[2];
    const int rank = (int)cl.block_rank();
    const int lane = tid & 31, warp = tid >> 5;
    const bool idle = rank * NC >= n;
    auto at = [&](int gi) -> E { return *cl.map_shared_rank(s + S::px(gi % NC), gi / NC); };
#pragma unroll 1
    for (int w = NC; w < N; w <<= 1) {
      const int p0 = rank * NC;
      const int base = p0 & ~(2 * w - 1);
      const int bb = base + w;
      // runs of this round's pair: A = [base, base + wa), B = [bb, bb + wb)
      // (with G not a power of two the last pair may be short or single)
      const int wa = min(w, N - base), wb = max(0, min(w, N - bb));
      if (idle || wb == 0) {  // nothing to merge: the same barriers as the others
        cl.sync();
        __syncthreads();
        cl.sync();
        __syncthreads();
        __syncthreads();
        continue;
      }
#pragma unroll
      for (int k = 0; k < R; k++) s[S::px(tid * R + k)] = x[k];
      cl.sync();
      if (warp < 2) {
        // smallest i in [lo, hi] with B[d-1-i] < A[i] (hi if none): i elements
        // of the first d outputs come from A
        const int d = p0 - base + warp * NC;
        int lo = d > wb ? d - wb : 0, hi = d < wa ? d : wa;
        while (hi - lo > 32) {
          const int step = (hi - lo + 31) / 32;
          const int q = lo + lane * step;
          const bool p = q < hi && K::lt(at(bb + d - 1 - q), at(base + q));
          const unsigned m = __ballot_sync(0xffffffffu, p);
          const int last = min(31, (hi - 1 - lo) / step);  // last probe inside [lo, hi)
          const int f = m ? __ffs(m) - 1 : 32;
          const int nlo = f == 0 ? lo : lo + (min(f, last + 1) - 1) * step + 1;
          const int nhi = f == 32 ? hi : lo + f * step;
          lo = nlo;
          hi = nhi;
        }
        const int q = lo + lane;
        const bool p = q < hi && K::lt(at(bb + d - 1 - q), at(base + q));
        const unsigned m = __ballot_sync(0xffffffffu, p);
        if (lane == 0) split[warp] = m ? lo + __ffs(m) - 1 : hi;
      }
      __syncthreads();
      const int d0 = p0 - base;
      const int a0 = split[0], a1 = split[1];
      const int b0 = d0 - a0;
      const int la = a1 - a0;  // window: A[a0, a1) then B[b0, b0 + NC - la)
#pragma unroll
      for (int k = 0; k < R; k++) {
        const int e = k * T + tid;
        x[k] = at(e < la ? base + a0 + e : bb + b0 + (e - la));
      }
      cl.sync();  // every CTA has copied its window: shared memory may be overwritten
#pragma unroll
      for (int k = 0; k < R; k++) s[S::px(k * T + tid)] = x[k];
      __syncthreads();
      const int lb = NC - la, dd = tid * R;
      int lo = dd > lb ? dd - lb : 0, hi = dd < la ? dd : la;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (K::lt(s[S::px(la + dd - 1 - mid)], s[S::px(mid)]))
          hi = mid;
        else
          lo = mid + 1;
      }
      serial_merge<K, R, kLookahead>(x, lo, dd - lo, la, lb,
                                     [&](int run, int i) { return s[S::px((run ? la : 0) + i)]; });
      __syncthreads();  // the window is read before the next round (or the store) overwrites it
    }
  }
};

}  // namespace sq
