// SquareSort engine kernels (Algorithm 1 of Koucky & Matejka, Section 2).
//
// The recursion is run breadth-first in rounds.  Each round:
//   k_leaf          sorts every pending leaf (n <= cutoff: Algorithm 1's
//                   simple_sort) in registers + shared memory;
//   k_plan          numbers the work of every node whose columns are sorted;
//   k_pivots        draws, sorts and checks those nodes' pivot samples;
//   k_count         one pass over each sorted column: bucket totals per block
//                   of columns and the start of every 64-bucket segment
//                   (Section 2.2: a sorted column and the sorted pivots are
//                   walked together, a merge);
//   k_scan/k_bstart prefix sums: bucket starts and per-block offsets;
//   k_skew          SkewTranspose (Algorithm 2 / 3) as a tiled stable
//                   partition staged in shared memory;
//   k_expand_*      spawn the bucket / column children (Algorithm 1's
//                   recursive calls) as leaves or new nodes.
// A leaf finishing decrements its parent's pending count; the last column
// makes the parent ready for the next round, the last bucket completes it.
#pragma once
#include "sq_radix.cuh"
#include "sq_sorter.cuh"

namespace sq {

// ------------------------------------------------------------ helpers ------

template <int DT>
struct LeafCfg;
// Leaf classes (elements per class): c0 = warp x 2 (64), c1 = warp x 16
// (512), c2 = 128 x 16 (2048), c3 = 512 x 16 (8192), and c4..c10 = clusters
// of g = 2..8 CTAs of 512 x 16 (g * 8192 elements: a leaf takes the
// smallest cluster that holds it).  All are merge sorts; the cluster rounds
// copy each CTA's merge window out of the others' shared memory.  Pivot
// samples use the single-CTA sorters only.
template <int DT>
struct LeafCfg;
// max_pivots: the largest sample one CTA sorts; max_pivots_big: the largest
// that a cluster of 8 CTAs sorts (k_pivots_cluster; uint32 keys only, whose
// sort then reaches n = 2^32 - 1), 0 for none.
template <>
struct LeafCfg<DT_U32> {
  static constexpr int nclass = kLeafClasses;
  static constexpr u32 max_pivots = 16384;
  static constexpr u32 max_pivots_big = 65535;
};
template <>
struct LeafCfg<DT_F32> {
  static constexpr int nclass = kLeafClasses;
  static constexpr u32 max_pivots = 8192;
  static constexpr u32 max_pivots_big = 0;
};
template <>
struct LeafCfg<DT_U64> {
  static constexpr int nclass = kLeafClasses;
  static constexpr u32 max_pivots = 8192;
  static constexpr u32 max_pivots_big = 0;
};
constexpr u32 kClusterPart = 8192;  // elements per CTA of the cluster classes
__host__ __device__ __forceinline__ u32 class_cap(int c) {
  return c == 0 ? 64u : c == 1 ? 512u : c == 2 ? 2048u : (u32)(c - 2) * kClusterPart;
}

__host__ __device__ __forceinline__ int class_of(u32 n, int nclass) {
  if (n <= 2048) return n <= 64 ? 0 : n <= 512 ? 1 : 2;
  const int c = 2 + (int)((n + kClusterPart - 1) / kClusterPart);
  return c < nclass ? c : nclass - 1;
}

// e lies below pivot p: e < p under Algorithm 1 (bucket j = [p_j, p_{j+1})),
// e <= p under the appendix variant (bucket i = (p_{i-1}, p_i]).
template <class K>
__device__ __forceinline__ bool below_p(const typename K::elem_t &e, const typename K::elem_t &p, bool le) {
  return le ? !K::lt(p, e) : K::lt(e, p);
}

// number of pivots in piv[lo, hi) that e is not below (its bucket, from lo)
template <class K>
__device__ __forceinline__ int upper_bound_e(const typename K::elem_t *piv, int lo, int hi,
                                             const typename K::elem_t &e, bool le = false) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (below_p<K>(e, piv[mid], le))
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// Bucket (number of pivots <= e) of an element that every lane of the warp
// holds, given that it is at least lo: the lanes first probe 32 pivots
// kSpan apart, then the kSpan pivots of the interval found; larger jumps
// fall back to a binary search.  Replaces a serial search of log2(np) steps.
// (kSpan: about the buckets a warp's group of elements spans on uniform
// input, at most 32.)
template <class K, int kSpan = 4>
__device__ __forceinline__ int warp_bucket_from(const typename K::elem_t *piv, int lo, int np,
                                                const typename K::elem_t &e, bool lep = false) {
  static_assert(kSpan >= 2 && kSpan <= 32, "probe spacing");
  const int lane = threadIdx.x & 31;
  int idx = lo + (lane + 1) * kSpan - 1;  // probes lo+3, lo+7, ...
  bool le = idx < np && !below_p<K>(e, piv[idx], lep);
  u32 m = __ballot_sync(0xffffffffu, le);
  if (m == 0xffffffffu) return upper_bound_e<K>(piv, lo + 32 * kSpan, np, e, lep);
  const int base = lo + __popc(m) * kSpan;  // e is not below any pivot before base
  idx = base + (lane < kSpan - 1 ? lane : kSpan - 1);
  le = lane < kSpan - 1 && idx < np && !below_p<K>(e, piv[idx], lep);
  m = __ballot_sync(0xffffffffu, le);
  return base + __popc(m);
}

static __device__ __forceinline__ u32 block_excl_scan_u32(u32 v, u32 *warp_tot, u32 &total) {
  // any blockDim multiple of 32, <= 1024; warp_tot: 32 words of shared memory
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  u32 inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const u32 o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    u32 t = lane < nw ? warp_tot[lane] : 0, ti = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u32 o = __shfl_up_sync(0xffffffffu, ti, d);
      if (lane >= d) ti += o;
    }
    warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  const u32 r = warp_tot[w] + inc - v;
  total = warp_tot[32];
  __syncthreads();
  return r;
}

static __device__ __forceinline__ u64 block_excl_scan_u64(u64 v, u64 *warp_tot, u64 &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  u64 inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const u64 o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    u64 t = lane < nw ? warp_tot[lane] : 0, ti = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const u64 o = __shfl_up_sync(0xffffffffu, ti, d);
      if (lane >= d) ti += o;
    }
    warp_tot[lane] = ti - t;
    if (lane == 31) warp_tot[32] = ti;
  }
  __syncthreads();
  const u64 r = warp_tot[w] + inc - v;
  total = warp_tot[32];
  __syncthreads();
  return r;
}

// Ready-list position of the node owning work item u: the last entry of the
// non-decreasing array base[0..cnt) that is <= u (base[0] = 0).  Called by a
// whole warp; each round narrows the range 32-fold.
__device__ __forceinline__ u32 warp_find(const u32 *base, u32 cnt, u32 u) {
  const int lane = threadIdx.x & 31;
  u32 lo = 0, hi = cnt;
  while (hi - lo > 1) {
    const u32 step = (hi - lo + 31) / 32;
    const u32 idx = lo + lane * step;
    const bool le = idx < hi && base[idx] <= u;
    const u32 m = __ballot_sync(0xffffffffu, le);
    const u32 last = 31 - __clz(m);
    lo = lo + last * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// Grabs the next work item of a persistent kernel (warp 0) and finds its
// node; returns the item in *u and the ready-list index in *ri (shared).
__device__ __forceinline__ void grab_item(const Ctx &c, u32 *cursor, u32 total, int which, u32 ready_count,
                                          u32 *s_u, u32 *s_ri) {
  if ((threadIdx.x >> 5) == 0) {
    u32 u = 0;
    if ((threadIdx.x & 31) == 0) u = atomicAdd(cursor, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    u32 ri = 0;
    if (u < total) ri = warp_find(c.wbase + (u64)which * c.ready_cap, ready_count, u);
    if ((threadIdx.x & 31) == 0) {
      *s_u = u;
      *s_ri = ri;
    }
  }
}

// A leaf that its leaf kernel could not sort exactly goes to this round's
// fix list, which k_fixup sorts with the (key, val) merge sort.
__device__ __forceinline__ void push_fix(const Ctx &c, Leaf L) {
  const u32 i = atomicAdd(&c.status->fix_count, 1u);
  L.flags |= LEAF_IN_OUT;
  if (i < c.fix_cap)
    c.fix[i] = L;
  else
    atomicOr(&c.status->error, ERRB_LIST);
}

// A finished unit of work (leaf or completed node) reports to its parent.
static __device__ void child_done(const Ctx &c, u32 parent, u32 kind, u32 inst) {
  for (;;) {
    if (parent == kNone) {
      const u32 d = atomicAdd(&c.status->done, 1u);
      c.done_list[d % c.ninst] = inst;  // a ring in a persistent session
      return;
    }
    Node *p = &c.nodes[parent];
    if (atomicSub(&p->pending, 1) != 1) return;
    if (kind == KIND_COL) {  // every column of p is sorted: p is ready
      const u32 r = atomicAdd(&c.cnt_nxt->ready, 1u);
      if (r < c.ready_cap)
        c.ready_nxt[r] = parent;
      else
        atomicOr(&c.status->error, ERRB_LIST);
      atomicMax(&c.cnt_nxt->max_ready_k, p->k);
      atomicAdd(&c.cnt_nxt->ready_elems, (u64)p->n);
      return;
    }
    // every bucket of p is sorted: p is complete; report to its own parent
    kind = p->kind;
    inst = p->inst;
    parent = p->parent;
  }
}

// ---------------------------------------------------------------- leaves ---

// Keys whose bits the leaf element does not keep (K::lossy: NaN float32
// keys) are listed per leaf in shared memory while the leaf is loaded: the
// count, then kNanCap vals and kNanCap keys.  After the sort they sit at the
// end of the leaf in val order (every NaN has the largest ordinal, ties go
// by val) and get their bits back.  A leaf with more such keys is copied to
// its output and left to the fix list's exact (key, val) sort.
constexpr u32 kNanCap = 64;
constexpr u32 kNanWords = 1 + 2 * kNanCap;

template <class K>
__device__ __forceinline__ void nan_note(u32 *nl, typename K::key_t k, u32 v) {
  if constexpr (K::lossy) {
    if (!K::exact(k)) {
      const u32 i = atomicAdd(&nl[0], 1u);
      if (i < kNanCap) {
        nl[1 + i] = v;
        nl[1 + kNanCap + i] = (u32)k;
      }
    }
  }
}

// Rank of list entry i among all listed keys: by val, then (list, entry).
__device__ __forceinline__ u32 nan_rank(const u32 *nl, u32 cnt, u32 v, u32 i) {
  u32 r = 0;
  for (u32 j = 0; j < cnt; j++) {
    const u32 vj = nl[1 + j];
    r += (vj < v) || (vj == v && j < i);
  }
  return r;
}

// CTAs per SM the one-CTA leaf kernels are built for (a register budget):
// with 8-byte elements about 80 registers a thread for the small classes,
// 64 for the 512-thread class.
template <int DT, int T, bool WARP>
constexpr int kLeafMinBlocks() {
  return sizeof(typename KT<DT>::elem_t) != 8 ? 1 : WARP ? 3 : T <= 128 ? 6 : T >= 512 ? 2 : 1;
}

// Shared memory of a leaf CTA's sort (before its NaN lists).
template <int DT, int T, int R, bool WARP>
__host__ __device__ constexpr size_t leaf_sort_bytes() {
  return (size_t)(WARP ? 8 : 1) * Sorter<KT<DT>, T, R, WARP>::SMEM * sizeof(typename KT<DT>::elem_t);
}

// Shared memory of a radix leaf CTA: the sort's element slots, the NaN list
// (float32 keys), then the radix counters and scratch.
template <int DT, int T, int R>
__host__ __device__ constexpr size_t radix_ws_offset() {
  return (leaf_sort_bytes<DT, T, R, false>() + (KT<DT>::lossy ? 4 * kNanWords : 0) + 15) & ~(size_t)15;
}
template <int DT, int T, int R>
__host__ __device__ constexpr size_t radix_leaf_bytes() {
  return radix_ws_offset<DT, T, R>() + RadixLeaf<KT<DT>, T, R>::kBytes;
}

// A leaf whose ascending runs descend (Sorter::runs) is moved run by run:
// every output position, in coalesced order, takes its element from the
// loaded copy in s.  Returns false (nothing written) if the runs do not
// descend.  Kept out of line: the test needs registers that the merge sort,
// the common path, must not lose.
template <class S>
__device__ __noinline__ bool leaf_runs(const typename S::E *s, int tid, u32 n, u32 *w, typename S::RunInfo *ri,
                                       typename S::K::key_t *ok, u32 *ov) {
  typedef typename S::K K;
  if (!S::runs(s, tid, n, w, ri)) return false;
  constexpr int T = S::N / S::R;
#pragma unroll 4
  for (int k = 0; k < S::R; k++) {
    const u32 o = (u32)(k * T + tid);
    if (o < n) {
      const u32 j = n - 1u - o;
      const typename S::E e = s[S::px((int)S::run_source(j, ri[j / S::R], (int)(j % S::R)))];
      ok[o] = K::key(e);
      ov[o] = K::val(e);
    }
  }
  return true;
}
// The same for a cluster's leaf (pre: 2 reversed, 3 rotated at rot, 4 runs
// to be tested), every CTA writing its part of the output from the parts in
// the cluster's shared memories.
template <class CS>
__device__ __noinline__ bool leaf_move_cluster(const typename CS::E *s, int tid, u32 n, int pre, u32 rot,
                                               typename CS::PreW *w, typename CS::S::K::key_t *ok, u32 *ov) {
  typedef typename CS::S S;
  typedef typename S::K K;
  constexpr int T = S::N / S::R, R = S::R, NC = CS::NC;
  if (pre == 4 && !CS::runs(s, tid, n, w)) return false;
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const u32 q0 = (u32)cl.block_rank() * NC;
#pragma unroll 4
  for (int k = 0; k < R; k++) {
    const u32 o = q0 + (u32)(k * T + tid);
    if (o < n) {
      u32 src;
      if (pre == 2) {
        src = n - 1u - o;
      } else if (pre == 3) {
        src = o + rot < n ? o + rot : o + rot - n;
      } else {
        const u32 j = n - 1u - o;
        const typename S::RunInfo r = cl.map_shared_rank(w, (int)(j / NC))->ri[(j % NC) / R];
        src = S::run_source(j, r, (int)(j % R));
      }
      const typename S::E e = *cl.map_shared_rank(s + S::px((int)(src % NC)), (int)(src / NC));
      ok[o] = K::key(e);
      ov[o] = K::val(e);
    }
  }
  return true;
}

template <int DT, int T, int R, bool WARP>
__global__ void __launch_bounds__(WARP ? 256 : T, kLeafMinBlocks<DT, T, WARP>()) k_leaf(const Ctx *__restrict__ cp, int cls, u32 count) {
  const Ctx &c = *cp;
  typedef KT<DT> K;
  typedef Sorter<K, T, R, WARP> S;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *smem = reinterpret_cast<E *>(smem_raw);
  constexpr int groups = WARP ? 8 : 1;
  const int g = WARP ? (threadIdx.x >> 5) : 0;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  u32 *nl = reinterpret_cast<u32 *>(smem_raw + leaf_sort_bytes<DT, T, R, WARP>()) + g * kNanWords;  // K::lossy only
  const bool dyn = count == kDev;  // a fixed-size grid: every group takes the next leaf
  const u32 cnt = dyn ? min(c.cnt_cur->leaves[cls], c.leaf_cap[cls]) : count;
  __shared__ u32 s_li[groups];
  __shared__ u32 s_pre[groups][S::kPreWords];
  __shared__ u32 s_run[groups][S::kRunWords];
  __shared__ typename S::RunInfo s_ri[groups][T];
  auto next_leaf = [&](u32 done_li) -> u32 {
    if (!dyn) return done_li == kNone ? blockIdx.x * groups + g : cnt;  // one leaf per group
    u32 li = 0;
    if (tid == 0) s_li[g] = atomicAdd(&c.status->cur_leaf[cls], 1u);
    S::sync();
    li = s_li[g];
    S::sync();
    return li;
  };
  for (u32 li = next_leaf(kNone); li < cnt; li = next_leaf(li)) {
    const Leaf L = c.leaves_cur[cls][li];
    const Inst I = c.inst[L.inst];
    E *s = smem + g * S::SMEM;
    E x[R];
    const u32 out = (L.flags >> 8) & 0xffu;
    const bool from_src = (L.flags & LEAF_SRC) != 0;
    const key_t *ik = (const key_t *)(from_src ? I.skeys : I.keys) + L.off;
    const u32 *iv = (from_src ? I.svals : I.vals) + L.off;
    key_t *ok = (key_t *)(out ? I.dkeys : I.fkeys) + L.off;
    u32 *ov = (out ? I.dvals : I.fvals) + L.off;
    const bool moves = (const void *)ik != (const void *)ok || iv != ov;  // else sorted in place
    u32 nn = 0;
    if constexpr (K::lossy) {
      if (tid == 0) nl[0] = 0;
      S::sync();
    }
    S::load(x, s, tid, ik, iv, L.n, [&](key_t k, u32 v) { nan_note<K>(nl, k, v); });
    if constexpr (K::lossy) {
      nn = nl[0];
      S::sync();  // read before the list is reset for the group's next leaf
      if (nn > kNanCap) {  // too many to restore: the fix list's exact (key, val) sort takes the leaf
        if (moves)
          for (u32 p = tid; p < L.n; p += T) {
            ok[p] = ik[p];
            ov[p] = iv[p];
          }
        if (tid == 0) push_fix(c, L);
        continue;
      }
    }
    u32 rot = 0;
    int pre = S::presorted(x, s, tid, L.n, s_pre[g], rot);
    if (pre == 4) {  // runs in descending order: every element straight to its place, else sorted
      if (!leaf_runs<S>(s, tid, L.n, s_run[g], s_ri[g], ok, ov)) pre = 0;
#pragma unroll
      for (int k = 0; k < R; k++) x[k] = s[S::px(tid * R + k)];
      S::sync();  // (the moved leaf is written before its NaNs get their bits back)
    }
    if (pre == 0) S::sort(x, s, tid);
    if (pre < 4 && (pre != 1 || moves)) {  // (a sorted leaf in place is left as it is)
      const int n = (int)L.n, r = pre == 3 ? (int)rot : 0;
      const bool rev = pre == 2;
      S::store_mapped(x, s, tid, ok, ov, L.n, [&](int i) { return rev ? n - 1 - i : (i >= r ? i - r : i + n - r); });
    }
    if constexpr (K::lossy) {
      if (nn && (pre != 1 || moves)) {  // (a sorted leaf left in place kept its bits)
        for (u32 i = tid; i < nn; i += T) ok[L.n - nn + nan_rank(nl, nn, nl[1 + i], i)] = (key_t)nl[1 + kNanCap + i];
        S::sync();
      }
    }
    if (tid == 0) {
      __threadfence();
      child_done(c, L.parent, L.flags & 0xffu, L.inst);
    }
  }
}

// Stores the first n elements of a group's s (already in output order),
// coalesced; ends with a barrier.
template <class S>
__device__ __forceinline__ void store_from_s(const typename S::E *s, int tid, typename S::K::key_t *keys, u32 *vals,
                                             u32 n) {
  constexpr int T = S::N / S::R;
#pragma unroll
  for (int k = 0; k < S::R; k++) {
    const int p = k * T + tid;
    if ((u32)p < n) {
      const typename S::E e = s[S::px(p)];
      keys[p] = S::K::key(e);
      vals[p] = S::K::val(e);
    }
  }
  __syncthreads();
}

// The merge sort of a leaf whose radix order failed the (key, val) check
// (equal keys whose vals do not ascend in input order): the leaf is taken
// from s (blocked layout) and put back there sorted.  Out of line and fed
// through shared memory, so that the radix path keeps its registers (an
// array passed by reference to a call would live in local memory).
template <class S>
__device__ __noinline__ void leaf_merge_fallback(typename S::E *s, int tid) {
  typename S::E x[S::R];
#pragma unroll
  for (int k = 0; k < S::R; k++) x[k] = s[S::px(tid * S::R + k)];
  __syncthreads();
  S::sort(x, s, tid);
#pragma unroll
  for (int k = 0; k < S::R; k++) s[S::px(tid * S::R + k)] = x[k];
  __syncthreads();
}

// A leaf of the radix class: one CTA of T threads x R elements, loaded and
// checked for presorted input as in k_leaf, then sorted by RadixLeaf (or
// merge sorted when the radix order is not the (key, val) order).  Leaves
// of 32-bit key ordinals only (uint32, float32 one-word elements).
// CTAs per SM a radix leaf kernel is built for: one for the 16K class (its
// 32 elements a thread need the registers), else the merge kernels' budget.
template <int DT, int T, int R>
constexpr int kRadixMinBlocks() {
  return T * R >= 16384 ? 1 : kLeafMinBlocks<DT, T, false>();
}

template <int DT, int T, int R>
__global__ void __launch_bounds__(T, (kRadixMinBlocks<DT, T, R>())) k_leaf_radix(const Ctx *__restrict__ cp, int cls, u32 count) {
  const Ctx &c = *cp;
  typedef KT<DT> K;
  typedef Sorter<K, T, R, false> S;
  typedef RadixLeaf<K, T, R> RL;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *s = reinterpret_cast<E *>(smem_raw);
  u32 *nl = reinterpret_cast<u32 *>(smem_raw + leaf_sort_bytes<DT, T, R, false>());  // K::lossy only
  u32 *ws = reinterpret_cast<u32 *>(smem_raw + radix_ws_offset<DT, T, R>());
  const int tid = threadIdx.x;
  const bool dyn = count == kDev;  // a fixed-size grid: every CTA takes the next leaf
  const u32 cnt = dyn ? min(c.cnt_cur->leaves[cls], c.leaf_cap[cls]) : count;
  __shared__ u32 s_li;
  __shared__ u32 s_pre[S::kPreWords];
  __shared__ u32 s_run[S::kRunWords];
  __shared__ typename S::RunInfo s_ri[T];
  auto next_leaf = [&](u32 done_li) -> u32 {
    if (!dyn) return done_li == kNone ? blockIdx.x : cnt;  // one leaf per CTA
    if (tid == 0) s_li = atomicAdd(&c.status->cur_leaf[cls], 1u);
    __syncthreads();
    const u32 li = s_li;
    __syncthreads();
    return li;
  };
  for (u32 li = next_leaf(kNone); li < cnt; li = next_leaf(li)) {
    const Leaf L = c.leaves_cur[cls][li];
    const Inst I = c.inst[L.inst];
    E x[R];
    const u32 out = (L.flags >> 8) & 0xffu;
    const bool from_src = (L.flags & LEAF_SRC) != 0;
    const key_t *ik = (const key_t *)(from_src ? I.skeys : I.keys) + L.off;
    const u32 *iv = (from_src ? I.svals : I.vals) + L.off;
    key_t *ok = (key_t *)(out ? I.dkeys : I.fkeys) + L.off;
    u32 *ov = (out ? I.dvals : I.fvals) + L.off;
    const bool moves = (const void *)ik != (const void *)ok || iv != ov;  // else sorted in place
    u32 nn = 0;
    if constexpr (K::lossy) {
      if (tid == 0) nl[0] = 0;
      __syncthreads();
    }
    S::load(x, s, tid, ik, iv, L.n, [&](key_t k, u32 v) { nan_note<K>(nl, k, v); });
    if constexpr (K::lossy) {
      nn = nl[0];
      __syncthreads();  // read before the list is reset for the next leaf
      if (nn > kNanCap) {  // too many to restore: the fix list's exact (key, val) sort takes the leaf
        if (moves)
          for (u32 p = tid; p < L.n; p += T) {
            ok[p] = ik[p];
            ov[p] = iv[p];
          }
        if (tid == 0) push_fix(c, L);
        continue;
      }
    }
    // (the presorted test and the runs read the leaf from s: x is reloaded
    // afterwards, so that it holds no registers meanwhile)
    u32 rot = 0;
    int pre = S::presorted_s(s, tid, L.n, s_pre, rot);
    if (pre == 4) {  // runs in descending order: every element straight to its place, else sorted
      if (!leaf_runs<S>(s, tid, L.n, s_run, s_ri, ok, ov)) pre = 0;
      __syncthreads();  // (the moved leaf is written before its NaNs get their bits back)
    }
    if (pre == 1) {  // sorted: s holds the leaf in order (a sorted leaf in place is left as it is)
      if (moves) store_from_s<S>(s, tid, ok, ov, L.n);
    } else if (pre != 4) {
#pragma unroll
      for (int k = 0; k < R; k++) x[k] = s[S::px(tid * R + k)];
      __syncthreads();  // every thread holds its elements before any writes s (the sort, or the moved store)
      if (pre == 0 && !RL::sort(x, s, tid, L.n, ws)) {  // (RL::sort ends with a barrier: s is free)
#pragma unroll
        for (int k = 0; k < R; k++) s[S::px(tid * R + k)] = x[k];
        __syncthreads();
        leaf_merge_fallback<S>(s, tid);
#pragma unroll
        for (int k = 0; k < R; k++) x[k] = s[S::px(tid * R + k)];
        __syncthreads();
      }
      const int n = (int)L.n, r = pre == 3 ? (int)rot : 0;
      const bool rev = pre == 2;
      S::store_mapped(x, s, tid, ok, ov, L.n, [&](int i) { return rev ? n - 1 - i : (i >= r ? i - r : i + n - r); });
    }
    if constexpr (K::lossy) {
      if (nn && (pre != 1 || moves)) {  // (a sorted leaf left in place kept its bits)
        for (u32 i = tid; i < nn; i += T) ok[L.n - nn + nan_rank(nl, nn, nl[1 + i], i)] = (key_t)nl[1 + kNanCap + i];
        __syncthreads();
      }
    }
    if (tid == 0) {
      __threadfence();
      child_done(c, L.parent, L.flags & 0xffu, L.inst);
    }
  }
}

#ifndef SQ_CLUSTER_MINB
#define SQ_CLUSTER_MINB 2  // CTAs per SM the 512-thread 8-byte-element cluster kernels are built for
#endif
// A leaf of a cluster merge class: CTA `rank` of the cluster loads and
// sorts positions [rank*NC, (rank+1)*NC) of the leaf, then the cluster merges
// through distributed shared memory (ClusterSorter).
template <int DT, int T, int R, int G>
__global__ void __launch_bounds__(T, (T <= 512 && sizeof(typename KT<DT>::elem_t) == 8) ? SQ_CLUSTER_MINB : 1) k_leaf_cluster(const Ctx *__restrict__ cp, int cls, u32 count) {
  const Ctx &c = *cp;
  typedef KT<DT> K;
  typedef ClusterSorter<K, T, R, G> CS;
  typedef typename CS::S S;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *s = reinterpret_cast<E *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const bool dyn = count == kDev;  // a fixed-size grid: every cluster takes the next leaf
  const u32 cnt = dyn ? min(c.cnt_cur->leaves[cls], c.leaf_cap[cls]) : count;
  const int tid = threadIdx.x;
  u32 *nl = reinterpret_cast<u32 *>(smem_raw + leaf_sort_bytes<DT, T, R, false>());  // K::lossy only: this part's NaNs
  __shared__ u32 s_li;
  __shared__ typename CS::PreW s_pre;
  auto next_leaf = [&](u32 done_li) -> u32 {
    if (!dyn) return done_li == kNone ? blockIdx.x / G : cnt;  // one leaf per cluster
    if (rank == 0 && tid == 0) s_li = atomicAdd(&c.status->cur_leaf[cls], 1u);
    cl.sync();
    const u32 li = *cl.map_shared_rank(&s_li, 0);
    cl.sync();  // read everywhere before rank 0 takes the next
    return li;
  };
  for (u32 li = next_leaf(kNone); li < cnt; li = next_leaf(li)) {  // the whole cluster
    const Leaf L = c.leaves_cur[cls][li];
    const Inst I = c.inst[L.inst];
    const u64 off = L.off + (u64)rank * CS::NC;
    const u32 nr = L.n > (u32)rank * CS::NC ? min((u32)CS::NC, L.n - (u32)rank * CS::NC) : 0u;
    const u32 out = (L.flags >> 8) & 0xffu;
    const bool from_src = (L.flags & LEAF_SRC) != 0;
    const key_t *ik = (const key_t *)(from_src ? I.skeys : I.keys) + L.off;
    const u32 *iv = (from_src ? I.svals : I.vals) + L.off;
    key_t *ok = (key_t *)(out ? I.dkeys : I.fkeys) + L.off;
    u32 *ov = (out ? I.dvals : I.fvals) + L.off;
    const bool moves = (const void *)ik != (const void *)ok || iv != ov;  // else sorted in place
    const u32 q0 = (u32)rank * CS::NC;  // this CTA's part of the leaf: [q0, q0 + nr)
    E x[R];
    u32 nn = 0, total = 0;
    if constexpr (K::lossy) {
      if (tid == 0) nl[0] = 0;
      __syncthreads();
    }
    S::load(x, s, tid, ik + q0, iv + q0, nr, [&](key_t k, u32 v) { nan_note<K>(nl, k, v); });
    if constexpr (K::lossy) {
      cl.sync();  // every part's list is complete
      u32 most = 0;
      for (int r = 0; r < G; r++) {
        const u32 m = *cl.map_shared_rank(nl, r);
        total += m;
        most = max(most, m);
      }
      nn = nl[0];
      cl.sync();  // the counts are read before any list changes
      if (most > kNanCap) {  // too many to restore: the fix list's exact (key, val) sort takes the leaf
        if (moves)
          for (u32 p = tid; p < nr; p += T) {
            ok[q0 + p] = ik[q0 + p];
            ov[q0 + p] = iv[q0 + p];
          }
        cl.sync();
        if (rank == 0 && tid == 0) push_fix(c, L);
        continue;
      }
    }
    u32 rot = 0;
    int pre = CS::presorted(x, s, tid, L.n, &s_pre, rot);
    if (pre >= 2) {  // reversed, rotated, or runs in descending order (if they pass the test): moved
      if (!leaf_move_cluster<CS>(s, tid, L.n, pre, rot, &s_pre, ok, ov)) pre = 0;
#pragma unroll
      for (int k = 0; k < R; k++) x[k] = s[S::px(tid * R + k)];
    }
    if (pre <= 1) {
      if (pre == 0) CS::sort(x, s, tid, (int)L.n);
      if (pre == 0 || moves) S::store(x, s, tid, ok + q0, ov + q0, nr);  // a sorted leaf in place stays
    }
    cl.sync();  // (also: no part changes before every CTA has read what it moves)
    if constexpr (K::lossy) {
      if (total && (pre != 1 || moves)) {  // the leaf's NaNs end it, in val order (then by part, entry)
        for (u32 i = tid; i < nn; i += T) {
          const u32 v = nl[1 + i];
          u32 r = 0;
          for (int q = 0; q < G; q++) {
            const u32 *ql = cl.map_shared_rank(nl, q);
            const u32 qn = ql[0];
            for (u32 j = 0; j < qn; j++) {
              const u32 vj = ql[1 + j];
              r += (vj < v) || (vj == v && (q < rank || (q == rank && j < i)));
            }
          }
          ok[L.n - total + r] = (key_t)nl[1 + kNanCap + i];
        }
        cl.sync();  // the lists are read before the next leaf resets them
      }
    }
    if (rank == 0 && tid == 0) {
      __threadfence();
      child_done(c, L.parent, L.flags & 0xffu, L.inst);
    }
  }
}

// A leaf of a radix cluster class: CTA `rank` of the cluster loads
// positions [rank*NC, (rank+1)*NC) of the leaf (NC = T*R); the presorted
// test and the moves of k_leaf_cluster, else every CTA sorts its part with
// RadixLeaf (merge sorting it instead when the radix order is not the
// (key, val) order) and the parts are merged by the cluster's staged
// cross-CTA merge rounds (ClusterSorter::merge_rounds).
template <int DT, int T, int R, int G>
__global__ void __launch_bounds__(T, 1) k_leaf_radix_cluster(const Ctx *__restrict__ cp, int cls, u32 count) {
  const Ctx &c = *cp;
  typedef KT<DT> K;
  typedef ClusterSorter<K, T, R, G> CS;
  typedef typename CS::S S;
  typedef RadixLeaf<K, T, R> RL;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *s = reinterpret_cast<E *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const bool dyn = count == kDev;  // a fixed-size grid: every cluster takes the next leaf
  const u32 cnt = dyn ? min(c.cnt_cur->leaves[cls], c.leaf_cap[cls]) : count;
  const int tid = threadIdx.x;
  u32 *nl = reinterpret_cast<u32 *>(smem_raw + leaf_sort_bytes<DT, T, R, false>());  // K::lossy only: this part's NaNs
  u32 *ws = reinterpret_cast<u32 *>(smem_raw + radix_ws_offset<DT, T, R>());
  __shared__ u32 s_li;
  __shared__ typename CS::PreW s_pre;
  auto next_leaf = [&](u32 done_li) -> u32 {
    if (!dyn) return done_li == kNone ? blockIdx.x / G : cnt;  // one leaf per cluster
    if (rank == 0 && tid == 0) s_li = atomicAdd(&c.status->cur_leaf[cls], 1u);
    cl.sync();
    const u32 li = *cl.map_shared_rank(&s_li, 0);
    cl.sync();  // read everywhere before rank 0 takes the next
    return li;
  };
  for (u32 li = next_leaf(kNone); li < cnt; li = next_leaf(li)) {  // the whole cluster
    const Leaf L = c.leaves_cur[cls][li];
    const Inst I = c.inst[L.inst];
    const u32 nr = L.n > (u32)rank * CS::NC ? min((u32)CS::NC, L.n - (u32)rank * CS::NC) : 0u;
    const u32 out = (L.flags >> 8) & 0xffu;
    const bool from_src = (L.flags & LEAF_SRC) != 0;
    const key_t *ik = (const key_t *)(from_src ? I.skeys : I.keys) + L.off;
    const u32 *iv = (from_src ? I.svals : I.vals) + L.off;
    key_t *ok = (key_t *)(out ? I.dkeys : I.fkeys) + L.off;
    u32 *ov = (out ? I.dvals : I.fvals) + L.off;
    const bool moves = (const void *)ik != (const void *)ok || iv != ov;  // else sorted in place
    const u32 q0 = (u32)rank * CS::NC;  // this CTA's part of the leaf: [q0, q0 + nr)
    E x[R];
    u32 nn = 0, total = 0;
    if constexpr (K::lossy) {
      if (tid == 0) nl[0] = 0;
      __syncthreads();
    }
    S::load(x, s, tid, ik + q0, iv + q0, nr, [&](key_t k, u32 v) { nan_note<K>(nl, k, v); });
    if constexpr (K::lossy) {
      cl.sync();  // every part's list is complete
      u32 most = 0;
      for (int r = 0; r < G; r++) {
        const u32 m = *cl.map_shared_rank(nl, r);
        total += m;
        most = max(most, m);
      }
      nn = nl[0];
      cl.sync();  // the counts are read before any list changes
      if (most > kNanCap) {  // too many to restore: the fix list's exact (key, val) sort takes the leaf
        if (moves)
          for (u32 p = tid; p < nr; p += T) {
            ok[q0 + p] = ik[q0 + p];
            ov[q0 + p] = iv[q0 + p];
          }
        cl.sync();
        if (rank == 0 && tid == 0) push_fix(c, L);
        continue;
      }
    }
    // (the presorted test and the moves read the leaf from shared memory; x
    // is reloaded afterwards, so that it holds no registers meanwhile)
    u32 rot = 0;
    int pre = CS::presorted_s(s, tid, L.n, &s_pre, rot);
    if (pre >= 2) {  // reversed, rotated, or runs in descending order (if they pass the test): moved
      if (!leaf_move_cluster<CS>(s, tid, L.n, pre, rot, &s_pre, ok, ov)) pre = 0;
    }
    if (pre == 1) {  // sorted: s holds this part in order (a sorted leaf in place stays)
      if (moves) store_from_s<S>(s, tid, ok + q0, ov + q0, nr);
    } else if (pre == 0) {
#pragma unroll
      for (int k = 0; k < R; k++) x[k] = s[S::px(tid * R + k)];
      {
        cl.sync();  // every CTA has read what it moves or tests in the others' parts
        if (!RL::sort(x, s, tid, nr, ws)) {  // this part only (RL::sort ends with a barrier: s is free)
#pragma unroll
          for (int k = 0; k < R; k++) s[S::px(tid * R + k)] = x[k];
          __syncthreads();
          leaf_merge_fallback<S>(s, tid);
#pragma unroll
          for (int k = 0; k < R; k++) x[k] = s[S::px(tid * R + k)];
          __syncthreads();
        }
        CS::merge_rounds(x, s, tid, (int)L.n);
      }
      S::store(x, s, tid, ok + q0, ov + q0, nr);
    }
    cl.sync();  // (also: no part changes before every CTA has read what it moves)
    if constexpr (K::lossy) {
      if (total && (pre != 1 || moves)) {  // the leaf's NaNs end it, in val order (then by part, entry)
        for (u32 i = tid; i < nn; i += T) {
          const u32 v = nl[1 + i];
          u32 r = 0;
          for (int q = 0; q < G; q++) {
            const u32 *ql = cl.map_shared_rank(nl, q);
            const u32 qn = ql[0];
            for (u32 j = 0; j < qn; j++) {
              const u32 vj = ql[1 + j];
              r += (vj < v) || (vj == v && (q < rank || (q == rank && j < i)));
            }
          }
          ok[L.n - total + r] = (key_t)nl[1 + kNanCap + i];
        }
        cl.sync();  // the lists are read before the next leaf resets them
      }
    }
    if (rank == 0 && tid == 0) {
      __threadfence();
      child_done(c, L.parent, L.flags & 0xffu, L.inst);
    }
  }
}

// The (key, val) merge sort of the round's fix list (leaves a leaf kernel
// could not sort exactly): clusters of G CTAs loop over the list; each leaf
// sits in its output buffer.
template <int DT, int T, int R, int G>
__global__ void __launch_bounds__(T, 1) k_fixup(const Ctx *__restrict__ cp) {
  const Ctx &c = *cp;
  typedef KT<DT> K;
  typedef ClusterSorter<K, T, R, G> CS;
  typedef typename CS::S S;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ u32 s_item;
  E *s = reinterpret_cast<E *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), tid = threadIdx.x;
  for (;;) {
    if (rank == 0 && tid == 0) s_item = atomicAdd(&c.status->cur_fix, 1u);
    cl.sync();
    const u32 item = *cl.map_shared_rank(&s_item, 0);
    cl.sync();  // everyone has read the item before rank 0 grabs the next
    if (item >= min(c.status->fix_count, c.fix_cap)) break;
    const Leaf L = c.fix[item];
    const Inst I = c.inst[L.inst];
    const u32 out = (L.flags >> 8) & 0xffu;
    key_t *kk = (key_t *)(out ? I.dkeys : I.fkeys) + L.off;
    u32 *vv = (out ? I.dvals : I.fvals) + L.off;
    const u64 off = (u64)rank * CS::NC;
    const u32 nr = L.n > (u32)off ? min((u32)CS::NC, L.n - (u32)off) : 0u;
    E x[R];
    S::load(x, s, tid, kk + off, vv + off, nr);
    CS::sort(x, s, tid, (int)L.n);
    S::store(x, s, tid, kk + off, vv + off, nr);
    cl.sync();
    if (rank == 0 && tid == 0) {
      __threadfence();
      child_done(c, L.parent, L.flags & 0xffu, L.inst);
    }
  }
}

// ------------------------------------------------------------------ plan ---

static __global__ void __launch_bounds__(1024) k_plan(const Ctx *__restrict__ cp, u32 ready_count, int kw) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = c.cnt_cur->ready;
  __shared__ u64 wt[33];
  __shared__ u64 carry[5];
  if (threadIdx.x < 5) carry[threadIdx.x] = 0;
  __syncthreads();
  for (u32 base = 0; base < ready_count; base += blockDim.x) {
    const u32 i = base + threadIdx.x;
    u64 v[5] = {0, 0, 0, 0, 0};
    Node *nd = nullptr;
    if (i < ready_count) {
      nd = &c.nodes[c.ready_cur[i]];
      const u32 ncb = (nd->cols + kCountCols - 1) / kCountCols;
      const u32 nkb = (nd->k + kSkewBkts - 1) / kSkewBkts;
      const u32 ncs = (nd->cols + kSkewCols - 1) / kSkewCols;
      nd->ncb = ncb;
      nd->nkb = nkb;
      nd->ncs = ncs;
      v[0] = ncb;
      v[1] = (u64)ncs * nkb;
      v[2] = (nd->k + 31) / 32;
      v[3] = meta_layout(nd->k, nd->cols, ncb, nkb, kw).total;
      v[4] = (nd->k + kExpandChunk - 1) / kExpandChunk;
    }
    u64 ex[5], tot[5];
#pragma unroll
    for (int q = 0; q < 5; q++) ex[q] = block_excl_scan_u64(v[q], wt, tot[q]);
    if (nd) {
      nd->unit_base = (u32)(carry[0] + ex[0]);
      nd->tile_base = (u32)(carry[1] + ex[1]);
      nd->srow_base = (u32)(carry[2] + ex[2]);
      nd->meta = carry[3] + ex[3];
      c.wbase[i] = nd->unit_base;
      c.wbase[(u64)c.ready_cap + i] = nd->tile_base;
      c.wbase[2ull * c.ready_cap + i] = nd->srow_base;
      c.wbase[3ull * c.ready_cap + i] = (u32)(carry[4] + ex[4]);
    }
    __syncthreads();
    if (threadIdx.x < 5) carry[threadIdx.x] += tot[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c.status->units = (u32)carry[0];
    c.status->tiles = (u32)carry[1];
    c.status->srows = (u32)carry[2];
    c.status->echunks = (u32)carry[4];
    c.status->meta_words = carry[3];
    if (carry[3] > c.meta_cap || carry[1] > 0xffffffffull) atomicOr(&c.status->error, ERRB_ARENA);
  }
}

// ---------------------------------------------------------------- pivots ---
// Algorithm 1, pivot step: draw k-1 positions of the column-sorted node array
// D with replacement, sort the drawn elements, and redraw the whole sample if
// two are equal or the smallest is min(D) (the smallest column head).

// The element just below e in the (key, val) order of integer keys (e itself
// for the minimum).  Float keys never take the appendix variant.
template <class K>
__device__ __forceinline__ typename K::elem_t pred_elem(typename K::elem_t e) {
  if constexpr (K::key_words == 2) {  // uint64 keys: (key, val)
    if (e.x) {
      --e.x;
    } else if (e.k) {
      --e.k;
      e.x = 0xffffffffu;
    }
    return e;
  } else if constexpr (sizeof(typename K::elem_t) == 8 && !K::lossy) {  // uint32 keys: key << 32 | val
    return e ? e - 1 : e;
  } else {
    return e;
  }
}

// Records a node's accepted pivot sample in the trace.
__device__ __forceinline__ void trace_node(const Ctx &c, const Node *nd, u32 attempts) {
  if (!c.trace) return;
  const u32 ti = atomicAdd(&c.status->trace_used, 1u);
  if (ti < c.trace_cap) {
    TraceRec tr;
    tr.off = nd->off;
    tr.n = nd->n;
    tr.m = nd->k;
    tr.hash = nd->hash;
    tr.depth = nd->depth;
    tr.kind = nd->kind;
    tr.attempts = attempts;
    tr.index = nd->index;
    c.trace[ti] = tr;
  } else {
    atomicOr(&c.status->error, ERRB_TRACE);
  }
}

// The pivot step of the paper's appendix listing: k (= m) samples drawn with
// replacement from the node's input A (which the column sorts, writing D,
// leave as it was), sorted; the largest becomes the greatest pair, K::top()
// (the listing's INT_MAX; it stays implicit: bucket k-1 takes everything
// above pivot k-2); a sample equal to the one after it is replaced by its
// predecessor (each comparison with the sample as drawn: the listing lowers
// only the earlier one of a pair).  One sample, no redraws.
template <class K, class S, int T, int R, bool WARP>
__device__ __forceinline__ void pivots_appendix(const Ctx &c, Node *nd, typename K::elem_t *s, int tid) {
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  const u32 ns = nd->k;  // samples
  const Inst I = c.inst[nd->inst];
  const key_t *ak = (const key_t *)(nd->src ? I.skeys : I.keys) + nd->off;
  const u32 *av = (nd->src ? I.svals : I.vals) + nd->off;
  const u64 n = nd->n;
  const u64 sa = attempt_seed(nd->hash, 0);
  const bool stored = nd->samp != kNoSamp;  // drawn when the node was expanded (see sample_appendix)
  const key_t *sk = stored ? reinterpret_cast<const key_t *>(c.samp + nd->samp) : nullptr;
  const u32 *sv = stored ? c.samp + nd->samp + (u64)ns * K::key_words : nullptr;
  E x[R];
#pragma unroll
  for (int q = 0; q < R; q++) {
    const u32 r = tid * R + q;
    if (r < ns) {
      if (stored) {
        x[q] = K::make(sk[r], sv[r]);
      } else {
        const u64 t = __umul64hi(draw(sa, r), n);
        x[q] = K::make(ak[t], av[t]);
      }
    } else {
      x[q] = K::top();
    }
  }
  S::sort(x, s, tid);
  s[tid] = x[0];
  S::sync();
  const E after = s[tid + 1];  // the next thread's first sample (read before anyone rewrites s)
  const MetaLayout ML = meta_layout(nd->k, nd->cols, nd->ncb, nd->nkb, K::key_words);
  key_t *pk = reinterpret_cast<key_t *>(c.meta + nd->meta + ML.pk);
  u32 *pv = c.meta + nd->meta + ML.pv;
#pragma unroll
  for (int q = 0; q < R; q++) {
    const u32 r = tid * R + q;
    if (r + 1 < ns) {  // (sample ns-1 is now the greatest pair)
      E e = x[q];
      const E nx = r + 2 < ns ? (q + 1 < R ? x[q + 1] : after) : K::top();
      if (K::eq(e, nx)) e = pred_elem<K>(e);
      pk[r] = K::key(e);
      pv[r] = K::val(e);
    }
  }
  if (tid == 0) {
    nd->attempts = 1;
    // one guard count per bucket chunk of k_expand_buckets (the columns are
    // done: nothing else counts on pending until then)
    nd->pending = (int)((nd->k + kExpandChunk - 1) / kExpandChunk);
    trace_node(c, nd, 1);
  }
  S::sync();  // the group is done with s before it takes the next node
}

template <class K, class S, int T, int R, bool WARP>
__device__ __forceinline__ void pivots_node(const Ctx &c, Node *nd, typename K::elem_t *s, int tid) {
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  const u32 np = nd->k - 1;  // pivots to draw
  const Inst I = c.inst[nd->inst];
  if (I.variant == VAR_APPENDIX) {
    pivots_appendix<K, S, T, R, WARP>(c, nd, s, tid);
    return;
  }
  const key_t *dk = (const key_t *)I.dkeys + nd->off;
  const u32 *dv = I.dvals + nd->off;
  const u64 n = nd->n;

  // min(D) over the column heads
  E mn = K::top();
  for (u32 i = tid; i < nd->cols; i += T) {
    const u64 p = (u64)i * nd->rows;
    if (p < n) {
      const E e = K::make(dk[p], dv[p]);
      if (K::lt(e, mn)) mn = e;
    }
  }
  mn = warp_min<K>(mn);
  if (!WARP) {
    if ((tid & 31) == 0) s[tid >> 5] = mn;
    __syncthreads();
    if (tid < 32) {
      E v = tid < T / 32 ? s[tid] : K::top();
      v = warp_min<K>(v);
      if (tid == 0) s[0] = v;
    }
    __syncthreads();
    mn = s[0];
    __syncthreads();
  }

  const MetaLayout ML = meta_layout(nd->k, nd->cols, nd->ncb, nd->nkb, K::key_words);
  key_t *pk = reinterpret_cast<key_t *>(c.meta + nd->meta + ML.pk);
  u32 *pv = c.meta + nd->meta + ML.pv;
  for (int a = 0; a < kMaxAttempts; a++) {
    const u64 sa = attempt_seed(nd->hash, (u64)a);
    E x[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
      const u32 r = tid * R + q;
      if (r < np) {
        const u64 t = __umul64hi(draw(sa, r), n);
        x[q] = K::make(dk[t], dv[t]);
      } else {
        x[q] = K::top();
      }
    }
    S::sort(x, s, tid);
    bool bad = false;
#pragma unroll
    for (int q = 0; q + 1 < R; q++)
      if (tid * R + q + 1 < np && K::eq(x[q], x[q + 1])) bad = true;
    s[tid] = x[0];
    S::sync();
    if (tid * R + R < np && K::eq(x[R - 1], s[tid + 1])) bad = true;
    if (tid == 0 && K::eq(x[0], mn)) bad = true;
    bool any;
    if (WARP)
      any = __any_sync(0xffffffffu, bad);
    else
      any = __syncthreads_or(bad);
    if (!any) {
#pragma unroll
      for (int q = 0; q < R; q++) {
        const u32 r = tid * R + q;
        if (r < np) {
          pk[r] = K::key(x[q]);
          pv[r] = K::val(x[q]);
        }
      }
      if (tid == 0) {
        nd->attempts = (u32)a + 1;
        if (c.trace) {
          const u32 ti = atomicAdd(&c.status->trace_used, 1u);
          if (ti < c.trace_cap) {
            TraceRec tr;
            tr.off = nd->off;
            tr.n = nd->n;
            tr.m = nd->k;
            tr.hash = nd->hash;
            tr.depth = nd->depth;
            tr.kind = nd->kind;
            tr.attempts = (u32)a + 1;
            tr.index = nd->index;
            c.trace[ti] = tr;
          } else {
            atomicOr(&c.status->error, ERRB_TRACE);
          }
        }
      }
      S::sync();  // the group is done with s before it takes the next node
      return;
    }
    S::sync();
  }
  if (tid == 0) atomicOr(&c.status->error, ERRB_ATTEMPTS);
  S::sync();
}

template <int DT, int T, int R, bool WARP>
__global__ void __launch_bounds__(WARP ? 256 : T) k_pivots(const Ctx *__restrict__ cp, u32 ready_count, u32 pmin, u32 pmax) {
  const Ctx &c = *cp;
  typedef KT<DT> K;
  typedef Sorter<K, T, R, WARP> S;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *smem = reinterpret_cast<E *>(smem_raw);
  constexpr int groups = WARP ? 8 : 1;
  const int g = WARP ? (threadIdx.x >> 5) : 0;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  // one node per warp (WARP) or per CTA; a fixed-size grid strides over the list
  for (u32 ri = blockIdx.x * groups + g; ri < ready_count; ri += gridDim.x * groups) {
    const u32 id = c.ready_cur[ri];
    Node *nd = &c.nodes[id];
    // elements this group sorts: the k-1 drawn pivots, or the appendix
    // variant's k samples
    const u32 need = c.inst[nd->inst].variant == VAR_APPENDIX ? nd->k : nd->k - 1;
    if (need <= pmin || need > pmax) continue;
    if (nd->meta + meta_layout(nd->k, nd->cols, nd->ncb, nd->nkb, K::key_words).total > c.meta_cap) continue;
    pivots_node<K, S, T, R, WARP>(c, nd, smem + g * S::SMEM, tid);
  }
}

// Pivot step of nodes whose sample is larger than one CTA sorts (k - 1 in
// (max_pivots, 8 * 8192]): one cluster of 8 CTAs of 512 x 16 per node.  CTA
// rank draws sample positions [rank*8192, rank*8192 + 8192) and sorts them,
// the cluster's merge rounds order the whole sample, and Algorithm 1's
// checks (no two drawn elements equal, the smallest above min(D)) and
// redraws run across the cluster, the element after a CTA's part and the
// cluster's outcome read through distributed shared memory.  Besides pk / pv
// the pivots go to the node's pe section as whole elements, where the count
// reads them.
template <int DT>
__global__ void __launch_bounds__(512, 1) k_pivots_cluster(const Ctx *__restrict__ cp, u32 ready_count, u32 pmin) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  typedef KT<DT> K;
  constexpr int T = 512, R = 16, G = 8;
  typedef ClusterSorter<K, T, R, G> CS;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *s = reinterpret_cast<E *>(smem_raw);
  __shared__ E s_first[T];  // every thread's first sorted element
  __shared__ E s_red[T / 32];
  __shared__ E s_min;
  __shared__ int s_bad;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 ncl = gridDim.x / G;
  for (u32 ri = blockIdx.x / G; ri < ready_count; ri += ncl) {  // (the same node for the whole cluster)
    Node *nd = &c.nodes[c.ready_cur[ri]];
    const u32 np = nd->k - 1;  // pivots to draw
    const Inst I = c.inst[nd->inst];
    if (np <= pmin || I.variant == VAR_APPENDIX) continue;
    const MetaLayout ML = meta_layout(nd->k, nd->cols, nd->ncb, nd->nkb, K::key_words);
    if (nd->meta + ML.total > c.meta_cap) continue;
    const key_t *dk = (const key_t *)I.dkeys + nd->off;
    const u32 *dv = I.dvals + nd->off;
    const u64 n = nd->n;
    // min(D) over the column heads: CTA rank takes every G-th block of T columns
    E mn = K::top();
    for (u32 i = (u32)rank * T + tid; i < nd->cols; i += G * T) {
      const u64 p = (u64)i * nd->rows;
      if (p < n) {
        const E e = K::make(dk[p], dv[p]);
        if (K::lt(e, mn)) mn = e;
      }
    }
    mn = warp_min<K>(mn);
    if (lane == 0) s_red[warp] = mn;
    __syncthreads();
    if (tid == 0) {
      E v = s_red[0];
      for (int w = 1; w < T / 32; w++)
        if (K::lt(s_red[w], v)) v = s_red[w];
      s_min = v;
    }
    cl.sync();
    if (rank == 0 && tid == 0)
      for (int r = 1; r < G; r++) {
        const E o = *cl.map_shared_rank(&s_min, r);
        if (K::lt(o, mn)) mn = o;
      }
    if (rank == 0 && tid == 0) mn = K::lt(s_min, mn) ? s_min : mn;
    key_t *pk = reinterpret_cast<key_t *>(c.meta + nd->meta + ML.pk);
    u32 *pv = c.meta + nd->meta + ML.pv;
    E *pe = reinterpret_cast<E *>(c.meta + nd->meta + ML.pe);
    const u32 q0 = (u32)rank * CS::NC + (u32)tid * R;  // this thread's first sample position
    bool done = false;
    for (int a = 0; a < kMaxAttempts && !done; a++) {
      const u64 sa = attempt_seed(nd->hash, (u64)a);
      E x[R];
#pragma unroll
      for (int q = 0; q < R; q++) {
        const u32 r = q0 + q;
        if (r < np) {
          const u64 t = __umul64hi(draw(sa, r), n);
          x[q] = K::make(dk[t], dv[t]);
        } else {
          x[q] = K::top();
        }
      }
      CS::sort(x, s, tid, (int)np);
      bool bad = false;
#pragma unroll
      for (int q = 0; q + 1 < R; q++)
        if (q0 + q + 1 < np && K::eq(x[q], x[q + 1])) bad = true;
      s_first[tid] = x[0];
      cl.sync();  // (every CTA's firsts written; every merge-round read of s done)
      if (q0 + R < np) {
        const E nx = tid + 1 < T ? s_first[tid + 1] : *cl.map_shared_rank(&s_first[0], rank + 1);
        if (K::eq(x[R - 1], nx)) bad = true;
      }
      if (rank == 0 && tid == 0 && K::eq(x[0], mn)) bad = true;
      const int any = __syncthreads_or(bad);
      if (tid == 0) s_bad = any;
      cl.sync();
      int cbad = 0;
      for (int r = 0; r < G; r++) cbad |= *cl.map_shared_rank(&s_bad, r);
      cl.sync();  // the outcomes and firsts are read before the next attempt rewrites them
      if (!cbad) {
#pragma unroll
        for (int q = 0; q < R; q++) {
          const u32 r = q0 + q;
          if (r < np) {
            pk[r] = K::key(x[q]);
            pv[r] = K::val(x[q]);
            pe[r] = x[q];
          }
        }
        if (rank == 0 && tid == 0) {
          nd->attempts = (u32)a + 1;
          trace_node(c, nd, (u32)a + 1);
        }
        done = true;
      }
    }
    if (!done && rank == 0 && tid == 0) atomicOr(&c.status->error, ERRB_ATTEMPTS);
    cl.sync();  // the node is finished by every CTA before the cluster takes the next
  }
}

// Exclusive prefix sum over a warp (and the warp total).
__device__ __forceinline__ u32 warp_excl_scan(u32 v, u32 &total) {
  const int lane = threadIdx.x & 31;
  u32 inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const u32 o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - v;
}

// ----------------------------------------------------------------- count ---
// One pass over the sorted columns of a block of kCountCols columns
// (Section 2.2: each sorted column is scanned against the sorted pivots).
// The block's columns are cut into warp chunks of 32*kCountE elements that
// never cross a column end; every warp takes a contiguous run of chunks,
// kCountE consecutive elements a lane.  A chunk's buckets run from its first
// element's (carried from the warp's previous chunk of the column) to the
// next element's (one warp-wide probe); a chunk with no pivot in that range
// is one bucket and costs no search at all.  Otherwise a lane finds its first
// element's bucket by binary search within the chunk's range and steps over
// the pivots below each next element.  Produces the block's per-bucket totals
// T[I][j], per column the start P[Jb][i] of every kSkewBkts-bucket segment
// (the first position whose bucket is at least Jb*kSkewBkts; the column's
// length past its last bucket), and every element's tag (its bucket within
// its segment) for the SkewTranspose.  GP: the launch for nodes with more
// than kCountSmemPivots pivots, read from the node's pe section in global
// memory (cached in L1/L2), the bucket totals added straight into the
// block's row of T; the other launch keeps pivots and totals in shared
// memory.  Each launch takes only its own nodes' units.

constexpr int kCountE = 8;     // count: consecutive elements a lane
constexpr int kCountStep = 8;  // count: pivots stepped over one by one before a binary search
constexpr u32 kPiece = 256;  // skew: elements per warp work piece

// Bucket of an element that every lane of the warp holds, among the pivots
// piv[lo, hi) (the result is in [lo, hi]): 32-way probes, narrowing the range
// 32-fold a round.
template <class K>
__device__ __forceinline__ int warp_bucket_in(const typename K::elem_t *piv, int lo, int hi,
                                              const typename K::elem_t &e, bool le) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) >> 5;
    const int idx = lo + (lane + 1) * step - 1;
    const bool nb = idx < hi && !below_p<K>(e, piv[idx], le);
    const int cnt = __popc(__ballot_sync(0xffffffffu, nb));
    lo = min(lo + cnt * step, hi);
    hi = min(hi, lo + step - 1);
  }
  const bool nb = lo + lane < hi && !below_p<K>(e, piv[lo + lane], le);
  return lo + __popc(__ballot_sync(0xffffffffu, nb));
}

// P[Jb][col] = pos for the segments that start between a bucket bp (-1 before
// a column's first element) and a bucket b >= bp: Jb in (bp/64, b/64].  Out
// of line: it is rare (a segment spans 64 buckets), and inlined at every
// element of the unrolled loop it made the kernel wait on instruction fetch.
static __device__ __noinline__ void count_seg_starts(u32 *P, u32 cols, u32 col, int bp, int b, u32 pos) {
  for (int Jb = (bp + (int)kSkewBkts) / (int)kSkewBkts; Jb <= b / (int)kSkewBkts; ++Jb)
    P[(u64)Jb * cols + col] = pos;
}

template <int DT, bool GP>
__global__ void __launch_bounds__(1024) k_count(const Ctx *__restrict__ cp, u32 ready_count, u32 kmax) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  typedef KT<DT> K;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  constexpr int EL = sizeof(E) > 8 ? kCountE / 2 : kCountE;  // (three-word elements: half, within 64 registers)
  constexpr u32 CH = 32 * EL;  // elements of a warp chunk
  static_assert(EL % 4 == 0, "128-bit payload loads and word tag stores take 4 elements at a time");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *piv_s = reinterpret_cast<E *>(smem_raw);
  u32 *hist_s = reinterpret_cast<u32 *>(piv_s + (kmax > 1 ? kmax - 1 : 1));
  __shared__ u32 s_u, s_ri;
  __shared__ u32 s_cpre[kCountCols + 1];  // chunks before each column of the block
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NT = blockDim.x, NW = NT >> 5;
  u32 cur = kNone;
  for (;;) {
    grab_item(c, GP ? &c.status->cur_count_big : &c.status->cur_count, c.status->units, 0, ready_count, &s_u,
              &s_ri);
    __syncthreads();
    const u32 u = s_u;
    if (u >= c.status->units) break;
    const u32 id = c.ready_cur[s_ri];
    const Node nd = c.nodes[id];
    __syncthreads();  // (s_u / s_ri are read everywhere before warp 0 may take the next unit)
    if ((nd.k - 1 > kCountSmemPivots) != GP) continue;  // the other launch's node
    const int np = (int)nd.k - 1;
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, K::key_words);
    u32 *meta = c.meta + nd.meta;
    const u32 Iblk = u - nd.unit_base;
    const E *piv = GP ? reinterpret_cast<const E *>(meta + ML.pe) : piv_s;
    u32 *hist = GP ? meta + ML.T + (u64)Iblk * nd.k : hist_s;
    if (!GP && id != cur) {
      const key_t *pk = reinterpret_cast<const key_t *>(meta + ML.pk);
      for (int j = tid; j < np; j += NT) piv_s[j] = K::make(pk[j], meta[ML.pv + j]);
      cur = id;
    }
    for (u32 j = tid; j < nd.k; j += NT) hist[j] = 0;
    const Inst I = c.inst[nd.inst];
    const key_t *dk = (const key_t *)I.dkeys + nd.off;
    const u32 *dv = I.dvals + nd.off;
    uint8_t *tg = I.tags ? I.tags + nd.off : nullptr;
    u32 *P = meta + ML.P;
    const u32 rows = nd.rows, n = nd.n, cols = nd.cols, nkb = nd.nkb;
    const bool le = I.variant == VAR_APPENDIX;  // buckets bounded above by "<="
    const u32 i0 = Iblk * kCountCols;
    const u32 nc = min(cols, i0 + kCountCols) - i0;
    if (warp == 0) {
      u32 nch = 0;
      if ((u32)lane < nc) {
        const u32 i = i0 + lane;
        nch = (u32)((col_end(i, rows, cols, n) - col_begin(i, rows, n) + CH - 1) / CH);
      }
      u32 tot;
      const u32 ex = warp_excl_scan(nch, tot);
      if ((u32)lane <= nc) s_cpre[lane] = ex;  // (lane nc: the block's total)
    }
    __syncthreads();
    const u32 nck = s_cpre[nc];
    const u32 cw0 = (u32)((u64)nck * warp / NW), cw1 = (u32)((u64)nck * (warp + 1) / NW);
    u32 ci = 0;  // column (within the block) of chunk ck
    int lo = -1, bprev = -1;  // bucket of the chunk's first element and of the element before it
    for (u32 ck = cw0; ck < cw1; ++ck) {
      bool fresh = ck == cw0;
      while (s_cpre[ci + 1] <= ck) {
        ++ci;
        fresh = true;
      }
      const u32 col = i0 + ci;
      const u32 cb = (u32)col_begin(col, rows, n), ce = (u32)col_end(col, rows, cols, n);
      const u32 off = (ck - s_cpre[ci]) * CH;  // chunk start within the column
      const u32 g0 = cb + off;
      const u32 na = min(CH, ce - g0);  // elements in the chunk
      const u32 p0 = g0 + (u32)lane * EL;
      E ev[EL];
      if ((u32)(lane + 1) * EL <= na && (((uintptr_t)(dk + p0) | (uintptr_t)(dv + p0)) & 15) == 0) {
        // whole and 16-byte aligned (the same for every lane): 128-bit loads
        key_t kk[EL];
        u32 vv[EL];
#pragma unroll
        for (int q = 0; q < (int)(sizeof(key_t) * EL / 16); q++)
          reinterpret_cast<uint4 *>(kk)[q] = __ldg(reinterpret_cast<const uint4 *>(dk + p0) + q);
#pragma unroll
        for (int q = 0; q < EL / 4; q++) reinterpret_cast<uint4 *>(vv)[q] = __ldg(reinterpret_cast<const uint4 *>(dv + p0) + q);
#pragma unroll
        for (int r = 0; r < EL; r++) ev[r] = K::make(kk[r], vv[r]);
      } else {
#pragma unroll
        for (int r = 0; r < EL; r++)
          ev[r] = (u32)lane * EL + r < na ? K::make(dk[p0 + r], dv[p0 + r]) : K::top();
      }
      if (fresh) {  // the warp's first chunk in this column: search
        lo = warp_bucket_in<K>(piv, 0, np, shfl_e(ev[0], 0), le);
        bprev = -1;
        if (off) bprev = warp_bucket_in<K>(piv, 0, lo, K::make(dk[g0 - 1], dv[g0 - 1]), le);
      }
      const u32 llast = (na - 1) / EL, rlast = (na - 1) % EL;  // lane and slot of the last element
      const bool last_chunk = g0 + na == ce;
      // bucket of the element after the chunk (of its last element, for a column's last chunk)
      E mine = ev[0];
#pragma unroll
      for (int r = 1; r < EL; r++)
        if ((u32)r == rlast) mine = ev[r];
      const E elast = shfl_e(mine, llast);
      const E enx = last_chunk ? elast : K::make(dk[g0 + na], dv[g0 + na]);
      const int hn = warp_bucket_from<K, 16>(piv, lo, np, enx, le);
      const u32 nv = (u32)lane * EL < na ? min((u32)EL, na - (u32)lane * EL) : 0u;  // the lane's elements
      int blast;  // bucket of the chunk's last element
      if (lo == hn) {  // one bucket: no pivot between the chunk's first element and the next
        if (lane == 0) {
          atomicAdd(&hist[lo], na);
          count_seg_starts(P, cols, col, bprev, lo, off);
        }
        if (tg && nv) {
          uint8_t *tp = tg + p0;
          const u32 t = (u32)(lo & (kSkewBkts - 1)) * 0x01010101u;
          if (nv == EL && ((uintptr_t)tp & 3) == 0) {
#pragma unroll
            for (int w = 0; w < EL / 4; w++) reinterpret_cast<u32 *>(tp)[w] = t;
          } else {
            for (u32 r = 0; r < nv; r++) tp[r] = (uint8_t)t;
          }
        }
        blast = lo;
      } else {
        int bk[EL];
        int b = lane == 0 ? lo : (nv ? upper_bound_e<K>(piv, lo, hn, ev[0], le) : hn);
#pragma unroll
        for (int r = 0; r < EL; r++) {
          // up to kCountStep pivots stepped over one by one, a binary search past
          // that (a column of few distinct keys jumps over many pivots at once)
          if ((u32)r < nv) {
            const int lim = min(hn, b + kCountStep);
            while (b < lim && !below_p<K>(ev[r], piv[b], le)) ++b;
            if (b == lim && b < hn && !below_p<K>(ev[r], piv[b], le)) b = upper_bound_e<K>(piv, b + 1, hn, ev[r], le);
          }
          bk[r] = b;
        }
        // segment starts: at the lane's first element from the previous lane's last
        // bucket (the chunk's bprev for lane 0), then wherever the lane's buckets
        // enter a new segment
        int bp = __shfl_up_sync(0xffffffffu, bk[EL - 1], 1);
        if (lane == 0) bp = bprev;
        if (nv) {
          const u32 q0 = off + (u32)lane * EL;
          if (bp < 0 || (bp >> 6) != (bk[0] >> 6)) count_seg_starts(P, cols, col, bp, bk[0], q0);
#pragma unroll
          for (int r = 1; r < EL; r++)
            if ((u32)r < nv && (bk[r - 1] >> 6) != (bk[r] >> 6)) count_seg_starts(P, cols, col, bk[r - 1], bk[r], q0 + r);
          // bucket totals: one shared atomic per run of equal buckets in the lane
          int runb = bk[0];
          u32 runc = 1;
#pragma unroll
          for (int r = 1; r < EL; r++) {
            if ((u32)r >= nv) break;
            if (bk[r] != runb) {
              atomicAdd(&hist[runb], runc);
              runb = bk[r];
              runc = 0;
            }
            ++runc;
          }
          atomicAdd(&hist[runb], runc);
          if (tg) {
            uint8_t *tp = tg + p0;
            if (nv == EL && ((uintptr_t)tp & 3) == 0) {
#pragma unroll
              for (int w = 0; w < EL / 4; w++) {
                u32 wv = 0;
#pragma unroll
                for (int r = 0; r < 4; r++) wv |= (u32)(bk[4 * w + r] & (kSkewBkts - 1)) << (8 * r);
                reinterpret_cast<u32 *>(tp)[w] = wv;
              }
            } else {
#pragma unroll
              for (int r = 0; r < EL; r++)
                if ((u32)r < nv) tp[r] = (uint8_t)(bk[r] & (kSkewBkts - 1));
            }
          }
        }
        int lb = bk[0];
#pragma unroll
        for (int r = 1; r < EL; r++)
          if ((u32)r == rlast) lb = bk[r];
        blast = __shfl_sync(0xffffffffu, lb, llast);
      }
      if (last_chunk) {  // segments past the column's last bucket start at its end
        const u32 len = ce - cb;
        for (int Jb = blast / (int)kSkewBkts + 1 + lane; Jb < (int)nkb; Jb += 32) P[(u64)Jb * cols + col] = len;
      }
      bprev = blast;
      lo = hn;
    }
    __syncthreads();
    if (!GP) {
      u32 *T = meta + ML.T;
      for (u32 j = tid; j < nd.k; j += NT) T[(u64)Iblk * nd.k + j] = hist_s[j];
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ scans ---
// T[I][j] -> exclusive prefix over I (in place); b[j] <- bucket size.
// One work item = 32 buckets; 8 warps split the column blocks.

static __global__ void __launch_bounds__(256) k_scan(const Ctx *__restrict__ cp, u32 ready_count, int kw) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  __shared__ u32 part[8][32];
  __shared__ u32 s_u, s_ri;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  for (;;) {
    grab_item(c, &c.status->cur_scan, c.status->srows, 2, ready_count, &s_u, &s_ri);
    __syncthreads();
    const u32 u = s_u;
    if (u >= c.status->srows) break;
    const Node nd = c.nodes[c.ready_cur[s_ri]];
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, kw);
    u32 *T = c.meta + nd.meta + ML.T;
    u32 *b = c.meta + nd.meta + ML.b;
    const u32 j = (u - nd.srow_base) * 32 + lane;
    const u32 len = (nd.ncb + 7) / 8;
    const u32 Ia = min(nd.ncb, seg * len), Ib = min(nd.ncb, Ia + len);
    u32 sum = 0;
    if (j < nd.k)
      for (u32 I = Ia; I < Ib; ++I) sum += T[(u64)I * nd.k + j];
    part[seg][lane] = sum;
    __syncthreads();
    u32 acc = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (q < seg) acc += part[q][lane];
      tot += part[q][lane];
    }
    if (j < nd.k) {
      for (u32 I = Ia; I < Ib; ++I) {
        const u32 t = T[(u64)I * nd.k + j];
        T[(u64)I * nd.k + j] = acc;
        acc += t;
      }
      if (seg == 0) b[j] = tot;
    }
    __syncthreads();
  }
}

// b[j] (sizes) -> bucket starts b[0..k]; one CTA per ready node at a time.
static __global__ void __launch_bounds__(1024) k_bstart(const Ctx *__restrict__ cp, u32 ready_count, int kw) {
  const Ctx &c = *cp;
  __shared__ u32 wt[33];
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  for (u32 ri = blockIdx.x; ri < ready_count; ri += gridDim.x) {
    const Node nd = c.nodes[c.ready_cur[ri]];
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, kw);
    u32 *b = c.meta + nd.meta + ML.b;
    u32 carry = 0;
    for (u32 base = 0; base < nd.k; base += blockDim.x) {
      const u32 j = base + threadIdx.x;
      const u32 v = j < nd.k ? b[j] : 0;
      u32 tot;
      const u32 ex = block_excl_scan_u32(v, wt, tot);
      if (j < nd.k) b[j] = carry + ex;
      carry += tot;
    }
    if (threadIdx.x == 0) {
      b[nd.k] = carry;
      if (carry != nd.n) atomicOr(&c.status->error, ERRB_SIZES);
    }
  }
}

// ------------------------------------------------------------------ skew ---
// SkewTranspose D -> A (Algorithms 2/3).  A tile is kSkewCols columns x
// kSkewBkts buckets: per column the segment [P[Jb][i], P[Jb+1][i]) (about
// kSkewBkts elements, a coalesced read), per bucket one contiguous run of the
// output (about kSkewCols elements, a coalesced write).  The tile's elements
// are taken in column-major order in chunks of CAP, classified by bucket,
// counted per (column, bucket), placed bucket-major in shared memory --
// within a bucket in column order and, per column, in sorted order, which is
// the order in which Algorithms 2 and 3 append them -- and written out.
// Tiles are numbered bucket-block-major so that neighbouring column blocks,
// whose runs of a bucket are adjacent in A, are written at about the same
// time and merge in L2.  Every step is parallel: prefix sums are warp scans.

template <int DT, int CAP>
struct SkewSmem {
  typedef typename KT<DT>::elem_t E;
  E out_e[CAP];
  E piv[kSkewBkts];
  u32 base[kSkewBkts], running[kSkewBkts], tot[kSkewBkts], ob[kSkewBkts];
  u32 seg_start[kSkewCols], seg_pre[kSkewCols + 1], piece_pre[kSkewCols + 1];
  // per (column, bucket) of the chunk: first and last chunk position of its
  // run (runs are contiguous inside a column); padded, the scans read columns
  u32 first[kSkewCols][kSkewBkts + 1];
  u32 last[kSkewCols][kSkewBkts + 1];
  uint16_t off[kSkewCols][kSkewBkts + 2];  // within a bucket: elements of lower columns
  uint8_t in_j[CAP], out_j[CAP];
  u32 s_u, s_ri, s_S;
};


template <int DT, int CAP, bool TAGS>
__global__ void __launch_bounds__(256) k_skew(const Ctx *__restrict__ cp, u32 ready_count) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  typedef KT<DT> K;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  typedef SkewSmem<DT, CAP> SM;
  static_assert(kSkewCols == 32 && kSkewBkts == 64, "warp scans assume 32 columns x 64 buckets");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
  for (;;) {
    grab_item(c, &c.status->cur_skew, c.status->tiles, 1, ready_count, &sm.s_u, &sm.s_ri);
    __syncthreads();
    const u32 u = sm.s_u;
    if (u >= c.status->tiles) break;
    const Node nd = c.nodes[c.ready_cur[sm.s_ri]];
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, K::key_words);
    const u32 *meta = c.meta + nd.meta;
    const u32 tile = u - nd.tile_base;
    const u32 Jb = tile / nd.ncs, Is = tile - Jb * nd.ncs;
    const u32 j0 = Jb * kSkewBkts, nk = min((u32)kSkewBkts, nd.k - j0);
    const u32 i0 = Is * kSkewCols, nc = min((u32)kSkewCols, nd.cols - i0);
    const u32 *P = meta + ML.P;
    // segments of this tile's columns; warp 0 also forms their prefix sums
    if (warp == 0) {
      u32 len_seg = 0, st = 0;
      if ((u32)lane < nc) {
        const u32 i = i0 + lane;
        const u64 cs = (u64)i * nd.rows;
        const u32 len = cs < nd.n ? (u32)(col_end(i, nd.rows, nd.cols, nd.n) - cs) : 0;
        u32 s0 = 0, s1 = 0;
        if (len) {
          s0 = P[(u64)Jb * nd.cols + i];
          s1 = Jb + 1 < nd.nkb ? P[(u64)(Jb + 1) * nd.cols + i] : len;
        }
        st = (u32)cs + s0;
        len_seg = s1 - s0;
      }
      u32 total;
      const u32 ex = warp_excl_scan(len_seg, total);
      sm.seg_start[lane] = st;
      sm.seg_pre[lane] = ex;
      if (lane == 0) {
        sm.seg_pre[nc] = total;
        sm.s_S = total;
      }
    }
    __syncthreads();
    const u32 S = sm.s_S;
    if (S == 0) continue;  // empty tile (common for sorted inputs)
    const key_t *pk = reinterpret_cast<const key_t *>(meta + ML.pk);
    const u32 *G = meta + ML.T;
    const u32 *b = meta + ML.b;
    if (tid + 1 < (int)nk) sm.piv[tid] = K::make(pk[j0 + tid], meta[ML.pv + j0 + tid]);
    if (tid < (int)nk) {
      sm.base[tid] = b[j0 + tid] + G[(u64)(Is * (kSkewCols / kCountCols)) * nd.k + j0 + tid];
      sm.running[tid] = 0;
    }
    const Inst I = c.inst[nd.inst];
    const key_t *dk = (const key_t *)I.dkeys + nd.off;
    const u32 *dv = I.dvals + nd.off;
    const uint8_t *tg = TAGS ? I.tags + nd.off : nullptr;
    key_t *ak = (key_t *)I.keys + nd.off;
    u32 *av = I.vals + nd.off;
    const int npiv = (int)nk - 1;
    for (u32 cs = 0; cs < S; cs += CAP) {
      const u32 L = min((u32)CAP, S - cs);
      for (u32 q = tid; q < kSkewCols * (kSkewBkts + 1); q += NT) {
        (&sm.first[0][0])[q] = 0xffffffffu;
        (&sm.last[0][0])[q] = 0;
      }
      // pieces of at most kPiece elements of each column's part of the chunk
      if (warp == 0) {
        u32 np_c = 0;
        if ((u32)lane < nc) {
          const u32 a = max(sm.seg_pre[lane], cs), e_ = min(sm.seg_pre[lane + 1], cs + L);
          np_c = e_ > a ? (e_ - a + kPiece - 1) / kPiece : 0;
        }
        u32 t;
        const u32 ex = warp_excl_scan(np_c, t);
        sm.piece_pre[lane] = ex;
        if (lane == 0) sm.piece_pre[kSkewCols] = t;
      }
      __syncthreads();
      // 1. one warp per piece, coalesced reads; buckets are monotone inside a
      //    column, so each group of 32 searches only between the previous
      //    group's last bucket and its own last.  Run starts and ends (per
      //    column and bucket) are recorded with shared-memory min / max.
      const u32 npieces = sm.piece_pre[kSkewCols];
      for (u32 pc = warp; pc < npieces; pc += NW) {
        u32 ci = 0;  // column of this piece: last with piece_pre <= pc
#pragma unroll
        for (u32 st = 16; st > 0; st >>= 1)
          if (ci + st < nc && sm.piece_pre[ci + st] <= pc) ci += st;
        const u32 a = max(sm.seg_pre[ci], cs);
        const u32 pa = a + (pc - sm.piece_pre[ci]) * kPiece;
        const u32 pe = min(min(sm.seg_pre[ci + 1], cs + L), pa + kPiece);
        int carry_b = -1;
        for (u32 g = pa; g < pe; g += 32) {
          const u32 q = g + lane;
          const bool valid = q < pe;
          const u32 vmask = __ballot_sync(0xffffffffu, valid);
          const int lastv = 31 - __clz(vmask);
          int jb;
          if constexpr (TAGS) {  // the count recorded every element's bucket
            jb = valid ? (int)tg[sm.seg_start[ci] + (q - sm.seg_pre[ci])] : 0;
          } else {
            E e = K::top();
            if (valid) {
              const u32 p = sm.seg_start[ci] + (q - sm.seg_pre[ci]);
              e = K::make(dk[p], dv[p]);
            }
            const int lo = carry_b < 0 ? 0 : carry_b;
            const E elast = shfl_e(e, lastv);
            const bool le = c.inst[nd.inst].variant == VAR_APPENDIX;
            const int hi = warp_bucket_from<K>(sm.piv, lo, npiv, elast, le);
            jb = valid ? upper_bound_e<K>(sm.piv, lo, hi, e, le) : hi;
          }
          const int prevb = __shfl_up_sync(0xffffffffu, jb, 1);
          const int nextb = __shfl_down_sync(0xffffffffu, jb, 1);
          if (valid) {
            const u32 ql = q - cs;
            sm.in_j[ql] = (uint8_t)jb;
            if (lane == 0 ? jb != carry_b : jb != prevb) atomicMin(&sm.first[ci][jb], ql);
            if (lane == lastv || nextb != jb) atomicMax(&sm.last[ci][jb], ql);
          }
          carry_b = __shfl_sync(0xffffffffu, jb, lastv);
        }
      }
      __syncthreads();
      // 2. per bucket: exclusive prefix over columns (off) and total (tot)
      for (u32 j = warp; j < kSkewBkts; j += NW) {
        const u32 f = sm.first[lane][j], l = sm.last[lane][j];
        u32 t;
        const u32 ex = warp_excl_scan(f <= l ? l - f + 1 : 0, t);
        sm.off[lane][j] = (uint16_t)ex;
        if (lane == 0) sm.tot[j] = t;
      }
      __syncthreads();
      if (warp == 0) {
        const u32 v0 = sm.tot[2 * lane], v1 = sm.tot[2 * lane + 1];
        u32 t;
        const u32 ex = warp_excl_scan(v0 + v1, t);
        sm.ob[2 * lane] = ex;
        sm.ob[2 * lane + 1] = ex + v0;
      }
      __syncthreads();
      // 3. bucket-major placement in shared memory; the same warps walk the
      //    same pieces and read their elements again (now cached)
      for (u32 pc = warp; pc < npieces; pc += NW) {
        u32 ci = 0;
#pragma unroll
        for (u32 st = 16; st > 0; st >>= 1)
          if (ci + st < nc && sm.piece_pre[ci + st] <= pc) ci += st;
        const u32 a = max(sm.seg_pre[ci], cs);
        const u32 pa = a + (pc - sm.piece_pre[ci]) * kPiece;
        const u32 pe = min(min(sm.seg_pre[ci + 1], cs + L), pa + kPiece);
        for (u32 q = pa + lane; q < pe; q += 32) {
          const u32 ql = q - cs;
          const u32 p = sm.seg_start[ci] + (q - sm.seg_pre[ci]);
          const u32 jl = sm.in_j[ql];
          const u32 slot = sm.ob[jl] + sm.off[ci][jl] + (ql - sm.first[ci][jl]);
          sm.out_e[slot] = K::make(dk[p], dv[p]);
          sm.out_j[slot] = (uint8_t)jl;
        }
      }
      __syncthreads();
      // 4. coalesced write of every bucket's run
      for (u32 s = tid; s < L; s += NT) {
        const u32 jl = sm.out_j[s];
        const u32 dest = sm.base[jl] + sm.running[jl] + (s - sm.ob[jl]);
        const E e = sm.out_e[s];
        if (dest < nd.n) {
          ak[dest] = K::key(e);
          av[dest] = K::val(e);
        } else {
          atomicOr(&c.status->error, ERRB_SIZES);
        }
      }
      __syncthreads();
      if (tid < (int)kSkewBkts) sm.running[tid] += sm.tot[tid];
      __syncthreads();
    }
  }
}

// SkewTranspose of a tile whose elements carry bucket tags (written by the
// count): every chunk of the tile, taken in column-major order, is a stable
// counting sort by tag -- which is exactly the order Algorithms 2 and 3
// append in (bucket, then column, then position).  Warp w ranks a
// contiguous part of the chunk (peers with the same tag from
// __match_any_sync; a (tag, warp) counter kept by the group's lowest lane),
// one scan over the (tag, warp) counters gives every element its slot in
// shared memory, and the chunk leaves with one coalesced run per bucket.
#ifndef SQ_SKEW_WARPS
#define SQ_SKEW_WARPS 2  // warps of a SkewTranspose CTA (each ranks 256 elements of a chunk)
#endif
constexpr u32 kSkewBig = 16384;   // tiles this large look for runs of one tag
constexpr u32 kSkewRunMin = 512;  // the shortest run copied straight
// Runs of one tag in a big SkewTranspose tile.  Tags ascend within a column
// segment (the column is sorted), so the stream positions from cs that share
// its tag form one run: to the end of its column and on through columns of
// that tag alone (t0/t1: a segment's first and last tag, 0xff if empty), or
// up to the first other tag in its column, found by a 32-way search (each
// warp its own, all alike).  Returns the run's end.
static __device__ __forceinline__ u32 skew_col_of(const u32 *seg_pre, u32 nc, u32 q) {
  u32 ci = 0;
#pragma unroll
  for (u32 st = 16; st > 0; st >>= 1)
    if (ci + st < nc && seg_pre[ci + st] <= q) ci += st;
  return ci;
}
static __device__ __noinline__ u32 skew_tag_run(const u32 *seg_start, const u32 *seg_pre, const uint8_t *t0,
                                         const uint8_t *t1, u32 nc, u32 cs, const uint8_t *tg, int lane) {
  const u32 ci = skew_col_of(seg_pre, nc, cs);
  const u32 p = seg_start[ci] + (cs - seg_pre[ci]);
  const u32 tS = tg[p];
  if (t1[ci] == tS) {
    u32 cj = ci + 1;
    while (cj < nc && (t0[cj] == 0xffu || (t0[cj] == tS && t1[cj] == tS))) ++cj;
    return seg_pre[cj];
  }
  u32 lo = p, hi = seg_start[ci] + (seg_pre[ci + 1] - seg_pre[ci]);  // tg[lo] == tS; hi: differs (or the end)
  while (hi - lo > 1) {
    const u32 step = (hi - lo + 31) / 32;
    const u32 pos = lo + step * (u32)(lane + 1);  // lane 31's is at or past hi
    const u32 ball = __ballot_sync(0xffffffffu, pos >= hi || tg[pos] != tS);
    const u32 f = (u32)__ffs((int)ball) - 1u;
    hi = min(hi, lo + step * (f + 1));
    lo += step * f;
  }
  return cs + (hi - p);
}
// Queues the run [cs, rend) of a big tile's stream, dest d0 on, as one
// RunCopy per column piece (lane l: the l-th column the run touches).  False
// (nothing to copy queued) when the list has no room: the caller copies the
// run.  Reserved slots left unused hold empty copies.
static __device__ __noinline__ bool queue_run(const Ctx &c, const Node &nd, const u32 *seg_start, const u32 *seg_pre,
                                              u32 nc, u32 cs, u32 rend, u32 d0, int lane) {
  const u32 c0 = skew_col_of(seg_pre, nc, cs), c1 = skew_col_of(seg_pre, nc, rend - 1);
  const u32 np = c1 - c0 + 1;  // <= kSkewCols
  u32 base = 0;
  if (lane == 0) base = atomicAdd(&c.status->runs_count, np);
  base = __shfl_sync(0xffffffffu, base, 0);
  const bool fits = (u64)base + np <= c.runs_cap && (u64)d0 + (rend - cs) <= nd.n;
  if ((u32)lane < np && base + lane < c.runs_cap) {
    const u32 ci = c0 + lane;
    const u32 qa = max(cs, seg_pre[ci]), qb = min(rend, seg_pre[ci + 1]);
    RunCopy r;
    r.src = nd.off + seg_start[ci] + (qa - seg_pre[ci]);
    r.dst = nd.off + d0 + (qa - cs);
    r.n = fits && qb > qa ? qb - qa : 0u;
    r.inst = nd.inst;
    c.runs[base + lane] = r;
  }
  return fits;
}

// Copies the run [cs, rend) of the tile's stream to dest d0 on, in order.
template <class key_t, int NW>
__device__ __noinline__ void skew_copy_run(const u32 *seg_start, const u32 *seg_pre, u32 nc, u32 cs, u32 rend, u32 d0,
                                           u32 nlim, const key_t *dk, const u32 *dv, key_t *ak, u32 *av, u32 *err,
                                           int tid) {
  constexpr int U = 8;
  for (u32 qb = cs; qb < rend; qb += U * 32 * NW) {
    key_t kk[U];
    u32 vv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {  // every load first
      const u32 q = qb + (u32)(u * 32 * NW + tid);
      if (q < rend) {
        const u32 c2 = skew_col_of(seg_pre, nc, q);
        const u32 p2 = seg_start[c2] + (q - seg_pre[c2]);
        kk[u] = dk[p2];
        vv[u] = dv[p2];
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const u32 q = qb + (u32)(u * 32 * NW + tid);
      if (q < rend) {
        const u32 dest = d0 + (q - cs);
        if (dest < nlim) {
          ak[dest] = kk[u];
          av[dest] = vv[u];
        } else {
          atomicOr(err, ERRB_SIZES);
        }
      }
    }
  }
}

template <int DT, int CAP>
struct SkewTagSmem {
  typedef typename KT<DT>::elem_t E;
  static constexpr int NW = SQ_SKEW_WARPS;  // warps of a CTA
  E out_e[CAP];
  uint8_t out_j[CAP];
  u32 cnt[kSkewBkts * (NW + 1)];  // (tag, warp), tag-major, padded rows
  u32 base[kSkewBkts], running[kSkewBkts], ob[kSkewBkts + 1], adj[kSkewBkts];
  u32 seg_start[kSkewCols], seg_pre[kSkewCols + 1];
  uint8_t seg_t0[kSkewCols], seg_t1[kSkewCols];  // a big tile's column segments: first and last tag (0xff: empty)
  u32 s_u, s_ri, s_S, s_big, s_queued;
};

template <int DT, int CAP>
__global__ void __launch_bounds__(32 * SQ_SKEW_WARPS, 32 / SQ_SKEW_WARPS) k_skew_tags(const Ctx *__restrict__ cp,
                                                                                   u32 ready_count) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  typedef KT<DT> K;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  typedef SkewTagSmem<DT, CAP> SM;
  constexpr int NW = SM::NW, PW = CAP / NW, GR = PW / 32;  // per warp: PW elements in GR groups
  static_assert(kSkewCols == 32 && kSkewBkts == 64 && PW % 32 == 0, "tile geometry");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 lt = (1u << lane) - 1u;
  for (;;) {
    grab_item(c, &c.status->cur_skew, c.status->tiles, 1, ready_count, &sm.s_u, &sm.s_ri);
    __syncthreads();
    const u32 u = sm.s_u;
    if (u >= c.status->tiles) break;
    const Node nd = c.nodes[c.ready_cur[sm.s_ri]];
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, K::key_words);
    const u32 *meta = c.meta + nd.meta;
    const u32 tile = u - nd.tile_base;
    const u32 Jb = tile / nd.ncs, Is = tile - Jb * nd.ncs;
    const u32 j0 = Jb * kSkewBkts, nk = min((u32)kSkewBkts, nd.k - j0);
    const u32 i0 = Is * kSkewCols, nc = min((u32)kSkewCols, nd.cols - i0);
    const u32 *P = meta + ML.P;
    const Inst I = c.inst[nd.inst];
    const uint8_t *tg = I.tags + nd.off;
    if (warp == 0) {  // the tile's column segments and their prefix sums
      u32 len_seg = 0, st = 0;
      if ((u32)lane < nc) {
        const u32 i = i0 + lane;
        const u64 cs = (u64)i * nd.rows;
        const u32 len = cs < nd.n ? (u32)(col_end(i, nd.rows, nd.cols, nd.n) - cs) : 0;
        u32 s0 = 0, s1 = 0;
        if (len) {
          s0 = P[(u64)Jb * nd.cols + i];
          s1 = Jb + 1 < nd.nkb ? P[(u64)(Jb + 1) * nd.cols + i] : len;
        }
        st = (u32)cs + s0;
        len_seg = s1 - s0;
      }
      u32 total;
      const u32 ex = warp_excl_scan(len_seg, total);
      sm.seg_start[lane] = st;
      sm.seg_pre[lane] = ex;
      // a big tile (sorted or reversed input: the tile on the diagonal gets
      // whole columns) notes its segments' first and last tags for the runs
      const bool big = total >= kSkewBig;
      u32 t0 = 0xffu, t1 = 0xffu;
      if (big && len_seg) {
        t0 = tg[st];
        t1 = tg[st + len_seg - 1];
      }
      sm.seg_t0[lane] = (uint8_t)t0;
      sm.seg_t1[lane] = (uint8_t)t1;
      if (lane == 0) {
        sm.seg_pre[32] = total;
        sm.s_S = total;
        sm.s_big = big;
      }
    }
    __syncthreads();
    const u32 S = sm.s_S;
    if (S == 0) continue;  // empty tile (common for sorted inputs)
    const u32 *G = meta + ML.T;
    const u32 *b = meta + ML.b;
    if (tid < (int)nk) {
      sm.base[tid] = b[j0 + tid] + G[(u64)(Is * (kSkewCols / kCountCols)) * nd.k + j0 + tid];
      sm.running[tid] = 0;
    }
    const key_t *dk = (const key_t *)I.dkeys + nd.off;
    const u32 *dv = I.dvals + nd.off;
    key_t *ak = (key_t *)I.keys + nd.off;
    u32 *av = I.vals + nd.off;
    for (int i = tid; i < kSkewBkts * (NW + 1); i += 32 * NW) sm.cnt[i] = 0;
    __syncthreads();
    for (u32 cs = 0; cs < S;) {
      if (sm.s_big) {  // a long run of one tag goes straight to its bucket
        const u32 rend = skew_tag_run(sm.seg_start, sm.seg_pre, sm.seg_t0, sm.seg_t1, nc, cs, tg, lane);
        const u32 c0 = skew_col_of(sm.seg_pre, nc, cs);
        const u32 tS = tg[sm.seg_start[c0] + (cs - sm.seg_pre[c0])];
        if (tS < nk && rend - cs >= kSkewRunMin) {
          const u32 d0 = sm.base[tS] + sm.running[tS];
          // warp 0 hands the run's column pieces to k_copy_runs, which copies
          // them with every SM (a tile's runs would otherwise be copied by
          // this CTA alone); if the list is full, the CTA copies the run here
          if (warp == 0) {
            const bool q = queue_run(c, nd, sm.seg_start, sm.seg_pre, nc, cs, rend, d0, lane);
            if (lane == 0) sm.s_queued = q;
          }
          __syncthreads();  // (also: running[tS] read everywhere)
          if (tid == 0) sm.running[tS] += rend - cs;
          if (!sm.s_queued)
            skew_copy_run<key_t, NW>(sm.seg_start, sm.seg_pre, nc, cs, rend, d0, nd.n, dk, dv, ak, av,
                                     &c.status->error, tid);
          __syncthreads();
          cs = rend;
          continue;
        }
      }
      const u32 L = min((u32)CAP, S - cs);
      // warp `warp` takes chunk positions [warp*PW, warp*PW + PW): first every
      // group's column, tag and element (independent loads), then the ranks
      E ev[GR];
      u32 rt[GR];  // tag, then tag << 16 | rank within the warp's part
#pragma unroll
      for (int g = 0; g < GR; g++) {
        const u32 ql = (u32)(warp * PW + g * 32 + lane);
        rt[g] = 0xffu;
        ev[g] = K::top();
        if (ql < L) {
          const u32 q = cs + ql;
          const u32 ci = skew_col_of(sm.seg_pre, nc, q);  // the last column with seg_pre <= q
          const u32 p = sm.seg_start[ci] + (q - sm.seg_pre[ci]);
          rt[g] = tg[p];
          ev[g] = K::make(dk[p], dv[p]);
        }
      }
#pragma unroll
      for (int g = 0; g < GR; g++) {
        const u32 t = rt[g];
        const bool valid = t < (u32)kSkewBkts;
        const u32 peers = __match_any_sync(0xffffffffu, t);
        const u32 before = __popc(peers & lt);
        u32 r0 = 0;
        if (valid && before == 0) {  // the group's lowest lane reserves its slots
          r0 = sm.cnt[t * (NW + 1) + warp];
          sm.cnt[t * (NW + 1) + warp] = r0 + (u32)__popc(peers);
        }
        r0 = __shfl_sync(0xffffffffu, r0, __ffs(peers) - 1);
        __syncwarp();
        rt[g] = (t << 16) | (r0 + before);
      }
      __syncthreads();
      // warp 0: per tag, the warps' exclusive offsets and the tag's start in
      // the chunk; every counter becomes the slot of its warp's first element
      if (warp == 0) {
        u32 tot[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int t = 2 * lane + h;
          u32 run = 0;
#pragma unroll
          for (int w2 = 0; w2 < NW; w2++) {
            const u32 v = sm.cnt[t * (NW + 1) + w2];
            sm.cnt[t * (NW + 1) + w2] = run;
            run += v;
          }
          tot[h] = run;
        }
        u32 total;
        const u32 ex = warp_excl_scan(tot[0] + tot[1], total);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int t = 2 * lane + h;
          const u32 o = ex + (h ? tot[0] : 0);
          sm.ob[t] = o;
#pragma unroll
          for (int w2 = 0; w2 < NW; w2++) sm.cnt[t * (NW + 1) + w2] += o;
          // output offset of the chunk's run of bucket t: dest = adj[t] + slot
          if (t < (int)nk) {
            sm.adj[t] = sm.base[t] + sm.running[t] - o;
            sm.running[t] += tot[h];
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int g = 0; g < GR; g++) {
        const u32 t = rt[g] >> 16;
        if (t < (u32)kSkewBkts) {
          const u32 slot = sm.cnt[t * (NW + 1) + warp] + (rt[g] & 0xffffu);
          sm.out_e[slot] = ev[g];
          sm.out_j[slot] = (uint8_t)t;
        }
      }
      __syncthreads();
      // one coalesced run per bucket; the counters are free for the next chunk
      for (u32 s2 = tid; s2 < L; s2 += 32 * NW) {
        const u32 dest = sm.adj[sm.out_j[s2]] + s2;
        const E e = sm.out_e[s2];
        if (dest < nd.n) {
          ak[dest] = K::key(e);
          av[dest] = K::val(e);
        } else {
          atomicOr(&c.status->error, ERRB_SIZES);
        }
      }
      for (int i = tid; i < kSkewBkts * (NW + 1); i += 32 * NW) sm.cnt[i] = 0;
      __syncthreads();
      cs += L;
    }
  }
}

// --------------------------------------------------------------- spawning ---
// Children are appended block-cooperatively: one global atomic per leaf class
// (and one for new nodes) per batch of blockDim.x children.

struct Child {
  u64 off;
  u64 hash;
  u32 n, inst, parent, kind, index, depth, out, src;
};

static __device__ void spawn_batch(const Ctx &c, bool has, const Child &ch, u32 *fresh_list, u32 *fresh_count,
                            int nclass) {
  __shared__ u32 ccount[kLeafClasses + 1], cbase[kLeafClasses + 1], fbase;
  __shared__ u64 celems[kLeafClasses + 1];
  if (threadIdx.x <= kLeafClasses) {
    ccount[threadIdx.x] = 0;
    celems[threadIdx.x] = 0;
  }
  __syncthreads();
  int cls = -1;
  u32 local = 0;
  if (has) {
    cls = ch.n <= c.inst[ch.inst].cutoff ? class_of(ch.n, nclass) : kLeafClasses;
    local = atomicAdd(&ccount[cls], 1u);
    atomicAdd(&celems[cls], (u64)ch.n);
  }
  __syncthreads();
  if (threadIdx.x < kLeafClasses) {
    const u32 q = ccount[threadIdx.x];
    cbase[threadIdx.x] = q ? atomicAdd(&c.cnt_nxt->leaves[threadIdx.x], q) : 0;
    if (q) atomicAdd(&c.cnt_nxt->leaf_elems[threadIdx.x], celems[threadIdx.x]);
  } else if (threadIdx.x == kLeafClasses) {
    const u32 q = ccount[kLeafClasses];
    cbase[kLeafClasses] = q ? atomicAdd(&c.status->nodes_used, q) : 0;
    fbase = q ? atomicAdd(fresh_count, q) : 0;
  }
  __syncthreads();
  if (has) {
    if (cls < kLeafClasses) {
      const u32 idx = cbase[cls] + local;
      if (idx < c.leaf_cap[cls]) {
        Leaf L;
        L.off = ch.off;
        L.n = ch.n;
        L.inst = ch.inst;
        L.parent = ch.parent;
        L.flags = ch.kind | (ch.out << 8) | (ch.src ? LEAF_SRC : 0u);
        c.leaves_nxt[cls][idx] = L;
      } else {
        atomicOr(&c.status->error, ERRB_LIST);
      }
    } else {
      const u32 id = cbase[kLeafClasses] + local;
      const u32 fi = fbase + local;
      if (id < c.node_cap && fi < c.fresh_cap) {
        Node nn;
        const u32 m = node_m(ch.n, c.inst[ch.inst].variant);
        nn.off = ch.off;
        nn.hash = ch.hash;
        nn.meta = 0;
        nn.samp = kNoSamp;
        nn.n = ch.n;
        nn.rows = nn.cols = nn.k = m;
        nn.inst = ch.inst;
        nn.parent = ch.parent;
        nn.kind = ch.kind;
        nn.index = ch.index;
        nn.depth = ch.depth;
        nn.out = ch.out;
        nn.pending = 0;
        nn.attempts = 0;
        nn.unit_base = nn.tile_base = nn.srow_base = 0;
        nn.ncb = nn.nkb = nn.ncs = 0;
        nn.src = ch.src;
        c.nodes[id] = nn;
        fresh_list[fi] = id;
      } else {
        atomicOr(&c.status->error, ERRB_NODES);
      }
    }
  }
  __syncthreads();
}

// The run copies queued by this round's SkewTranspose (D -> A): every warp
// takes the next one and copies it, eight loads in flight per lane.
template <int DT>
__global__ void __launch_bounds__(256) k_copy_runs(const Ctx *__restrict__ cp) {
  const Ctx &c = *cp;
  typedef typename KT<DT>::key_t key_t;
  const u32 count = min(c.status->runs_count, c.runs_cap);
  if (count == 0) return;
  const int lane = threadIdx.x & 31;
  for (;;) {
    u32 i = 0;
    if (lane == 0) i = atomicAdd(&c.status->runs_cursor, 1u);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= count) break;
    const RunCopy r = c.runs[i];
    const Inst I = c.inst[r.inst];
    const key_t *dk = (const key_t *)I.dkeys + r.src;
    const u32 *dv = I.dvals + r.src;
    key_t *ak = (key_t *)I.keys + r.dst;
    u32 *av = I.vals + r.dst;
    constexpr int U = 8;
    for (u32 qb = 0; qb < r.n; qb += U * 32) {
      key_t kk[U];
      u32 vv[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const u32 q = qb + (u32)(u * 32 + lane);
        if (q < r.n) {
          kk[u] = dk[q];
          vv[u] = dv[q];
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const u32 q = qb + (u32)(u * 32 + lane);
        if (q < r.n) {
          ak[q] = kk[u];
          av[q] = vv[u];
        }
      }
    }
  }
}

// The appendix variant's monochromatic rule for bucket j of a node (see
// k_expand_buckets), from the node's k-1 stored pivots.
template <int DT>
__device__ __forceinline__ bool mono_bucket(const u32 *meta, const MetaLayout &ML, u32 k, u32 j) {
  typedef KT<DT> K;
  typedef typename K::key_t key_t;
  typedef typename K::elem_t E;
  const key_t *pk = reinterpret_cast<const key_t *>(meta + ML.pk);
  const u32 *pv = meta + ML.pv;
  if (j == 0) return K::eq(K::make(pk[0], pv[0]), K::make(0, 0u));
  const E lo = K::make(pk[j - 1], pv[j - 1]);
  const E hi = j + 1 < k ? K::make(pk[j], pv[j]) : K::top();
  return K::lt(lo, hi) && K::eq(pred_elem<K>(hi), lo);
}

// Copies the monochromatic buckets of one k_expand_buckets chunk (each thread
// names its own, n = 0 for none) from A, where the SkewTranspose left them,
// to the node's output (D, or the final buffer); the block takes them in turn.
template <int DT>
__device__ void copy_mono_buckets(const Inst &I, u32 out, u64 off, u32 n) {
  typedef typename KT<DT>::key_t key_t;
  __shared__ u64 s_off[kExpandChunk];
  __shared__ u32 s_n[kExpandChunk];
  if (threadIdx.x < kExpandChunk) {
    s_off[threadIdx.x] = off;
    s_n[threadIdx.x] = n;
  }
  __syncthreads();
  const key_t *ak = (const key_t *)I.keys;
  const u32 *av = I.vals;
  key_t *ok = (key_t *)(out ? I.dkeys : I.fkeys);
  u32 *ov = out ? I.dvals : I.fvals;
  if ((const void *)ak != (const void *)ok || av != ov) {  // else already in place
    for (int t = 0; t < kExpandChunk; t++) {
      const u32 len = s_n[t];
      const u64 o = s_off[t];
      for (u32 i = threadIdx.x; i < len; i += blockDim.x) {
        ok[o + i] = ak[o + i];
        ov[o + i] = av[o + i];
      }
    }
  }
  __syncthreads();  // (s_off / s_n are reused by the block's next chunk)
}

// Bucket children of every ready node (Algorithm 1's last loop), spawned in
// work items of kExpandChunk buckets.  Every bucket of an Algorithm 1 node is
// non-empty (bucket j >= 1 holds pivot j, bucket 0 the minimum), so the node
// waits for exactly k children.
template <int DT>
__global__ void __launch_bounds__(256) k_expand_buckets(const Ctx *__restrict__ cp, u32 ready_count) {
  const Ctx &c = *cp;
  if (ready_count == kDev) ready_count = min(c.cnt_cur->ready, c.ready_cap);
  __shared__ u32 s_u, s_ri;
  for (;;) {
    grab_item(c, &c.status->cur_ebkt, c.status->echunks, 3, ready_count, &s_u, &s_ri);
    __syncthreads();
    const u32 u = s_u;
    if (u >= c.status->echunks) break;
    const u32 id = c.ready_cur[s_ri];
    const Node nd = c.nodes[id];
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, KT<DT>::key_words);
    const u32 *b = c.meta + nd.meta + ML.b;
    const u32 chunk = u - c.wbase[3ull * c.ready_cap + s_ri];
    // Under the appendix variant a bucket may be empty (a pivot lowered to
    // its predecessor need not be an element of the node), and a bucket
    // whose range holds a single (key, val) pair -- bucket j > 0 with pivot
    // j-1 the predecessor of pivot j (pivot k-1 the greatest pair), or bucket
        // 0 with pivot 0 the least pair -- holds only copies of it and is copied
    // to the node's output instead of sorted.  The node then waits for its
    // other buckets only, which every chunk adds to its pending count (the
    // pivot step set one guard per chunk; its children start in the next
    // round).
    const Inst I = c.inst[nd.inst];
    const bool var = I.variant == VAR_APPENDIX;
    if (!var && chunk == 0 && threadIdx.x == 0) c.nodes[id].pending = (int)nd.k;
    const u32 j = chunk * kExpandChunk + threadIdx.x;
    Child ch;
    bool has = false, mono = false;
    if (threadIdx.x < kExpandChunk && j < nd.k) {
      ch.n = b[j + 1] - b[j];
      has = true;
      if (ch.n == 0) {
        if (!var) atomicOr(&c.status->error, ERRB_SIZES);  // cannot happen for a valid Algorithm 1 sample
        has = false;
      } else if (var) {
        mono = mono_bucket<DT>(c.meta + nd.meta, ML, nd.k, j);
        has = !mono;
      }
      ch.off = nd.off + b[j];
      ch.hash = buc_hash(nd.hash, j);
      ch.inst = nd.inst;
      ch.parent = id;
      ch.kind = KIND_BUC;
      ch.index = j;
      ch.depth = nd.depth + 1;
      ch.out = nd.out;
      ch.src = 0;  // a bucket reads what its parent's SkewTranspose wrote
    }
    if (var) {
      // this chunk's waiting buckets replace its guard count; the last chunk
      // of a node none of whose buckets waits reports the node complete (its
      // copies are in place when the next kernel starts)
      const int waits = __syncthreads_count(has);
      if (__syncthreads_or(mono)) copy_mono_buckets<DT>(I, nd.out, mono ? nd.off + b[j] : 0, mono ? ch.n : 0);
      if (threadIdx.x == 0 && atomicAdd(&c.nodes[id].pending, waits - 1) + waits - 1 == 0)
        child_done(c, nd.parent, nd.kind, nd.inst);
    }
    spawn_batch(c, has, ch, c.fresh_cur, &c.cnt_cur->fresh, LeafCfg<DT>::nclass);
  }
}

// The appendix variant draws a node's pivot sample from its input before its
// columns are sorted.  A column that recurses rewrites its part of that
// input (its own SkewTranspose lands there), so a node with such a column
// copies its k draws to the sample store here, before its columns start, and
// its pivot step reads them back; a node whose columns are all leaves draws
// from its input at the pivot step, which the leaf sorts leave as it was.
template <int DT>
__device__ void sample_appendix(const Ctx &c, u32 id, const Node &nd, const Inst &I, u32 ncol) {
  typedef KT<DT> K;
  typedef typename K::key_t key_t;
  __shared__ u64 s_off;
  const u64 last = (u64)nd.n - (u64)(ncol - 1) * nd.rows;  // the last column runs to n
  if (max((u64)nd.rows, last) <= I.cutoff) return;         // (the same for the whole block)
  const u32 k = nd.k;
  const u64 words = ((u64)k * (K::key_words + 1) + 1) & ~1ull;  // (even: 8-byte keys stay aligned)
  if (threadIdx.x == 0) {
    u64 o = atomicAdd(&c.status->samp_used, words);
    if (o + words > c.samp_cap) {
      atomicOr(&c.status->error, ERRB_SAMP);
      o = kNoSamp;
    }
    s_off = o;
    c.nodes[id].samp = o;
  }
  __syncthreads();
  const u64 o = s_off;
  if (o == kNoSamp) return;
  const key_t *ak = (const key_t *)(nd.src ? I.skeys : I.keys) + nd.off;
  const u32 *av = (nd.src ? I.svals : I.vals) + nd.off;
  const u64 sa = attempt_seed(nd.hash, 0);
  key_t *sk = reinterpret_cast<key_t *>(c.samp + o);
  u32 *sv = c.samp + o + (u64)k * K::key_words;
  for (u32 r = threadIdx.x; r < k; r += blockDim.x) {
    const u64 t = __umul64hi(draw(sa, r), (u64)nd.n);
    sk[r] = ak[t];
    sv[r] = av[t];
  }
}

// Column children of every new node (Algorithm 1's first loop); new internal
// column nodes are expanded in the next round.
template <int DT>
__global__ void __launch_bounds__(256) k_expand_cols(const Ctx *__restrict__ cp) {
  const Ctx &c = *cp;
  __shared__ u32 s_u;
  for (;;) {
    if (threadIdx.x == 0) s_u = atomicAdd(&c.status->cur_expand, 1u);
    __syncthreads();
    const u32 u = s_u;
    if (u >= min(c.cnt_cur->fresh, c.fresh_cap)) break;
    const u32 id = c.fresh_cur[u];
    const Node nd = c.nodes[id];
    const u32 ncol = min(nd.cols, (u32)(((u64)nd.n + nd.rows - 1) / nd.rows));  // non-empty columns
    if (threadIdx.x == 0) c.nodes[id].pending = (int)ncol;
    const Inst I = c.inst[nd.inst];
    if (I.variant == VAR_APPENDIX) sample_appendix<DT>(c, id, nd, I, ncol);
    for (u32 base = 0; base < ncol; base += blockDim.x) {
      const u32 i = base + threadIdx.x;
      Child ch;
      const bool has = i < ncol;
      if (has) {
        const u64 st = (u64)i * nd.rows;
        ch.n = (u32)(i + 1 == ncol ? (u64)nd.n - st : (u64)nd.rows);  // (the last one runs to n)
        ch.off = nd.off + st;
        ch.hash = col_hash(nd.hash, i);
        ch.inst = nd.inst;
        ch.parent = id;
        ch.kind = KIND_COL;
        ch.index = i;
        ch.depth = nd.depth + 1;
        ch.out = 1;  // columns are sorted from A into D
        ch.src = nd.src;  // (reading where the node's own input lies)
      }
      spawn_batch(c, has, ch, c.fresh_nxt, &c.cnt_nxt->fresh, LeafCfg<DT>::nclass);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- round control ---

// Start of a round: zero the next round's counters and this round's work
// cursors (the pointers come from the round's context, so the same launch
// serves every run).
static __global__ void k_round_begin(const Ctx *__restrict__ cp) {
  const Ctx &c = *cp;
  constexpr u32 nc = sizeof(Counters) / 4;
  u32 *z = reinterpret_cast<u32 *>(c.cnt_nxt);
  for (u32 i = threadIdx.x; i < nc; i += blockDim.x) z[i] = 0;
  u32 *cur = &c.status->cur_count;
  if (threadIdx.x < kRoundCursors) cur[threadIdx.x] = 0;
}

// Totals of a graph-launched run (a host-driven run counts on the host).
struct GraphStats {
  unsigned long long rounds, nodes, leaf_elems, ready_elems;
  u32 grow;  // the loop stopped because the node pool needs to grow
  u32 pad;
};

// End of a round of a graph-launched run: add the round's work to the
// totals and set the loop condition -- another round runs unless every
// instance is done, an error is latched, the node pool must grow first (the
// host grows it and relaunches), or the round limit is reached.  `next` is
// the condition of the body's second round (0 when this is that round).
static __global__ void k_round_end(const Ctx *__restrict__ cp, cudaGraphConditionalHandle loop,
                                   cudaGraphConditionalHandle next, int has_next, GraphStats *gs,
                                   unsigned long long max_rounds) {
  const Ctx &c = *cp;
  const Counters &C = *c.cnt_cur;
  unsigned long long le = 0;
  for (int cl = 0; cl < kLeafClasses; cl++) le += C.leaf_elems[cl];
  gs->rounds += 1;
  gs->nodes += C.ready;
  gs->leaf_elems += le;
  gs->ready_elems += C.ready_elems;
  const Status &S = *c.status;
  const bool grow = (u64)S.nodes_used + c.fresh_cap > c.node_cap;
  if (grow) gs->grow = 1;
  const bool more = !(S.error & ~ERRB_TRACE) && S.done < c.ninst && !grow && gs->rounds < max_rounds;
  cudaGraphSetConditional(loop, more ? 1u : 0u);
  if (has_next) cudaGraphSetConditional(next, more ? 1u : 0u);
}

// ------------------------------------------------ stand-alone SkewTranspose ---

// Caller-supplied pivots -> the node's metadata.
template <int DT>
__global__ void k_put_pivots(const Ctx *__restrict__ cp, const typename KT<DT>::key_t *pk, const u32 *pv) {
  const Ctx &c = *cp;
  const Node &nd = c.nodes[c.ready_cur[0]];
  const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, KT<DT>::key_words);
  const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j + 1 < nd.k) {
    reinterpret_cast<typename KT<DT>::key_t *>(c.meta + nd.meta + ML.pk)[j] = pk[j];
    c.meta[nd.meta + ML.pv + j] = pv[j];
  }
}

// Bucket starts b[0..k] -> the caller's 64-bit array.
template <int DT>
__global__ void k_get_bstart(const Ctx *__restrict__ cp, u64 *out) {
  const Ctx &c = *cp;
  const Node &nd = c.nodes[c.ready_cur[0]];
  const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, KT<DT>::key_words);
  const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j <= nd.k) out[j] = c.meta[nd.meta + ML.b + j];
}

}  // namespace sq
