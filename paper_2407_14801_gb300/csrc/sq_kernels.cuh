// SquareSort engine kernels (Algorithm 1 of Koucky & Matejka, Section 2).
//
// The recursion is run breadth-first in rounds.  Each round:
//   k_leaf          sorts every pending leaf (n <= cutoff: Algorithm 1's
//                   simple_sort) in registers + shared memory;
//   k_plan          numbers the work of every node whose columns are sorted;
//   k_pivots        draws, sorts and checks those nodes' pivot samples;
//   k_count         one pass over each sorted column: bucket totals per block
//                   of columns and the start of every 64-bucket segment
//                   (Section 2.2, "scan of the column simultaneously with the
//                   scan of the pivots");
//   k_scan/k_bstart prefix sums: bucket starts and per-block offsets;
//   k_skew          SkewTranspose (Algorithm 2 / 3) as a tiled stable
//                   partition staged in shared memory;
//   k_expand_*      spawn the bucket / column children (Algorithm 1's
//                   recursive calls) as leaves or new nodes.
// A leaf finishing decrements its parent's pending count; the last column
// makes the parent ready for the next round, the last bucket completes it.
#pragma once
#include "sq_sorter.cuh"

namespace sq {

// ------------------------------------------------------------ helpers ------

template <int DT>
struct LeafCfg;
template <>
struct LeafCfg<DT_U32> {
  static constexpr int nclass = 5;
};
template <>
struct LeafCfg<DT_F32> {
  static constexpr int nclass = 4;
};
template <>
struct LeafCfg<DT_U64> {
  static constexpr int nclass = 4;
};
// Class c sorts up to class_cap(c) elements: c0 = warp x 2, c1 = warp x 16,
// c2 = 128 x 16, c3 = 512 x 16, c4 = 1024 x 16 (uint32 keys only).
__host__ __device__ __forceinline__ u32 class_cap(int c) {
  return c == 0 ? 64u : c == 1 ? 512u : c == 2 ? 2048u : c == 3 ? 8192u : 16384u;
}

__host__ __device__ __forceinline__ int class_of(u32 n, int nclass) {
  int c = 0;
  while (c < nclass - 1 && n > class_cap(c)) ++c;
  return c;
}

// number of pivots <= e in piv[lo, hi)
template <class K>
__device__ __forceinline__ int upper_bound_e(const typename K::elem_t *piv, int lo, int hi,
                                             const typename K::elem_t &e) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (K::lt(e, piv[mid]))
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
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

// Ready-list position of the node owning work item u (nodes are numbered in
// list order, so *_base increases along the list).
template <int FIELD>
__device__ __forceinline__ u32 find_owner(const Ctx &c, u32 ready_count, u32 u) {
  u32 lo = 0, hi = ready_count;  // last index with base <= u
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    const Node &nd = c.nodes[c.ready_cur[mid]];
    const u32 b = FIELD == 0 ? nd.unit_base : (FIELD == 1 ? nd.tile_base : nd.srow_base);
    if (b <= u)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// A finished unit of work (leaf or completed node) reports to its parent.
static __device__ void child_done(const Ctx &c, u32 parent, u32 kind, u32 inst) {
  for (;;) {
    if (parent == kNone) {
      const u32 d = atomicAdd(&c.status->done, 1u);
      c.done_list[d] = inst;
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

template <int DT, int T, int R, bool WARP>
__global__ void __launch_bounds__(WARP ? 256 : T) k_leaf(Ctx c, int cls, u32 count) {
  typedef KT<DT> K;
  typedef Sorter<K, T, R, WARP> S;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *smem = reinterpret_cast<E *>(smem_raw);
  constexpr int groups = WARP ? 8 : 1;
  const int g = WARP ? (threadIdx.x >> 5) : 0;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const u32 li = blockIdx.x * groups + g;
  if (li >= count) return;  // a whole warp (WARP) or the whole CTA
  const Leaf L = c.leaves_cur[cls][li];
  const Inst I = c.inst[L.inst];
  E *s = smem + g * S::SMEM;
  E x[R];
  S::load(x, s, tid, (const key_t *)I.keys + L.off, I.vals + L.off, L.n);
  S::sort(x, s, tid);
  const u32 out = L.flags >> 8;
  key_t *ok = (key_t *)(out ? I.dkeys : I.keys) + L.off;
  u32 *ov = (out ? I.dvals : I.vals) + L.off;
  S::store(x, s, tid, ok, ov, L.n);
  if (tid == 0) {
    __threadfence();
    child_done(c, L.parent, L.flags & 0xffu, L.inst);
  }
}

// ------------------------------------------------------------------ plan ---

static __global__ void __launch_bounds__(1024) k_plan(Ctx c, u32 ready_count, int kw) {
  __shared__ u64 wt[33];
  __shared__ u64 carry[4];
  if (threadIdx.x < 4) carry[threadIdx.x] = 0;
  __syncthreads();
  for (u32 base = 0; base < ready_count; base += blockDim.x) {
    const u32 i = base + threadIdx.x;
    u64 v[4] = {0, 0, 0, 0};
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
    }
    u64 ex[4], tot[4];
#pragma unroll
    for (int q = 0; q < 4; q++) ex[q] = block_excl_scan_u64(v[q], wt, tot[q]);
    if (nd) {
      nd->unit_base = (u32)(carry[0] + ex[0]);
      nd->tile_base = (u32)(carry[1] + ex[1]);
      nd->srow_base = (u32)(carry[2] + ex[2]);
      nd->meta = carry[3] + ex[3];
    }
    __syncthreads();
    if (threadIdx.x < 4) carry[threadIdx.x] += tot[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c.status->units = (u32)carry[0];
    c.status->tiles = (u32)carry[1];
    c.status->srows = (u32)carry[2];
    c.status->meta_words = carry[3];
    if (carry[3] > c.meta_cap || carry[1] > 0xffffffffull) atomicOr(&c.status->error, ERRB_ARENA);
  }
}

// ---------------------------------------------------------------- pivots ---
// Algorithm 1, pivot step: draw k-1 positions of the column-sorted node array
// D with replacement, sort the drawn elements, and redraw the whole sample if
// two are equal or the smallest is min(D) (the smallest column head).

template <int DT, int T, int R, bool WARP>
__global__ void __launch_bounds__(WARP ? 256 : T) k_pivots(Ctx c, u32 ready_count, u32 pmin, u32 pmax) {
  typedef KT<DT> K;
  typedef Sorter<K, T, R, WARP> S;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *smem = reinterpret_cast<E *>(smem_raw);
  constexpr int groups = WARP ? 8 : 1;
  const int g = WARP ? (threadIdx.x >> 5) : 0;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const u32 ri = blockIdx.x * groups + g;
  if (ri >= ready_count) return;
  const u32 id = c.ready_cur[ri];
  Node *nd = &c.nodes[id];
  const u32 np = nd->k - 1;  // pivots to draw
  if (np <= pmin || np > pmax) return;
  if (nd->meta + meta_layout(nd->k, nd->cols, nd->ncb, nd->nkb, K::key_words).total > c.meta_cap) return;
  const Inst I = c.inst[nd->inst];
  const key_t *dk = (const key_t *)I.dkeys + nd->off;
  const u32 *dv = I.dvals + nd->off;
  const u64 n = nd->n;
  E *s = smem + g * S::SMEM;

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
      return;
    }
    S::sync();
  }
  if (tid == 0) atomicOr(&c.status->error, ERRB_ATTEMPTS);
}

// ----------------------------------------------------------------- count ---
// One pass over the sorted columns of a block of kCountCols columns: each
// thread takes a contiguous chunk, finds the bucket of its first element by
// binary search over the pivots and walks the rest.  Produces the block's
// per-bucket totals T[I][j] and, per column, the start P[Jb][i] of every
// kSkewBkts-bucket segment.

template <int DT>
__global__ void __launch_bounds__(1024) k_count(Ctx c, u32 ready_count, u32 kmax) {
  typedef KT<DT> K;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *piv = reinterpret_cast<E *>(smem_raw);
  u32 *hist = reinterpret_cast<u32 *>(piv + (kmax > 1 ? kmax - 1 : 1));
  int *lastb = reinterpret_cast<int *>(hist + kmax);
  __shared__ u32 s_u, s_ri;
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  u32 cur = kNone;
  for (;;) {
    if (tid == 0) {
      const u32 u = atomicAdd(&c.status->cur_count, 1u);
      s_u = u;
      if (u < c.status->units) s_ri = find_owner<0>(c, ready_count, u);
    }
    __syncthreads();
    const u32 u = s_u;
    if (u >= c.status->units) break;
    const u32 id = c.ready_cur[s_ri];
    const Node nd = c.nodes[id];
    const int np = (int)nd.k - 1;
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, K::key_words);
    u32 *meta = c.meta + nd.meta;
    if (id != cur) {
      const key_t *pk = reinterpret_cast<const key_t *>(meta + ML.pk);
      for (int j = tid; j < np; j += NT) piv[j] = K::make(pk[j], meta[ML.pv + j]);
      cur = id;
    }
    for (u32 j = tid; j < nd.k; j += NT) hist[j] = 0;
    __syncthreads();
    const Inst I = c.inst[nd.inst];
    const key_t *dk = (const key_t *)I.dkeys + nd.off;
    const u32 *dv = I.dvals + nd.off;
    u32 *P = meta + ML.P;
    const u32 Iblk = u - nd.unit_base;
    const u32 i0 = Iblk * kCountCols;
    const u32 i1 = min(nd.cols, i0 + kCountCols);
    const u32 q0 = (u32)min((u64)i0 * nd.rows, (u64)nd.n);
    const u32 q1 = (u32)min((u64)i1 * nd.rows, (u64)nd.n);
    const u32 S = q1 - q0;
    const u32 chunk = (S + NT - 1) / NT;
    const u32 a = q0 + min(S, (u32)tid * chunk);
    const u32 b = q0 + min(S, (u32)tid * chunk + chunk);
    int bprev = -1, firstb = -1, runb = -1;
    u32 run = 0;
    if (a < b) {
      u32 i = a / nd.rows;
      u32 pos = a - i * nd.rows;
      u32 len = min(nd.rows, nd.n - i * nd.rows);
      for (u32 p = a; p < b; p++) {
        const E e = K::make(dk[p], dv[p]);
        int bk;
        if (p == a || pos == 0) {
          bk = upper_bound_e<K>(piv, 0, np, e);
        } else {
          bk = bprev;
          const int lim = min(np, bk + 8);
          while (bk < lim && !K::lt(e, piv[bk])) ++bk;
          if (bk == lim && bk < np && !K::lt(e, piv[bk])) bk = upper_bound_e<K>(piv, bk, np, e);
        }
        if (p == a) firstb = bk;
        if (bk == runb) {
          ++run;
        } else {
          if (run) atomicAdd(&hist[runb], run);
          runb = bk;
          run = 1;
        }
        if (p != a || pos == 0) {
          const int pb = pos == 0 ? -1 : bprev;
          for (int Jb = (pb + kSkewBkts) / kSkewBkts; Jb <= bk / kSkewBkts; ++Jb) P[(u64)Jb * nd.cols + i] = pos;
        }
        if (pos + 1 == len)
          for (u32 Jb = bk / kSkewBkts + 1; Jb < nd.nkb; ++Jb) P[(u64)Jb * nd.cols + i] = len;
        bprev = bk;
        if (++pos == len) {
          ++i;
          pos = 0;
          len = (u64)i * nd.rows < nd.n ? min(nd.rows, nd.n - i * nd.rows) : 0;
        }
      }
      if (run) atomicAdd(&hist[runb], run);
    }
    lastb[tid] = bprev;
    __syncthreads();
    if (a < b) {
      const u32 i = a / nd.rows;
      const u32 pos = a - i * nd.rows;
      if (pos != 0) {  // segment starts between the previous thread's last element and ours
        const int pb = lastb[tid - 1];
        for (int Jb = (pb + kSkewBkts) / kSkewBkts; Jb <= firstb / kSkewBkts; ++Jb)
          P[(u64)Jb * nd.cols + i] = pos;
      }
    }
    u32 *T = meta + ML.T;
    for (u32 j = tid; j < nd.k; j += NT) T[(u64)Iblk * nd.k + j] = hist[j];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ scans ---
// T[I][j] -> exclusive prefix over I (in place); b[j] <- bucket size.
// One work item = 32 buckets; 8 warps split the column blocks.

static __global__ void __launch_bounds__(256) k_scan(Ctx c, u32 ready_count, int kw) {
  __shared__ u32 part[8][32];
  __shared__ u32 s_u, s_ri;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      const u32 u = atomicAdd(&c.status->cur_scan, 1u);
      s_u = u;
      if (u < c.status->srows) s_ri = find_owner<2>(c, ready_count, u);
    }
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

// b[j] (sizes) -> bucket starts b[0..k]; one CTA per ready node.
static __global__ void __launch_bounds__(1024) k_bstart(Ctx c, u32 ready_count, int kw) {
  __shared__ u32 wt[33];
  const Node nd = c.nodes[c.ready_cur[blockIdx.x]];
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

// ------------------------------------------------------------------ skew ---
// SkewTranspose D -> A.  A tile is kSkewCols columns x kSkewBkts buckets:
// per column the segment [P[Jb][i], P[Jb+1][i]) (about kSkewBkts elements,
// one coalesced read), per bucket one contiguous run of the output (about
// kSkewCols elements, one coalesced write).  The tile's elements are taken in
// column-major order (chunks of CAP), their bucket found among the tile's
// pivots, and placed bucket-major in shared memory: within a bucket they keep
// column order and, per column, sorted order -- exactly the order in which
// Algorithm 2 (and Algorithm 3) append them.

template <int DT, int CAP>
struct SkewSmem {
  typedef typename KT<DT>::elem_t E;
  E piv[kSkewBkts];
  E in_e[CAP];
  E out_e[CAP];
  u32 base[kSkewBkts], running[kSkewBkts], tot[kSkewBkts], ob[kSkewBkts];
  u32 seg_start[kSkewCols], seg_pre[kSkewCols + 1];
  uint16_t first[kSkewCols][kSkewBkts];
  uint16_t cnt[kSkewCols][kSkewBkts];
  uint8_t in_j[CAP], in_c[CAP], out_j[CAP];
  u32 s_u, s_ri;
};

template <int DT, int CAP>
__global__ void __launch_bounds__(256) k_skew(Ctx c, u32 ready_count) {
  typedef KT<DT> K;
  typedef typename K::elem_t E;
  typedef typename K::key_t key_t;
  typedef SkewSmem<DT, CAP> SM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const int tid = threadIdx.x, NT = blockDim.x;
  for (;;) {
    if (tid == 0) {
      const u32 u = atomicAdd(&c.status->cur_skew, 1u);
      sm.s_u = u;
      if (u < c.status->tiles) sm.s_ri = find_owner<1>(c, ready_count, u);
    }
    __syncthreads();
    const u32 u = sm.s_u;
    if (u >= c.status->tiles) break;
    const Node nd = c.nodes[c.ready_cur[sm.s_ri]];
    const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, K::key_words);
    const u32 *meta = c.meta + nd.meta;
    const u32 tile = u - nd.tile_base;
    const u32 Is = tile / nd.nkb, Jb = tile - Is * nd.nkb;
    const u32 j0 = Jb * kSkewBkts, nk = min((u32)kSkewBkts, nd.k - j0);
    const u32 i0 = Is * kSkewCols, nc = min((u32)kSkewCols, nd.cols - i0);
    const Inst I = c.inst[nd.inst];
    const key_t *dk = (const key_t *)I.dkeys + nd.off;
    const u32 *dv = I.dvals + nd.off;
    key_t *ak = (key_t *)I.keys + nd.off;
    u32 *av = I.vals + nd.off;
    const key_t *pk = reinterpret_cast<const key_t *>(meta + ML.pk);
    const u32 *P = meta + ML.P;
    const u32 *G = meta + ML.T;
    const u32 *b = meta + ML.b;
    if (tid + 1 < (int)nk) sm.piv[tid] = K::make(pk[j0 + tid], meta[ML.pv + j0 + tid]);
    if (tid < (int)nk) {
      sm.base[tid] = b[j0 + tid] + G[(u64)(Is * (kSkewCols / kCountCols)) * nd.k + j0 + tid];
      sm.running[tid] = 0;
    }
    if (tid < (int)nc) {
      const u32 i = i0 + tid;
      const u64 cs = (u64)i * nd.rows;
      const u32 len = cs < nd.n ? (u32)min((u64)nd.rows, nd.n - cs) : 0;
      u32 s0 = 0, s1 = 0;
      if (len) {
        s0 = P[(u64)Jb * nd.cols + i];
        s1 = Jb + 1 < nd.nkb ? P[(u64)(Jb + 1) * nd.cols + i] : len;
      }
      sm.seg_start[tid] = (u32)cs + s0;
      sm.seg_pre[tid + 1] = s1 - s0;  // lengths; prefix below
    }
    __syncthreads();
    if (tid == 0) {
      sm.seg_pre[0] = 0;
      for (u32 q = 1; q <= nc; q++) sm.seg_pre[q] += sm.seg_pre[q - 1];
    }
    __syncthreads();
    const u32 S = sm.seg_pre[nc];
    for (u32 cs = 0; cs < S; cs += CAP) {
      const u32 L = min((u32)CAP, S - cs);
      for (u32 q = tid; q < nc * kSkewBkts; q += NT) (&sm.cnt[0][0])[q] = 0;
      for (u32 ql = tid; ql < L; ql += NT) {
        const u32 q = cs + ql;
        u32 lo = 0, hi = nc;  // last column with seg_pre <= q
        while (hi - lo > 1) {
          const u32 mid = (lo + hi) >> 1;
          if (sm.seg_pre[mid] <= q)
            lo = mid;
          else
            hi = mid;
        }
        const u32 p = sm.seg_start[lo] + (q - sm.seg_pre[lo]);
        const E e = K::make(dk[p], dv[p]);
        sm.in_e[ql] = e;
        sm.in_j[ql] = (uint8_t)upper_bound_e<K>(sm.piv, 0, (int)nk - 1, e);
        sm.in_c[ql] = (uint8_t)lo;
      }
      __syncthreads();
      for (u32 ql = tid; ql < L; ql += NT) {
        const uint8_t jl = sm.in_j[ql], ci = sm.in_c[ql];
        if (ql == 0 || sm.in_c[ql - 1] != ci || sm.in_j[ql - 1] != jl) sm.first[ci][jl] = (uint16_t)ql;
      }
      __syncthreads();
      for (u32 ql = tid; ql < L; ql += NT) {
        const uint8_t jl = sm.in_j[ql], ci = sm.in_c[ql];
        if (ql + 1 == L || sm.in_c[ql + 1] != ci || sm.in_j[ql + 1] != jl)
          sm.cnt[ci][jl] = (uint16_t)(ql - sm.first[ci][jl] + 1);
      }
      __syncthreads();
      if (tid < (int)nk) {
        u32 acc = 0;
        for (u32 ci = 0; ci < nc; ci++) {
          const u32 t = sm.cnt[ci][tid];
          sm.cnt[ci][tid] = (uint16_t)acc;
          acc += t;
        }
        sm.tot[tid] = acc;
      }
      __syncthreads();
      if (tid == 0) {
        u32 acc = 0;
        for (u32 jl = 0; jl < nk; jl++) {
          sm.ob[jl] = acc;
          acc += sm.tot[jl];
        }
      }
      __syncthreads();
      for (u32 ql = tid; ql < L; ql += NT) {
        const uint8_t jl = sm.in_j[ql], ci = sm.in_c[ql];
        const u32 slot = sm.ob[jl] + sm.cnt[ci][jl] + (ql - sm.first[ci][jl]);
        sm.out_e[slot] = sm.in_e[ql];
        sm.out_j[slot] = jl;
      }
      __syncthreads();
      for (u32 s = tid; s < L; s += NT) {
        const uint8_t jl = sm.out_j[s];
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
      if (tid < (int)nk) sm.running[tid] += sm.tot[tid];
      __syncthreads();
    }
  }
}

// --------------------------------------------------------------- spawning ---
// Children are appended block-cooperatively: one global atomic per leaf class
// (and one for new nodes) per batch of blockDim.x children.

struct Child {
  u64 off;
  u64 hash;
  u32 n, inst, parent, kind, index, depth, out;
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
    cls = ch.n <= c.cutoff ? class_of(ch.n, nclass) : kLeafClasses;
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
        L.flags = ch.kind | (ch.out << 8);
        c.leaves_nxt[cls][idx] = L;
      } else {
        atomicOr(&c.status->error, ERRB_LIST);
      }
    } else {
      const u32 id = cbase[kLeafClasses] + local;
      const u32 fi = fbase + local;
      if (id < c.node_cap && fi < c.fresh_cap) {
        Node nn;
        const u32 m = isqrt_ceil(ch.n);
        nn.off = ch.off;
        nn.hash = ch.hash;
        nn.meta = 0;
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
        nn.pad = 0;
        c.nodes[id] = nn;
        fresh_list[fi] = id;
      } else {
        atomicOr(&c.status->error, ERRB_NODES);
      }
    }
  }
  __syncthreads();
}

// Bucket children of every ready node (Algorithm 1's last loop).
template <int DT>
__global__ void __launch_bounds__(256) k_expand_buckets(Ctx c, u32 ready_count) {
  __shared__ u32 wt[33];
  const u32 id = c.ready_cur[blockIdx.x];
  const Node nd = c.nodes[id];
  const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, KT<DT>::key_words);
  const u32 *b = c.meta + nd.meta + ML.b;
  u32 nonempty = 0;
  for (u32 j = threadIdx.x; j < nd.k; j += blockDim.x) nonempty += b[j + 1] > b[j];
  u32 tot;
  block_excl_scan_u32(nonempty, wt, tot);
  if (threadIdx.x == 0) c.nodes[id].pending = (int)tot;
  __syncthreads();
  for (u32 base = 0; base < nd.k; base += blockDim.x) {
    const u32 j = base + threadIdx.x;
    Child ch;
    bool has = false;
    if (j < nd.k) {
      ch.n = b[j + 1] - b[j];
      has = ch.n > 0;
      ch.off = nd.off + b[j];
      ch.hash = buc_hash(nd.hash, j);
      ch.inst = nd.inst;
      ch.parent = id;
      ch.kind = KIND_BUC;
      ch.index = j;
      ch.depth = nd.depth + 1;
      ch.out = nd.out;
    }
    spawn_batch(c, has, ch, c.fresh_cur, &c.cnt_cur->fresh, LeafCfg<DT>::nclass);
  }
}

// Column children of every new node (Algorithm 1's first loop); new internal
// column nodes are expanded in the next round.
template <int DT>
__global__ void __launch_bounds__(256) k_expand_cols(Ctx c) {
  __shared__ u32 s_u;
  for (;;) {
    if (threadIdx.x == 0) s_u = atomicAdd(&c.status->cur_expand, 1u);
    __syncthreads();
    const u32 u = s_u;
    if (u >= min(c.cnt_cur->fresh, c.fresh_cap)) break;
    const u32 id = c.fresh_cur[u];
    const Node nd = c.nodes[id];
    const u32 ncol = (u32)(((u64)nd.n + nd.rows - 1) / nd.rows);  // non-empty columns
    if (threadIdx.x == 0) c.nodes[id].pending = (int)ncol;
    for (u32 base = 0; base < ncol; base += blockDim.x) {
      const u32 i = base + threadIdx.x;
      Child ch;
      const bool has = i < ncol;
      if (has) {
        const u64 st = (u64)i * nd.rows;
        ch.n = (u32)min((u64)nd.rows, (u64)nd.n - st);
        ch.off = nd.off + st;
        ch.hash = col_hash(nd.hash, i);
        ch.inst = nd.inst;
        ch.parent = id;
        ch.kind = KIND_COL;
        ch.index = i;
        ch.depth = nd.depth + 1;
        ch.out = 1;  // columns are sorted from A into D
      }
      spawn_batch(c, has, ch, c.fresh_nxt, &c.cnt_nxt->fresh, LeafCfg<DT>::nclass);
    }
    __syncthreads();
  }
}

// ------------------------------------------------ stand-alone SkewTranspose ---

// Caller-supplied pivots -> the node's metadata.
template <int DT>
__global__ void k_put_pivots(Ctx c, const typename KT<DT>::key_t *pk, const u32 *pv) {
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
__global__ void k_get_bstart(Ctx c, u64 *out) {
  const Node &nd = c.nodes[c.ready_cur[0]];
  const MetaLayout ML = meta_layout(nd.k, nd.cols, nd.ncb, nd.nkb, KT<DT>::key_words);
  const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j <= nd.k) out[j] = c.meta[nd.meta + ML.b + j];
}

}  // namespace sq
