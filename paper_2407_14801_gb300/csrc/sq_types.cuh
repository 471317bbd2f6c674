// Element order, random source and shared data structures of the SquareSort
// engine (device and host).  Nothing here is shared with the CPU oracle.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sq {

typedef unsigned long long u64;
typedef uint32_t u32;

enum : int { DT_U32 = 0, DT_U64 = 1, DT_F32 = 2, DT_F32W = 3 };
// DT_F32W: float32 keys held as one 64-bit compare word in the leaf sorts
// (exact for every key but NaN; the leaf kernels restore NaN bits).

// Status bits latched by kernels in Status::error.
enum : u32 {
  ERRB_ATTEMPTS = 1u,  // pivot sampling exhausted kMaxAttempts
  ERRB_NODES = 2u,     // node pool full
  ERRB_LIST = 4u,      // a work list full
  ERRB_ARENA = 8u,     // per-round metadata arena full
  ERRB_SIZES = 16u,    // bucket sizes do not add up (internal error)
  ERRB_TRACE = 32u,    // trace buffer full (records dropped)
  ERRB_SAMP = 64u,     // appendix-variant sample store full
};

constexpr u32 kNone = 0xffffffffu;
constexpr int kMaxAttempts = 256;  // pivot samples per node before giving up
constexpr int kLeafClasses = 11;
constexpr uint32_t kRadixClassesAll = 0x7FCu;  // leaf classes 2..10 (512..64K elements) have radix kernels

// Child kinds (Algorithm 1): the root, a column sort, a bucket sort.
enum : u32 { KIND_ROOT = 0, KIND_COL = 1, KIND_BUC = 2 };

// ------------------------------------------------------------ key order ----
// Elements are (key, val) pairs ordered by (ordinal(key), val).  ordinal is
// the identity for uint32/uint64; for float32 bit patterns it is IEEE order
// with -0 < +0 and every NaN above +inf, all NaNs equal.

__host__ __device__ __forceinline__ u32 f32_ordinal(u32 b) {
  if ((b & 0x7fffffffu) > 0x7f800000u) return 0xffffffffu;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Inverse of f32_ordinal on non-NaN keys (a NaN maps to 0x7fffffff).
__host__ __device__ __forceinline__ u32 f32_from_ordinal(u32 o) { return (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o; }

// Three-word element: 64-bit compare word plus a 32-bit word.
struct __align__(16) E3 {
  u64 k;
  u32 x;
  u32 pad;
};

template <int DT>
struct KT;

// uint32 keys: one 64-bit word (key << 32 | val), compared as an integer.
template <>
struct KT<DT_U32> {
  typedef u32 key_t;
  typedef u64 elem_t;
  typedef u32 ord_t;
  static constexpr int key_words = 1;
  static constexpr bool lossy = false;
  static constexpr bool top_is_value = true;  // top() is bit-identical to any element equal to it
  // Loaded by asynchronous copies: the key's and the val's bytes land at
  // these offsets of the element, which raw() then completes in place.
  static constexpr bool async_load = true;
  static constexpr int key_off = 4, val_off = 0;  // (little-endian: key << 32 | val)
  __device__ __forceinline__ static elem_t raw(elem_t e) { return e; }
  __device__ __forceinline__ static bool exact(key_t) { return true; }
  __device__ __forceinline__ static ord_t ord_key(key_t k) { return k; }
  __device__ __forceinline__ static key_t pad_key() { return 0xffffffffu; }
  __device__ __forceinline__ static elem_t make(key_t k, u32 v) { return ((u64)k << 32) | v; }
  __device__ __forceinline__ static key_t key(elem_t e) { return (u32)(e >> 32); }
  __device__ __forceinline__ static u32 val(elem_t e) { return (u32)e; }
  __device__ __forceinline__ static bool lt(elem_t a, elem_t b) { return a < b; }
  __device__ __forceinline__ static bool eq(elem_t a, elem_t b) { return a == b; }
  __device__ __forceinline__ static elem_t top() { return ~0ull; }
};

// float32 keys: compare word (ordinal << 32 | val); the raw bits ride along.
template <>
struct KT<DT_F32> {
  typedef u32 key_t;
  typedef E3 elem_t;
  typedef u32 ord_t;
  static constexpr int key_words = 1;
  static constexpr bool lossy = false;
  static constexpr bool top_is_value = false;  // an element may equal top() in order but carry other key bits
  static constexpr bool async_load = false;
  static constexpr int key_off = 0, val_off = 0;
  __device__ __forceinline__ static elem_t raw(elem_t e) { return e; }
  __device__ __forceinline__ static bool exact(key_t) { return true; }
  __device__ __forceinline__ static ord_t ord_key(key_t k) { return f32_ordinal(k); }
  __device__ __forceinline__ static key_t pad_key() { return 0xffffffffu; }  // a NaN: ordinal max
  __device__ __forceinline__ static elem_t make(key_t k, u32 v) {
    E3 e;
    e.k = ((u64)f32_ordinal(k) << 32) | v;
    e.x = k;
    e.pad = 0;
    return e;
  }
  __device__ __forceinline__ static key_t key(elem_t e) { return e.x; }
  __device__ __forceinline__ static u32 val(elem_t e) { return (u32)e.k; }
  __device__ __forceinline__ static bool lt(elem_t a, elem_t b) { return a.k < b.k; }
  __device__ __forceinline__ static bool eq(elem_t a, elem_t b) { return a.k == b.k; }
  __device__ __forceinline__ static elem_t top() {
    E3 e;
    e.k = ~0ull;
    e.x = 0xffffffffu;
    e.pad = 0;
    return e;
  }
};

// float32 keys in leaf sorts: the compare word alone, key bits recovered
// from the ordinal.  NaN keys are not recovered (every NaN has one
// ordinal): `lossy` tells the leaf kernels to record and restore them.
template <>
struct KT<DT_F32W> {
  typedef u32 key_t;
  typedef u64 elem_t;
  typedef u32 ord_t;
  static constexpr int key_words = 1;
  static constexpr bool lossy = true;
  static constexpr bool top_is_value = true;  // top() is bit-identical to any element equal to it
  static constexpr bool async_load = true;    // the key's bits, then raw() makes them the ordinal
  static constexpr int key_off = 4, val_off = 0;
  __device__ __forceinline__ static elem_t raw(elem_t e) {
    return ((u64)f32_ordinal((u32)(e >> 32)) << 32) | (u32)e;  // (top() stays top())
  }
  __device__ __forceinline__ static bool exact(key_t k) { return (k & 0x7fffffffu) <= 0x7f800000u; }
  __device__ __forceinline__ static ord_t ord_key(key_t k) { return f32_ordinal(k); }
  __device__ __forceinline__ static key_t pad_key() { return 0xffffffffu; }
  __device__ __forceinline__ static elem_t make(key_t k, u32 v) { return ((u64)f32_ordinal(k) << 32) | v; }
  __device__ __forceinline__ static key_t key(elem_t e) { return f32_from_ordinal((u32)(e >> 32)); }
  __device__ __forceinline__ static u32 val(elem_t e) { return (u32)e; }
  __device__ __forceinline__ static bool lt(elem_t a, elem_t b) { return a < b; }
  __device__ __forceinline__ static bool eq(elem_t a, elem_t b) { return a == b; }
  __device__ __forceinline__ static elem_t top() { return ~0ull; }
};

// uint64 keys: (key, val) compared lexicographically.
template <>
struct KT<DT_U64> {
  typedef u64 key_t;
  typedef E3 elem_t;
  typedef u64 ord_t;
  static constexpr int key_words = 2;
  static constexpr bool lossy = false;
  static constexpr bool top_is_value = true;  // top() is bit-identical to any element equal to it
  static constexpr bool async_load = true;    // (pad is left as it is: no comparison reads it)
  static constexpr int key_off = 0, val_off = 8;
  __device__ __forceinline__ static elem_t raw(elem_t e) { return e; }
  __device__ __forceinline__ static bool exact(key_t) { return true; }
  __device__ __forceinline__ static ord_t ord_key(key_t k) { return k; }
  __device__ __forceinline__ static key_t pad_key() { return ~0ull; }
  __device__ __forceinline__ static elem_t make(key_t k, u32 v) {
    E3 e;
    e.k = k;
    e.x = v;
    e.pad = 0;
    return e;
  }
  __device__ __forceinline__ static key_t key(elem_t e) { return e.k; }
  __device__ __forceinline__ static u32 val(elem_t e) { return e.x; }
  __device__ __forceinline__ static bool lt(elem_t a, elem_t b) {
    return a.k < b.k || (a.k == b.k && a.x < b.x);
  }
  __device__ __forceinline__ static bool eq(elem_t a, elem_t b) { return a.k == b.k && a.x == b.x; }
  __device__ __forceinline__ static elem_t top() {
    E3 e;
    e.k = ~0ull;
    e.x = 0xffffffffu;
    e.pad = 0;
    return e;
  }
};

// --------------------------------------------------------- random source ----
// Counter-based SplitMix64 (Steele, Lea & Flood 2014): every node's pivots
// are a pure function of (seed, path from the root, attempt).
//   root hash      F(seed)
//   column child i F(h + gamma*(2i+1)),  bucket child j F(h + gamma*(2j+2))
//   attempt a      s_a = F(h ^ (0xd1b54a32d192ed03 * (a+1)))
//   draw r         F(s_a + gamma*(r+1)); position floor(draw * n / 2^64)

constexpr u64 kGamma = 0x9e3779b97f4a7c15ull;

__host__ __device__ __forceinline__ u64 mix64(u64 z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}
__host__ __device__ __forceinline__ u64 root_hash(u64 seed) { return mix64(seed); }
__host__ __device__ __forceinline__ u64 col_hash(u64 h, u64 i) { return mix64(h + kGamma * (2 * i + 1)); }
__host__ __device__ __forceinline__ u64 buc_hash(u64 h, u64 j) { return mix64(h + kGamma * (2 * j + 2)); }
__host__ __device__ __forceinline__ u64 attempt_seed(u64 h, u64 a) {
  return mix64(h ^ (0xd1b54a32d192ed03ull * (a + 1)));
}
__host__ __device__ __forceinline__ u64 draw(u64 s, u64 r) { return mix64(s + kGamma * (r + 1)); }

// Smallest m with m*m >= n (n < 2^53).
__host__ __device__ __forceinline__ u32 isqrt_ceil(u64 n) {
  if (n == 0) return 0;
  u64 m = (u64)sqrt((double)n);
  while (m * m < n) ++m;
  while (m > 1 && (m - 1) * (m - 1) >= n) --m;
  return (u32)m;
}

// Largest m with m*m <= n.
__host__ __device__ __forceinline__ u32 isqrt_floor(u64 n) {
  const u32 m = isqrt_ceil(n);
  return (u64)m * m > n ? m - 1 : m;
}

// The recursion a sort follows: Algorithm 1, or the variant of the paper's
// appendix listing (floor(sqrt n) columns, the last one running to n;
// pivots sampled from the node's input; buckets bounded above by "<=").
enum : u32 { VAR_ALG1 = 0, VAR_APPENDIX = 1 };

// Columns of a node (geometry rows x cols over n elements): column i spans
// [col_begin, col_end); the last column runs to n -- short or empty under
// Algorithm 1 (ceil(sqrt n) columns), the longest under the appendix variant.
__host__ __device__ __forceinline__ u64 col_begin(u64 i, u32 rows, u64 n) {
  const u64 b = i * rows;
  return b < n ? b : n;
}
__host__ __device__ __forceinline__ u64 col_end(u64 i, u32 rows, u32 cols, u64 n) {
  if (i + 1 >= cols) return n;
  const u64 e = (i + 1) * rows;
  return e < n ? e : n;
}
// m of a new node of n elements.
__host__ __device__ __forceinline__ u32 node_m(u64 n, u32 variant) {
  return variant == VAR_APPENDIX ? isqrt_floor(n) : isqrt_ceil(n);
}

// ------------------------------------------------------- work structures ----

// One sort instance: the caller's buffers (A) and the scratch copy (D).
struct Inst {
  void *keys;  // A keys
  u32 *vals;   // A vals
  void *dkeys; // D keys (scratch)
  u32 *dvals;  // D vals (scratch)
  const void *skeys;  // where the input is read (the root's columns, or the root leaf): A, or a mapped
  const u32 *svals;   //   host buffer that the first pass reads directly
  void *fkeys;        // where final leaves write: A, or a mapped host buffer that the last pass
  u32 *fvals;         //   writes directly
  uint8_t *tags;  // per element of D: its bucket within its 64-bucket block (written by the count)
  u64 n;
  u32 cutoff;   // leaf iff a node's n <= cutoff (per instance)
  u32 variant;  // VAR_ALG1 or VAR_APPENDIX
};

// A SquareSort call with n > cutoff (or a stand-alone SkewTranspose).
// Geometry: `cols` sorted columns of height `rows` (the last one short or
// empty) and `k` buckets; for SquareSort nodes rows = cols = k = ceil(sqrt n).
struct Node {
  u64 off;   // first element in the instance
  u64 hash;  // path hash
  u64 meta;  // word offset of this round's metadata in the arena
  u64 samp;  // appendix variant: word offset of the node's pivot sample in the sample store, or kNoSamp
  u32 n, rows, cols, k;
  u32 inst, parent, kind, index;
  u32 depth, out;  // out: 0 = result lands in A, 1 = in D
  int pending;     // column children, later bucket children, still running
  u32 attempts;
  u32 unit_base, tile_base, srow_base;  // this round's work numbering
  u32 ncb, nkb, ncs;                    // count blocks, bucket blocks, skew column blocks
  u32 src;  // 1: the node's input is the instance's source (the root, and column children of such nodes)
};

constexpr u64 kNoSamp = ~0ull;  // the sample is read from the node's input at its pivot step

// A leaf: sorted in one group of threads (n <= cutoff).
struct Leaf {
  u64 off;
  u32 n, inst, parent, flags;  // flags: kind | out << 8 | LEAF_IN_OUT | LEAF_SRC
};
constexpr u32 LEAF_IN_OUT = 1u << 16;  // input already sits in the output buffer
constexpr u32 LEAF_SRC = 1u << 17;     // input is read from the instance's source (Inst::skeys)

// Per-parity list counters (zeroed before the round that fills them).
struct Counters {
  u32 leaves[kLeafClasses];
  u32 ready;
  u32 fresh;
  u32 max_ready_k;
  u64 leaf_elems[kLeafClasses];  // elements in each leaf list (for byte counts)
  u64 ready_elems;
};

// Global engine status, read back after every round.
struct Status {
  u32 error;
  u32 done;
  u32 nodes_used;
  u32 trace_used;
  // per-round work totals written by the plan step
  u32 units, tiles, srows, echunks;
  u64 meta_words;
  u64 samp_used;  // words of the appendix-variant sample store handed out
  // persistent-kernel work cursors (zeroed every round, with fix_count and
  // the leaf cursors of graph-launched rounds)
  u32 cur_count, cur_scan, cur_skew, cur_expand, cur_ebkt, cur_fix, fix_count;
  u32 cur_leaf[kLeafClasses];
  u32 runs_count, runs_cursor;  // this round's run copies (RunCopy list)
  u32 cur_count_big;             // the count's units of nodes whose pivots stay in global memory
};
constexpr int kRoundCursors = 7 + kLeafClasses + 3;  // Status words from cur_count on, zeroed every round

// One column's piece of a run of one bucket tag in a big SkewTranspose tile:
// n elements from D at src to A at dst (element offsets in the instance).
struct RunCopy {
  u64 src, dst;
  u32 n, inst;
};

// A trace record, one per recursing node (written when its pivots are chosen).
struct TraceRec {
  u64 off, n, m, hash;
  u32 depth, kind, attempts, index;
};

// A launch's item count that the kernel reads from the round's counters
// (graph-launched rounds, whose launches do not change from run to run).
constexpr u32 kDev = 0xffffffffu;

// Tile geometry (count blocks, skew tiles).
constexpr int kCountCols = 16;  // columns per count unit (block-total granularity)
constexpr int kSkewCols = 32;   // columns per skew tile (multiple of kCountCols)
constexpr int kSkewBkts = 64;   // buckets per skew tile / P-table granularity
constexpr int kExpandChunk = 256;  // bucket children spawned per work item

// Everything a kernel needs, passed by value.
struct Ctx {
  Inst *inst;
  Node *nodes;
  u32 node_cap;
  // lists, current parity (read) and next parity (write)
  Leaf *leaves_cur[kLeafClasses];
  Leaf *leaves_nxt[kLeafClasses];
  u32 leaf_cap[kLeafClasses];
  u32 *ready_cur, *ready_nxt;
  u32 ready_cap;
  u32 *fresh_cur, *fresh_nxt;
  u32 fresh_cap;
  u32 *wbase;  // per ready node, in list order: first count unit, tile, scan row, bucket chunk (4 x ready_cap)
  Counters *cnt_cur, *cnt_nxt;
  Status *status;
  u32 *meta;  // this round's arena (words)
  u64 meta_cap;
  u32 *done_list;  // instance ids in completion order
  TraceRec *trace;
  u32 trace_cap;
  u32 cutoff;
  Leaf *fix;    // leaves whose radix result failed the (key, val) check this round
  u32 fix_cap;
  u32 class_cap[kLeafClasses];  // max elements per leaf class
  int recurse;                  // 0 for a stand-alone SkewTranspose
  u32 ninst;                    // instances of the run
  RunCopy *runs;                // run copies the SkewTranspose hands to k_copy_runs
  u32 runs_cap;
  u32 *samp;                    // appendix variant: pivot samples of nodes whose columns recurse
  u64 samp_cap;                 // (words)
};

// Metadata layout of a ready node (32-bit words from Node::meta), each
// section 4-word aligned: pivot keys (k-1, kw words each), pivot vals (k-1),
// T[j][I] block totals -> exclusive prefixes (k * ncb), P[Jb][i] segment
// starts (nkb * cols), bucket starts b[0..k] (k+1).
struct MetaLayout {
  u64 pk, pv, T, P, b, pe, total;
};

// Pivots that the count keeps in shared memory (with its k bucket totals):
// larger nodes keep them, as whole elements, in their metadata (section pe)
// and the count reads them from there.
constexpr u32 kCountSmemPivots = 16384;

__host__ __device__ __forceinline__ u64 align4(u64 x) { return (x + 3) & ~3ull; }

__host__ __device__ __forceinline__ MetaLayout meta_layout(u32 k, u32 cols, u32 ncb, u32 nkb, int kw) {
  MetaLayout L;
  u64 p = 0;
  L.pk = p;
  p += align4((u64)(k - 1) * kw);
  L.pv = p;
  p += align4(k - 1);
  L.T = p;
  p += align4((u64)k * ncb);
  L.P = p;
  p += align4((u64)nkb * cols);
  L.b = p;
  p += align4((u64)k + 1);
  L.pe = p;
  if (k - 1 > kCountSmemPivots) p += align4((u64)(k - 1) * 4);  // (room for 16-byte elements)
  L.total = p;
  return L;
}

}  // namespace sq
