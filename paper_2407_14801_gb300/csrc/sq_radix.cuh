// Radix base case for one CTA: a stable least-significant-digit radix sort
// of a leaf by its key ordinal, used as Algorithm 1's simple_sort for keys
// whose ordinal is 32 bits wide (uint32, and float32 through its one-word
// compare element).
//
// Why the key alone suffices (usually): a leaf's elements must end in
// (ordinal(key), val) order.  A stable sort by key leaves equal keys in
// their input order, which is that order whenever equal keys already appear
// with ascending vals.  That holds at every node of the recursion when the
// payload is the original index: it holds for the input, a column or bucket
// is a contiguous range of its parent, the column sorts order equal keys by
// val, and the SkewTranspose is a stable partition that takes column i's
// elements of a bucket before column i+1's (whose equal keys have larger
// vals).  It is not assumed: the sorted leaf is checked for strictly
// ascending (ordinal, val) words, and the caller merge sorts the leaf when
// the check fails.  The result is therefore always the unique sorted
// permutation, bit for bit the merge sort's.
//
// Each pass orders the elements by one BITS-bit digit of (ordinal - min):
// every thread counts its R elements' digits in private 16-bit counters in
// shared memory (counter (digit d, thread t) at d*T + t), one exclusive scan
// over (digit, thread) turns the counts into the first output slot of each
// thread's elements of each digit, and the elements are scattered to their
// slots and read back in the blocked layout (thread t holds positions
// [t*R, t*R + R)).  The counts are read and bumped G elements at a time
// (duplicates within a group fixed up in registers) to shorten the chain of
// dependent shared-memory accesses.  The number of passes follows the key
// range of the leaf: ceil(log2(max - min + 1) / BITS).
#pragma once
#include "sq_sorter.cuh"

namespace sq {

template <class K, int T, int R, int BITS = 5, int G = 2>
struct RadixLeaf {
  typedef Sorter<K, T, R, false> S;
  typedef typename K::elem_t E;
  static_assert(sizeof(E) == 8 && K::top_is_value, "one 64-bit compare word: ordinal << 32 | val");
  static_assert(R % G == 0 && T % 32 == 0 && T <= 1024, "groups of G; whole warps");
  static constexpr int D = 1 << BITS;                 // digit values
  static constexpr int NCNT = D * T;                  // 16-bit counters
  static constexpr int CWORDS = NCNT / 2 + NCNT / 32; // one pad word per 16 words (the scan's rows)
  static constexpr int RED = 128;                     // min/max and scan scratch words
  static constexpr size_t kBytes = 4 * ((size_t)CWORDS + RED);
  static_assert(CWORDS % 4 == 0, "counters are zeroed 16 bytes at a time");
  static_assert((size_t)T * R < 65536, "slots fit the 16-bit counters");

  static_assert(D >= 32, "a thread's scan row spans whole 16-word groups");
  // Counter idx = d*T + t is 16-bit half (idx & 1) of word cw(idx); with T a
  // multiple of 32 its 16-bit slot is d * kStride + (t + 2 * (t >> 5)).
  __device__ __forceinline__ static int cw(int idx) { return (idx >> 1) + (idx >> 5); }
  static constexpr int kStride = T + T / 16;
  __device__ __forceinline__ static int tslot(int t) { return t + 2 * (t >> 5); }
  // Word i of thread j's scan row (counters [D*j, D*j + D)): cw(D*j) + i + i/16.
  __device__ __forceinline__ static int row_word(int base, int i) { return base + i + (i >> 4); }
  __device__ __forceinline__ static u32 hi(E e) { return (u32)(e >> 32); }

  // c[i] = count of digit d[i] before element i; the counters are bumped
  // past the group (the last write to a counter is the group's final count).
  __device__ __forceinline__ static void bump(uint16_t *c16, const int (&a)[G], const u32 (&d)[G], u32 (&c)[G]) {
#pragma unroll
    for (int i = 0; i < G; i++) c[i] = c16[a[i]];
#pragma unroll
    for (int i = 1; i < G; i++)
#pragma unroll
      for (int j = 0; j < i; j++) c[i] += d[i] == d[j] ? 1u : 0u;
#pragma unroll
    for (int i = 0; i < G; i++) c16[a[i]] = (uint16_t)(c[i] + 1u);
  }

  // x: the thread's R elements, blocked, as Sorter::load leaves them (all
  // of the leaf also in s, positions >= n holding top()); ws: kBytes of
  // shared memory.  On return x holds the leaf sorted by ordinal (stable),
  // positions >= n top() again.  Returns true when that order is strictly
  // ascending in (ordinal, val) -- the leaf's exact order; false leaves a
  // permutation of the leaf in x for the caller's merge sort.  Ends with a
  // barrier after every read of s.
  __device__ static bool sort(E (&x)[R], E *s, int tid, u32 n, u32 *ws) {
    u32 *cnt = ws;
    uint16_t *c16 = reinterpret_cast<uint16_t *>(cnt);
    u32 *red = ws + CWORDS;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int W = T / 32;
    const int ts = tslot(tid), row = cw(D * tid);
    u32 kmin = 0xffffffffu, kmax = 0;
#pragma unroll
    for (int q = 0; q < R; q++)
      if ((u32)(tid * R + q) < n) {
        kmin = min(kmin, hi(x[q]));
        kmax = max(kmax, hi(x[q]));
      }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if (lane == 0) {
      red[warp] = kmin;
      red[32 + warp] = kmax;
    }
    __syncthreads();
    kmin = __reduce_min_sync(0xffffffffu, lane < W ? red[lane] : 0xffffffffu);
    kmax = __reduce_max_sync(0xffffffffu, lane < W ? red[32 + lane] : 0u);
    const u32 range = n ? kmax - kmin : 0u;
    const int passes = range ? (32 - __clz((int)range) + BITS - 1) / BITS : 0;
    // ordinals as offsets from the minimum; padding takes the largest offset
    // (it follows every real element of that offset: it comes last in input order)
#pragma unroll
    for (int q = 0; q < R; q++) {
      const u32 o = (u32)(tid * R + q) < n ? hi(x[q]) - kmin : range;
      x[q] = ((u64)o << 32) | (u32)x[q];
    }
#pragma unroll 1
    for (int pass = 0; pass < passes; pass++) {
      const int sh = pass * BITS;
      for (int w = tid; w < CWORDS / 4; w += T) reinterpret_cast<uint4 *>(cnt)[w] = make_uint4(0, 0, 0, 0);
      __syncthreads();
#pragma unroll
      for (int q0 = 0; q0 < R; q0 += G) {
        int a[G];
        u32 d[G], c[G];
#pragma unroll
        for (int i = 0; i < G; i++) {
          d[i] = (hi(x[q0 + i]) >> sh) & (D - 1);
          a[i] = (int)d[i] * kStride + ts;
        }
        bump(c16, a, d, c);
      }
      __syncthreads();
      {  // exclusive scan over (digit, thread): thread j owns counters [D*j, D*j + D)
        u32 sum = 0;
#pragma unroll
        for (int i = 0; i < D / 2; i++) {
          const u32 w = cnt[row_word(row, i)];
          sum += (w * 0x10001u) >> 16;  // the word's two counts (each < 2^15)
        }
        u32 incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (lane == 31) red[64 + warp] = incl;
        __syncthreads();
        if (warp == 0) {
          const u32 v = lane < W ? red[64 + lane] : 0u;
          u32 iv = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, iv, o);
            if (lane >= o) iv += t;
          }
          if (lane < W) red[64 + lane] = iv - v;
        }
        __syncthreads();
        u32 run = red[64 + warp] + incl - sum;
#pragma unroll
        for (int i = 0; i < D / 2; i++) {
          const int wa = row_word(row, i);
          const u32 w = cnt[wa];
          const u32 lo = w & 0xffffu;
          cnt[wa] = run | ((run + lo) << 16);
          run += lo + (w >> 16);
        }
      }
      __syncthreads();
#pragma unroll
      for (int q0 = 0; q0 < R; q0 += G) {  // the same walk: each count is now the element's slot
        int a[G];
        u32 d[G], c[G];
#pragma unroll
        for (int i = 0; i < G; i++) {
          d[i] = (hi(x[q0 + i]) >> sh) & (D - 1);
          a[i] = (int)d[i] * kStride + ts;
        }
        bump(c16, a, d, c);
#pragma unroll
        for (int i = 0; i < G; i++) s[S::px((int)c[i])] = x[q0 + i];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < R; q++) x[q] = s[S::px(tid * R + q)];
    }
    // strictly ascending (offset, val) words <=> the (ordinal, val) order
    bool bad = false;
#pragma unroll
    for (int q = 0; q < R; q++) {
      const u32 p = (u32)(tid * R + q);
      if (p + 1 < n) {
        const E nx = q + 1 < R ? x[q + 1] : s[S::px((int)p + 1)];
        if (!(x[q] < nx)) bad = true;
      }
    }
#pragma unroll
    for (int q = 0; q < R; q++) {
      const u32 p = (u32)(tid * R + q);
      x[q] = p < n ? (((u64)(hi(x[q]) + kmin) << 32) | (u32)x[q]) : K::top();
    }
    return !__syncthreads_or(bad);
  }
};


}  // namespace sq
