/*
 * SquareSort CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded statement of SquareSort (Koucky & Matejka,
 * "SquareSort: a cache-oblivious sorting algorithm", Section 2): Algorithm 1
 * (SquareSort), Algorithm 2 (SkewTranspose) and Algorithm 3
 * (NaiveSkewTranspose), written step by step in the paper's order and
 * notation (0-based indices here, 1-based in the paper).  It exists only to
 * check the CUDA implementation: only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant generator with the CUDA path.
 *
 * Element order.  The paper assumes distinct elements (Section 2.1).  An
 * element here is a (key, val) pair ordered by (ordinal(key), val); with
 * distinct vals (the original index in every workload) all elements are
 * distinct.  ordinal() is the identity for uint32 and uint64 keys; for float32
 * it is IEEE order with -0 < +0 and every NaN above +inf, all NaNs equal.
 *
 * Readings of the paper where it is silent or inconsistent (listed again in
 * the design notes):
 *   - the base case of Algorithm 1 returns after simple_sort;
 *   - the cutoff c is a parameter (16 in Algorithm 1, 1000 in Section 4),
 *     leaf iff n <= c, c >= 2 (n = 2 would otherwise recurse forever);
 *   - m = ceil(sqrt(n)) by exact integer arithmetic, column i spans
 *     [min(i*m, n), min((i+1)*m, n)) (Algorithm 1, column loop);
 *   - bucket j is [p_j, p_{j+1}) with p_0 = -inf, p_m = +inf (Section 2), so
 *     Algorithm 3's comparison "A[col[j]] <= pivots[i]" is read as strict <;
 *   - buc[] enters SkewTranspose as bucket starts and leaves as bucket ends
 *     (the Lemma of Section 2.2.1; Algorithm 1's "shifted by one" remark);
 *   - pivots are sampled from D after the column sorts (Algorithm 1), with
 *     replacement, and the whole sample is redrawn if two sampled elements are
 *     equal or the smallest equals min(D) (Section 2.1, pivot paragraph);
 *     min(D) is the smallest column head;
 *   - the random source is a counter-based SplitMix64 stream keyed by the
 *     node's path (defined below), so that every node's pivots are a pure
 *     function of (seed, path, attempt); the paper leaves the RNG open.
 *
 * The appendix variant (the paper's Appendix listing, which Section 2.1 says
 * departs a little from Algorithm 1), selected by sqo_sort_appendix, for
 * integer keys as in the listing:
 *   - m = floor(sqrt(n)) columns of m elements, the last one extended to n;
 *   - m pivot samples drawn with replacement from the node's input A before
 *     the column sorts (draws r = 0..m-1 of attempt 0), sorted; the largest
 *     is replaced by the greatest pair (the listing's INT_MAX: a value of the
 *     order like any other, above or equal to every element); left to right,
 *     a sample equal to the next one is replaced by its predecessor in the
 *     (key, val) order (the listing's decrement; the least pair (0, 0), which
 *     has none, stays);
 *   - bucket i = { e : pivots[i-1] < e <= pivots[i] } (the listing's "<=");
 *   - a bucket whose range holds a single (key, val) pair holds only copies
 *     of it and is copied instead of sorted: as in the listing, bucket i > 0
 *     when pivots[i-1] is the predecessor of pivots[i]; and, because the
 *     order is bounded below where the listing's int keys are not, bucket 0
 *     when pivot 0 is the least pair (without it a node made only of copies
 *     of (0, 0) would recurse on itself forever);
 *   - no redraws: one sample per node;
 *   - the cutoff is at least 8, so that every node has m >= 3 samples (with
 *     m = 2 the one pivot of a node of equal elements is that element and
 *     its bucket 0 is the whole node again; the listing's cutoff is 1000).
 *
 * Random source (Steele, Lea & Flood 2014, "Fast splittable pseudorandom
 * number generators"; output function as in Vigna's splitmix64):
 *   F(z)           = z ^= z>>30; z *= 0xbf58476d1ce4e5b9; z ^= z>>27;
 *                    z *= 0x94d049bb133111eb; z ^= z>>31
 *   gamma          = 0x9e3779b97f4a7c15
 *   root hash      = F(seed)
 *   column child i = F(h + gamma*(2i+1));   bucket child j = F(h + gamma*(2j+2))
 *   attempt seed   = s_a = F(h ^ (0xd1b54a32d192ed03 * (a+1)))
 *   draw r         = u = F(s_a + gamma*(r+1)); position t = floor(u*n / 2^64)
 * (all arithmetic mod 2^64).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SQO_U32 0
#define SQO_U64 1
#define SQO_F32 2

#define SQO_OK 0
#define SQO_ERR_INVALID 1
#define SQO_ERR_NOMEM 2
#define SQO_ERR_ATTEMPTS 7

#define SQO_MAX_ATTEMPTS 256

typedef struct {
  uint64_t key; /* raw key bits (uint32 / float32 bits zero-extended) */
  uint32_t val;
} elem;

/* One record per SquareSort call that recursed (n > cutoff). */
typedef struct {
  uint64_t off;      /* first index of the node's range in the root array */
  uint64_t n;        /* node size */
  uint64_t m;        /* ceil(sqrt(n)) */
  uint64_t hash;     /* node path hash */
  uint32_t depth;    /* root = 0 */
  uint32_t kind;     /* 0 root, 1 column child, 2 bucket child */
  uint32_t attempts; /* pivot samples drawn (1 = first sample accepted) */
  uint32_t index;    /* column or bucket index within the parent (root: 0) */
} sqo_node;

typedef struct {
  int dtype;
  uint64_t cutoff;
  int skew_mode; /* 0: Algorithm 3 only; 1: Algorithm 2, threshold 4; 2: Algorithm 2, threshold 10 */
  int status;
  sqo_node *trace;
  uint64_t trace_cap;
  uint64_t trace_count;
  elem *root_skew; /* optional copy of the root's array right after its SkewTranspose */
  int variant;     /* 0: Algorithm 1; 1: the appendix listing's variant */
} ctx;

/* ---------------------------------------------------------------- order --- */

uint64_t sqo_ordinal(int dtype, uint64_t key) {
  if (dtype == SQO_F32) {
    uint32_t b = (uint32_t)key;
    if ((b & 0x7fffffffu) > 0x7f800000u) return 0xffffffffu; /* NaN: above +inf */
    if (b & 0x80000000u) return (uint32_t)~b;                /* negative: reverse */
    return b | 0x80000000u;                                  /* positive: shift up */
  }
  if (dtype == SQO_U32) return (uint32_t)key;
  return key;
}

static int elem_less(int dtype, const elem *a, const elem *b) {
  uint64_t oa = sqo_ordinal(dtype, a->key), ob = sqo_ordinal(dtype, b->key);
  if (oa != ob) return oa < ob;
  return a->val < b->val;
}

static int elem_equal(int dtype, const elem *a, const elem *b) {
  return sqo_ordinal(dtype, a->key) == sqo_ordinal(dtype, b->key) && a->val == b->val;
}

int sqo_less(int dtype, uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
  elem a = {ka, va}, b = {kb, vb};
  return elem_less(dtype, &a, &b);
}

/* qsort comparators, one per key type (qsort has no context argument). */
static int cmp_generic(int dtype, const void *x, const void *y) {
  const elem *a = (const elem *)x, *b = (const elem *)y;
  if (elem_less(dtype, a, b)) return -1;
  if (elem_less(dtype, b, a)) return 1;
  return 0;
}
static int cmp_u32(const void *x, const void *y) { return cmp_generic(SQO_U32, x, y); }
static int cmp_u64(const void *x, const void *y) { return cmp_generic(SQO_U64, x, y); }
static int cmp_f32(const void *x, const void *y) { return cmp_generic(SQO_F32, x, y); }

static void library_sort(int dtype, elem *a, uint64_t n) {
  int (*cmp)(const void *, const void *) =
      dtype == SQO_F32 ? cmp_f32 : (dtype == SQO_U64 ? cmp_u64 : cmp_u32);
  qsort(a, (size_t)n, sizeof(elem), cmp);
}

/* --------------------------------------------------------------- random --- */

#define GAMMA 0x9e3779b97f4a7c15ull

uint64_t sqo_fmix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}

uint64_t sqo_root_hash(uint64_t seed) { return sqo_fmix64(seed); }

/* kind 1 = column child, kind 2 = bucket child */
uint64_t sqo_child_hash(uint64_t h, int kind, uint64_t i) {
  uint64_t k = (kind == 1) ? (2 * i + 1) : (2 * i + 2);
  return sqo_fmix64(h + GAMMA * k);
}

uint64_t sqo_pivot_draw(uint64_t h, uint64_t attempt, uint64_t r) {
  uint64_t s = sqo_fmix64(h ^ (0xd1b54a32d192ed03ull * (attempt + 1)));
  return sqo_fmix64(s + GAMMA * (r + 1));
}

/* floor(u * n / 2^64), by 32-bit limbs so that no 128-bit type is needed. */
uint64_t sqo_scale(uint64_t u, uint64_t n) {
  uint64_t ul = u & 0xffffffffull, uh = u >> 32;
  uint64_t nl = n & 0xffffffffull, nh = n >> 32;
  uint64_t ll = ul * nl, lh = ul * nh, hl = uh * nl, hh = uh * nh;
  uint64_t mid = (ll >> 32) + (lh & 0xffffffffull) + (hl & 0xffffffffull);
  return hh + (lh >> 32) + (hl >> 32) + (mid >> 32);
}

/* Smallest m with m*m >= n, by bisection on integers. */
uint64_t sqo_isqrt_ceil(uint64_t n) {
  uint64_t lo = 0, hi = 0x100000000ull; /* hi*hi >= any n < 2^64 */
  if (n == 0) return 0;
  while (hi - lo > 1) { /* invariant: lo*lo < n <= hi*hi */
    uint64_t mid = lo + (hi - lo) / 2;
    if (mid * mid >= n) hi = mid;
    else lo = mid;
  }
  return hi;
}

/* Largest m with m*m <= n. */
uint64_t sqo_isqrt_floor(uint64_t n) {
  uint64_t m = sqo_isqrt_ceil(n);
  return (m * m > n) ? m - 1 : m;
}

/* --------------------------------------------------------- SkewTranspose --- */

/* Pivot list of a node: pivots[0..m-2] are sampled elements; index m-1 is the
 * +inf sentinel, which is a flag and never a key value. */
typedef struct {
  const elem *p;
  uint64_t m; /* number of buckets; index m-1 is +inf */
} pivots_t;

static int below_pivot(const ctx *c, const elem *e, const pivots_t *pv, uint64_t idx) {
  if (idx == pv->m - 1) return 1; /* everything is below +inf */
  if (c->variant) return !elem_less(c->dtype, &pv->p[idx], e); /* appendix: bucket i holds e <= pivot i */
  return elem_less(c->dtype, e, &pv->p[idx]);
}

/* Algorithm 3: for each bucket i (in order), for each sub-column j (in
 * order), move the head of column j while it lies below pivot i. */
static void naive_skew_transpose(const ctx *c, const elem *A, elem *D, uint64_t l, uint64_t *col,
                                 const uint64_t *colEnd, uint64_t k, const pivots_t *pv,
                                 uint64_t piv0, uint64_t *buc) {
  for (uint64_t i = 0; i < k; i++) {
    for (uint64_t j = 0; j < l; j++) {
      while (col[j] < colEnd[j] && below_pivot(c, &A[col[j]], pv, piv0 + i)) {
        D[buc[i]] = A[col[j]];
        buc[i] = buc[i] + 1;
        col[j] = col[j] + 1;
      }
    }
  }
}

/* Algorithm 2: split the l sub-columns and the k pivots in halves and recurse
 * in the order (C1,B1), (C2,B1), (C1,B2), (C2,B2). */
static void skew_transpose(const ctx *c, const elem *A, elem *D, uint64_t l, uint64_t *col,
                           const uint64_t *colEnd, uint64_t k, const pivots_t *pv, uint64_t piv0,
                           uint64_t *buc, uint64_t threshold) {
  if (l < threshold || k < threshold) {
    naive_skew_transpose(c, A, D, l, col, colEnd, k, pv, piv0, buc);
    return;
  }
  uint64_t l2 = l / 2, k2 = k / 2;
  skew_transpose(c, A, D, l2, col, colEnd, k2, pv, piv0, buc, threshold);
  skew_transpose(c, A, D, l - l2, col + l2, colEnd + l2, k2, pv, piv0, buc, threshold);
  skew_transpose(c, A, D, l2, col, colEnd, k - k2, pv, piv0 + k2, buc + k2, threshold);
  skew_transpose(c, A, D, l - l2, col + l2, colEnd + l2, k - k2, pv, piv0 + k2, buc + k2,
                 threshold);
}

static void run_skew(const ctx *c, const elem *A, elem *D, uint64_t l, uint64_t *col,
                     const uint64_t *colEnd, uint64_t k, const pivots_t *pv, uint64_t *buc) {
  if (c->skew_mode == 0)
    naive_skew_transpose(c, A, D, l, col, colEnd, k, pv, 0, buc);
  else
    skew_transpose(c, A, D, l, col, colEnd, k, pv, 0, buc, c->skew_mode == 1 ? 4 : 10);
}

/* Bucket sizes by one simultaneous scan of each sorted column with the sorted
 * pivots (Section 2.2, first paragraph): size[j] = #{elements in bucket j}. */
static void bucket_sizes(const ctx *c, const elem *D, uint64_t l, const uint64_t *col,
                         const uint64_t *colEnd, const pivots_t *pv, uint64_t *size) {
  for (uint64_t j = 0; j < pv->m; j++) size[j] = 0;
  for (uint64_t i = 0; i < l; i++) {
    uint64_t j = 0;
    for (uint64_t t = col[i]; t < colEnd[i]; t++) {
      while (!below_pivot(c, &D[t], pv, j)) j++;
      size[j]++;
    }
  }
}

/* ------------------------------------------------------------ SquareSort --- */

static void record(ctx *c, uint64_t off, uint64_t n, uint64_t m, uint64_t h, uint32_t depth,
                   uint32_t kind, uint32_t index, uint32_t attempts) {
  if (!c->trace) return;
  if (c->trace_count < c->trace_cap) {
    sqo_node *r = &c->trace[c->trace_count];
    r->off = off;
    r->n = n;
    r->m = m;
    r->hash = h;
    r->depth = depth;
    r->kind = kind;
    r->attempts = attempts;
    r->index = index;
  }
  c->trace_count++;
}

/* Pivot selection of Algorithm 1 on the column-sorted node array D[0..n):
 * m-1 positions drawn with replacement; the sample is redrawn when two drawn
 * elements are equal or its smallest element is min(D).  Writes the sorted
 * pivots to piv[0..m-2] and returns the number of samples drawn, or 0 when
 * SQO_MAX_ATTEMPTS samples all failed. */
static uint32_t select_pivots(const ctx *c, const elem *D, uint64_t n, uint64_t m,
                              const uint64_t *col, const uint64_t *colEnd, uint64_t h,
                              elem *piv) {
  const elem *mn = NULL; /* min(D) = the smallest column head */
  for (uint64_t i = 0; i < m; i++)
    if (col[i] < colEnd[i] && (mn == NULL || elem_less(c->dtype, &D[col[i]], mn)))
      mn = &D[col[i]];
  for (uint32_t a = 0; a < SQO_MAX_ATTEMPTS; a++) {
    for (uint64_t r = 0; r + 1 < m; r++) piv[r] = D[sqo_scale(sqo_pivot_draw(h, a, r), n)];
    library_sort(c->dtype, piv, m - 1); /* MergeSort in the paper: any sort gives the same set */
    int ok = !elem_equal(c->dtype, &piv[0], mn);
    for (uint64_t r = 0; ok && r + 2 < m; r++)
      if (elem_equal(c->dtype, &piv[r], &piv[r + 1])) ok = 0;
    if (ok) return a + 1;
  }
  return 0;
}

/* Algorithm 1: sort A[0..n) into D[0..n); A is clobbered.  off is the
 * position of A[0] in the root array (for the trace only). */
static void square_sort(ctx *c, elem *A, elem *D, uint64_t n, uint64_t off, uint64_t h,
                        uint32_t depth, uint32_t kind, uint32_t index) {
  if (c->status != SQO_OK) return;
  if (n <= c->cutoff) { /* simple_sort(A, D, n), then return */
    memcpy(D, A, (size_t)n * sizeof(elem));
    library_sort(c->dtype, D, n);
    return;
  }
  uint64_t m = sqo_isqrt_ceil(n);
  uint64_t *col = malloc(m * sizeof(uint64_t)), *colEnd = malloc(m * sizeof(uint64_t));
  uint64_t *buc = malloc((m + 1) * sizeof(uint64_t)), *size = malloc(m * sizeof(uint64_t));
  uint64_t *cur = malloc(m * sizeof(uint64_t));
  elem *piv = malloc((m > 1 ? m - 1 : 1) * sizeof(elem));
  if (!col || !colEnd || !buc || !size || !cur || !piv) {
    c->status = SQO_ERR_NOMEM;
    goto out;
  }
  /* span of each column */
  for (uint64_t i = 0; i < m; i++) {
    col[i] = (i * m < n) ? i * m : n;
    colEnd[i] = ((i + 1) * m < n) ? (i + 1) * m : n;
  }
  /* sort each column of A into D */
  for (uint64_t i = 0; i < m; i++)
    if (colEnd[i] > col[i])
      square_sort(c, A + col[i], D + col[i], colEnd[i] - col[i], off + col[i],
                  sqo_child_hash(h, 1, i), depth + 1, 1, (uint32_t)i);
  if (c->status != SQO_OK) goto out;
  /* select pivots */
  uint32_t attempts = select_pivots(c, D, n, m, col, colEnd, h, piv);
  record(c, off, n, m, h, depth, kind, index, attempts);
  if (attempts == 0) {
    c->status = SQO_ERR_ATTEMPTS;
    goto out;
  }
  pivots_t pv = {piv, m};
  /* bucket starts: buc[j] = #{t : D[t] < pivots[j-1]} */
  bucket_sizes(c, D, m, col, colEnd, &pv, size);
  buc[0] = 0;
  for (uint64_t j = 0; j < m; j++) buc[j + 1] = buc[j] + size[j];
  /* skew transpose D into A; cur[] holds the free-slot pointers */
  for (uint64_t j = 0; j < m; j++) cur[j] = buc[j];
  run_skew(c, D, A, m, col, colEnd, m, &pv, cur);
  if (depth == 0 && c->root_skew) memcpy(c->root_skew, A, (size_t)n * sizeof(elem));
  /* sort each bucket from A into D */
  for (uint64_t j = 0; j < m; j++)
    if (buc[j + 1] > buc[j])
      square_sort(c, A + buc[j], D + buc[j], buc[j + 1] - buc[j], off + buc[j],
                  sqo_child_hash(h, 2, j), depth + 1, 2, (uint32_t)j);
out:
  free(col);
  free(colEnd);
  free(buc);
  free(size);
  free(cur);
  free(piv);
}

/* ------------------------------------------------- the appendix variant --- */

/* The element just below e in the (key, val) order of integer keys (e itself
 * for the minimum element, which has no predecessor). */
static elem elem_pred(elem e) {
  if (e.val > 0) {
    e.val--;
  } else if (e.key > 0) {
    e.key--;
    e.val = 0xffffffffu;
  }
  return e;
}

/* The greatest (key, val) pair of a key type. */
static elem elem_top(int dtype) {
  elem t;
  t.key = dtype == SQO_U64 ? ~(uint64_t)0 : 0xffffffffu;
  t.val = 0xffffffffu;
  return t;
}

/* The appendix listing's pivot step, on the node's input A before its column
 * sorts: m samples with replacement, sorted; index m-1 becomes the greatest
 * pair; equal neighbours separated by replacing the lower one by its
 * predecessor. */
static void appendix_pivots(const ctx *c, const elem *A, uint64_t n, uint64_t m, uint64_t h, elem *smp) {
  for (uint64_t r = 0; r < m; r++) smp[r] = A[sqo_scale(sqo_pivot_draw(h, 0, r), n)];
  library_sort(c->dtype, smp, m);
  smp[m - 1] = elem_top(c->dtype);
  for (uint64_t r = 0; r + 1 < m; r++)
    if (elem_equal(c->dtype, &smp[r], &smp[r + 1])) smp[r] = elem_pred(smp[r]);
}

/* SquareSort as the appendix listing states it: A[0..n) sorted into D[0..n). */
static void square_sort_appendix(ctx *c, elem *A, elem *D, uint64_t n, uint64_t off, uint64_t h,
                                 uint32_t depth, uint32_t kind, uint32_t index) {
  if (c->status != SQO_OK) return;
  if (n <= c->cutoff) { /* the base case: a library sort */
    memcpy(D, A, (size_t)n * sizeof(elem));
    library_sort(c->dtype, D, n);
    return;
  }
  const uint64_t m = sqo_isqrt_floor(n);
  uint64_t *first = malloc(m * sizeof(uint64_t)), *last = malloc(m * sizeof(uint64_t));
  uint64_t *starts = malloc((m + 1) * sizeof(uint64_t)), *cnt = malloc(m * sizeof(uint64_t));
  uint64_t *slot = malloc(m * sizeof(uint64_t));
  elem *smp = malloc(m * sizeof(elem));
  if (!first || !last || !starts || !cnt || !slot || !smp) {
    c->status = SQO_ERR_NOMEM;
    goto done;
  }
  /* pivots from the input, before any column is sorted */
  appendix_pivots(c, A, n, m, h, smp);
  /* m columns of m elements; the last one runs to n */
  for (uint64_t i = 0; i < m; i++) {
    first[i] = i * m;
    last[i] = (i + 1 < m) ? (i + 1) * m : n;
  }
  for (uint64_t i = 0; i < m; i++)
    square_sort_appendix(c, A + first[i], D + first[i], last[i] - first[i], off + first[i],
                         sqo_child_hash(h, 1, i), depth + 1, 1, (uint32_t)i);
  if (c->status != SQO_OK) goto done;
  record(c, off, n, m, h, depth, kind, index, 1);
  pivots_t pv = {smp, m};
  bucket_sizes(c, D, m, first, last, &pv, cnt);
  starts[0] = 0;
  for (uint64_t b = 0; b < m; b++) starts[b + 1] = starts[b] + cnt[b];
  for (uint64_t b = 0; b < m; b++) slot[b] = starts[b];
  run_skew(c, D, A, m, first, last, m, &pv, slot);
  if (depth == 0 && c->root_skew) memcpy(c->root_skew, A, (size_t)n * sizeof(elem));
  for (uint64_t b = 0; b < m; b++) {
    const uint64_t len = starts[b + 1] - starts[b];
    int mono; /* the bucket's range holds one (key, val) pair: only copies of it */
    if (b == 0) {
      const elem least = {0, 0};
      mono = elem_equal(c->dtype, &smp[0], &least);
    } else {
      const elem lowp = elem_pred(smp[b]);
      mono = elem_less(c->dtype, &smp[b - 1], &smp[b]) && elem_equal(c->dtype, &lowp, &smp[b - 1]);
    }
    if (mono)
      memcpy(D + starts[b], A + starts[b], (size_t)len * sizeof(elem));
    else if (len)
      square_sort_appendix(c, A + starts[b], D + starts[b], len, off + starts[b],
                           sqo_child_hash(h, 2, b), depth + 1, 2, (uint32_t)b);
  }
done:
  free(first);
  free(last);
  free(starts);
  free(cnt);
  free(slot);
  free(smp);
}

/* ---------------------------------------------------------- entry points --- */

static void load_elems(int dtype, const void *keys, const uint32_t *vals, uint64_t n, elem *e) {
  for (uint64_t i = 0; i < n; i++) {
    e[i].key = (dtype == SQO_U64) ? ((const uint64_t *)keys)[i] : ((const uint32_t *)keys)[i];
    e[i].val = vals ? vals[i] : (uint32_t)i;
  }
}

static void store_elems(int dtype, const elem *e, uint64_t n, void *keys, uint32_t *vals) {
  for (uint64_t i = 0; i < n; i++) {
    if (dtype == SQO_U64) ((uint64_t *)keys)[i] = e[i].key;
    else ((uint32_t *)keys)[i] = (uint32_t)e[i].key;
    if (vals) vals[i] = e[i].val;
  }
}

/* Sorts (keys, vals) in place with SquareSort.  keys: uint32/float32-bits or
 * uint64 array of n; vals: uint32 payload (NULL: the position is used and not
 * returned).  trace (optional) receives one record per recursing call;
 * root_skew_keys/vals (optional) receive the root's array after its
 * SkewTranspose.  Returns SQO_OK or an error code. */
int sqo_sort(int dtype, void *keys, uint32_t *vals, uint64_t n, uint64_t seed, uint64_t cutoff,
             int skew_mode, sqo_node *trace, uint64_t trace_cap, uint64_t *trace_count,
             void *root_skew_keys, uint32_t *root_skew_vals) {
  if (dtype < 0 || dtype > 2 || cutoff < 2 || skew_mode < 0 || skew_mode > 2) return SQO_ERR_INVALID;
  if (n > 0xffffffffull) return SQO_ERR_INVALID;
  if (n == 0) {
    if (trace_count) *trace_count = 0;
    return SQO_OK;
  }
  elem *A = malloc((size_t)n * sizeof(elem)), *D = malloc((size_t)n * sizeof(elem));
  elem *rs = root_skew_keys ? malloc((size_t)n * sizeof(elem)) : NULL;
  if (!A || !D || (root_skew_keys && !rs)) {
    free(A);
    free(D);
    free(rs);
    return SQO_ERR_NOMEM;
  }
  load_elems(dtype, keys, vals, n, A);
  ctx c = {dtype, cutoff, skew_mode, SQO_OK, trace, trace_cap, 0, rs, 0};
  if (rs) memcpy(rs, A, (size_t)n * sizeof(elem)); /* a leaf root has no skew: keep input */
  square_sort(&c, A, D, n, 0, sqo_root_hash(seed), 0, 0, 0);
  if (c.status == SQO_OK) {
    store_elems(dtype, D, n, keys, vals);
    if (rs) store_elems(dtype, rs, n, root_skew_keys, root_skew_vals);
  }
  if (trace_count) *trace_count = c.trace_count;
  free(A);
  free(D);
  free(rs);
  return c.status;
}

/* Sorts (keys, vals) in place with the appendix variant (arguments as
 * sqo_sort; integer keys only: SQO_U32 or SQO_U64). */
int sqo_sort_appendix(int dtype, void *keys, uint32_t *vals, uint64_t n, uint64_t seed, uint64_t cutoff,
                      sqo_node *trace, uint64_t trace_cap, uint64_t *trace_count, void *root_skew_keys,
                      uint32_t *root_skew_vals) {
  /* cutoff >= 8: a node has n >= 9, so m = floor(sqrt n) >= 3; every column is smaller than the node, and so is
   * every bucket that is not copied (a bucket holding the whole node lies between two pivots that are an
   * element and its predecessor, or below a pivot equal to the least pair) */
  if ((dtype != SQO_U32 && dtype != SQO_U64) || cutoff < 8) return SQO_ERR_INVALID;
  if (n > 0xffffffffull) return SQO_ERR_INVALID;
  if (n == 0) {
    if (trace_count) *trace_count = 0;
    return SQO_OK;
  }
  elem *A = malloc((size_t)n * sizeof(elem)), *D = malloc((size_t)n * sizeof(elem));
  elem *rs = root_skew_keys ? malloc((size_t)n * sizeof(elem)) : NULL;
  if (!A || !D || (root_skew_keys && !rs)) {
    free(A);
    free(D);
    free(rs);
    return SQO_ERR_NOMEM;
  }
  load_elems(dtype, keys, vals, n, A);
  ctx c = {dtype, cutoff, 0, SQO_OK, trace, trace_cap, 0, rs, 1};
  if (rs) memcpy(rs, A, (size_t)n * sizeof(elem));
  square_sort_appendix(&c, A, D, n, 0, sqo_root_hash(seed), 0, 0, 0);
  if (c.status == SQO_OK) {
    store_elems(dtype, D, n, keys, vals);
    if (rs) store_elems(dtype, rs, n, root_skew_keys, root_skew_vals);
  }
  if (trace_count) *trace_count = c.trace_count;
  free(A);
  free(D);
  free(rs);
  return c.status;
}

/* SkewTranspose of `cols` sorted columns of height <= rows (column i is
 * [min(i*rows,n), min((i+1)*rows,n))) into k buckets bounded by the k-1
 * sorted pivots (bucket k-1 is bounded by +inf).  mode: 0 = Algorithm 3,
 * 1 = Algorithm 2 with threshold 4, 2 = Algorithm 2 with threshold 10.
 * bucket_start receives k+1 offsets (bucket j = [start[j], start[j+1])). */
int sqo_skew_transpose(int dtype, const void *keys_in, const uint32_t *vals_in, uint64_t n,
                       uint64_t rows, uint64_t cols, const void *piv_keys,
                       const uint32_t *piv_vals, uint64_t k, void *keys_out, uint32_t *vals_out,
                       uint64_t *bucket_start, int mode) {
  if (dtype < 0 || dtype > 2 || mode < 0 || mode > 2 || k == 0 || cols == 0) return SQO_ERR_INVALID;
  if (n > rows * cols) return SQO_ERR_INVALID;
  elem *A = malloc((n ? n : 1) * sizeof(elem)), *D = malloc((n ? n : 1) * sizeof(elem));
  elem *piv = malloc(k * sizeof(elem));
  uint64_t *col = malloc(cols * sizeof(uint64_t)), *colEnd = malloc(cols * sizeof(uint64_t));
  uint64_t *size = malloc(k * sizeof(uint64_t)), *cur = malloc(k * sizeof(uint64_t));
  int st = SQO_OK;
  if (!A || !D || !piv || !col || !colEnd || !size || !cur) {
    st = SQO_ERR_NOMEM;
    goto out;
  }
  load_elems(dtype, keys_in, vals_in, n, A);
  load_elems(dtype, piv_keys, piv_vals, k - 1, piv);
  for (uint64_t i = 0; i < cols; i++) {
    col[i] = (i * rows < n) ? i * rows : n;
    colEnd[i] = ((i + 1) * rows < n) ? (i + 1) * rows : n;
  }
  ctx c = {dtype, 2, mode, SQO_OK, NULL, 0, 0, NULL, 0};
  pivots_t pv = {piv, k};
  bucket_sizes(&c, A, cols, col, colEnd, &pv, size);
  bucket_start[0] = 0;
  for (uint64_t j = 0; j < k; j++) bucket_start[j + 1] = bucket_start[j] + size[j];
  for (uint64_t j = 0; j < k; j++) cur[j] = bucket_start[j];
  run_skew(&c, A, D, cols, col, colEnd, k, &pv, cur);
  store_elems(dtype, D, n, keys_out, vals_out);
out:
  free(A);
  free(D);
  free(piv);
  free(col);
  free(colEnd);
  free(size);
  free(cur);
  return st;
}

/* One SquareSort node's first steps (column sorts by a library sort, pivot
 * selection, bucket sizes) on keys 0..n-1 given in `keys` (distinct uint64
 * values, any order).  Used for the statistical checks of Section 3.  Writes
 * the m bucket sizes and returns the number of samples drawn (0 on failure). */
uint32_t sqo_node_buckets(const uint64_t *keys, uint64_t n, uint64_t h, uint64_t *sizes_out) {
  uint64_t m = sqo_isqrt_ceil(n);
  elem *D = malloc((size_t)n * sizeof(elem));
  elem *piv = malloc((m > 1 ? m - 1 : 1) * sizeof(elem));
  uint64_t *col = malloc(m * sizeof(uint64_t)), *colEnd = malloc(m * sizeof(uint64_t));
  uint32_t attempts = 0;
  if (!D || !piv || !col || !colEnd) goto out;
  for (uint64_t i = 0; i < n; i++) {
    D[i].key = keys[i];
    D[i].val = (uint32_t)i;
  }
  for (uint64_t i = 0; i < m; i++) {
    col[i] = (i * m < n) ? i * m : n;
    colEnd[i] = ((i + 1) * m < n) ? (i + 1) * m : n;
    if (colEnd[i] > col[i]) library_sort(SQO_U64, D + col[i], colEnd[i] - col[i]);
  }
  ctx c = {SQO_U64, 2, 0, SQO_OK, NULL, 0, 0, NULL, 0};
  attempts = select_pivots(&c, D, n, m, col, colEnd, h, piv);
  if (attempts) {
    pivots_t pv = {piv, m};
    bucket_sizes(&c, D, m, col, colEnd, &pv, sizes_out);
  }
out:
  free(D);
  free(piv);
  free(col);
  free(colEnd);
  return attempts;
}
