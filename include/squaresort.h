/*
 * squaresort.h -- C ABI of the GB300 SquareSort library (libsquaresort.so).
 *
 * SquareSort (Koucky & Matejka, "SquareSort: a cache-oblivious sorting
 * algorithm", arXiv 2407.14801) views n items as m = ceil(sqrt(n)) columns of
 * at most m items, sorts every column, picks m-1 random pivots, moves the
 * items bucket by bucket with a SkewTranspose and sorts every bucket,
 * recursing wherever a column or bucket is larger than the leaf cutoff
 * (Section 2, Algorithm 1).
 *
 * Conventions for every call below:
 *  - Pointers are plain addresses.  Key and payload buffers may be device
 *    memory (the fast path) or, for sq_sort / sq_sort_ex only, host memory.
 *    Page-locked (pinned, mapped) host buffers are read by the first pass
 *    and written by the last pass directly through the device mapping, with
 *    device memory only for the rounds between; other host memory is staged
 *    through device memory inside the call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work is ordered on it.  In the CUDA-graph launch mode (SQ_LAUNCH_GRAPH,
 *    see sq_set_launch_mode) sq_sort / sq_sort_ex without a trace and
 *    sq_sort_batch on device buffers are asynchronous: they enqueue the whole
 *    recursion and return; the buffers must not be touched until the stream
 *    has passed the work (sq_sync, or any later synchronisation of the
 *    stream).  Errors found on the device are latched and returned by
 *    sq_sync(stream) or by the next sq_sort / sq_sort_ex / sq_sort_batch on
 *    the same stream.  In the host-driven launch mode (the default; the
 *    engine reads each recursion round's work counts back to size the next
 *    round's launches, and was measured 2-4% faster on the 2^28 sort) and
 *    for host buffers, traced sorts, the SkewTranspose and the server calls,
 *    a call returns after its work is finished.
 *  - Element order: (key, val) pairs by (ordinal(key), val).  ordinal is the
 *    identity for SQ_U32 / SQ_U64; SQ_F32 keys are IEEE-754 binary32 bit
 *    patterns ordered -inf < ... < -0 < +0 < ... < +inf < NaN, every NaN equal
 *    (ties among NaNs broken by val); the bits of every key are preserved.
 *  - Errors are returned as sq_status, never thrown; sq_last_error() gives a
 *    thread-local message for the last failing call of the calling thread.
 */
#ifndef SQUARESORT_H
#define SQUARESORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *sq_stream_t; /* a cudaStream_t */

typedef enum { SQ_U32 = 0, SQ_U64 = 1, SQ_F32 = 2 } sq_dtype;

typedef enum {
  SQ_OK = 0,
  SQ_ERR_INVALID = 1,  /* bad argument (null pointer, size, dtype, cutoff) */
  SQ_ERR_NOMEM = 2,    /* device memory or an internal work list ran out */
  SQ_ERR_BUDGET = 3,   /* a request does not fit the server's HBM budget */
  SQ_ERR_TIMEOUT = 4,  /* a bounded wait ran out */
  SQ_ERR_CUDA = 5,     /* a CUDA runtime call failed */
  SQ_PENDING = 6,      /* sq_serve_poll: not finished yet */
  SQ_ERR_ATTEMPTS = 7, /* no acceptable pivot sample in 256 draws (e.g. repeated (key, val) pairs) */
  SQ_ERR_INTERNAL = 8  /* an engine invariant failed */
} sq_status;

/* Sort n (key, val) pairs in place (Algorithm 1, Section 2.1).
 *  keys : n keys of `dtype` (4 bytes for SQ_U32/SQ_F32, 8 for SQ_U64).
 *  vals : n uint32 payloads moved with their keys; ties between equal keys
 *         are broken by val, so with distinct vals the result is unique.
 *         NULL: the original position is used for ties and nothing is
 *         returned.
 *  n    : 0 <= n <= sq_max_n(dtype).
 *  seed : seeds the pivot draws; the result does not depend on it, the
 *         recursion (which pivots, how many redraws) does.
 * Scratch of n*(key bytes + 4) plus O(n/16) bytes of metadata comes from the
 * CUDA stream-ordered allocator and is released before return. */
sq_status sq_sort(void *keys, uint32_t *vals, uint64_t n, sq_dtype dtype, uint64_t seed, sq_stream_t stream);

/* Per-node record of a traced sort: one per SquareSort call with n > cutoff,
 * written when its pivots are accepted (Algorithm 1, pivot step). */
typedef struct {
  uint64_t off;      /* first element of the node in the array */
  uint64_t n;        /* node size */
  uint64_t m;        /* columns = buckets: ceil(sqrt(n)) (floor under SQ_APPENDIX) */
  uint64_t hash;     /* path hash that seeds its pivot draws */
  uint32_t depth;    /* root = 0 */
  uint32_t kind;     /* 0 root, 1 column child, 2 bucket child */
  uint32_t attempts; /* pivot samples drawn (1 = first accepted) */
  uint32_t index;    /* column / bucket index within the parent */
} sq_trace_rec;

/* Recursion variants.  SQ_ALGORITHM1 is Algorithm 1 (Section 2.1).
 * SQ_APPENDIX is the code the paper prints in its appendix, which Section 2.1
 * says departs a little from Algorithm 1: m = floor(sqrt n) columns of m
 * elements, the last one extended to the end of the node; m pivot samples
 * drawn once (no redraws) from the node's input before its columns are
 * sorted, the largest replaced by the greatest (key, val) pair and each
 * sample equal to the next one lowered to its predecessor in the (key, val)
 * order; bucket i holds the elements e with p_{i-1} < e <= p_i; a bucket
 * whose range holds a single pair (p_{i-1} the predecessor of p_i, or p_0 =
 * the least pair (0, 0)) is copied, not sorted.  Integer keys only (SQ_U32,
 * SQ_U64), a cutoff of at least 8 (so that every node draws m >= 3 samples),
 * and n < (p + 1)^2 with p = 16384 for SQ_U32, 8192 for SQ_U64 (the samples
 * are sorted by one CTA).  Repeated (key, val) pairs are allowed. */
typedef enum { SQ_ALGORITHM1 = 0, SQ_APPENDIX = 1 } sq_variant;

typedef struct {
  uint32_t cutoff;        /* leaf iff n <= cutoff; 0 = the default; 2..sq_max_leaf(dtype) */
  uint32_t trace_cap;     /* capacity of `trace` in records (0 = no trace) */
  sq_trace_rec *trace;    /* host array receiving node records (any order) */
  uint32_t *trace_count;  /* out: records produced (may exceed trace_cap) */
  uint32_t variant;       /* sq_variant; 0 = Algorithm 1 */
} sq_sort_opts;

/* sq_sort with an explicit leaf cutoff and an optional recursion trace.
 * opts may be NULL (= sq_sort). */
sq_status sq_sort_ex(void *keys, uint32_t *vals, uint64_t n, sq_dtype dtype, uint64_t seed, sq_stream_t stream,
                     const sq_sort_opts *opts);

/* Waits for the stream's work and returns the first error latched by an
 * asynchronous sq_sort / sq_sort_ex / sq_sort_batch on it (SQ_OK if none;
 * each latched error is returned once).  The paper has no counterpart: it is
 * the completion point of the asynchronous calls above.  An asynchronous
 * sort starts with room for 4 * n / cutoff + 4096 recursion nodes (several
 * times what sorts use) and cannot grow it; if a sort needs more it stops
 * unfinished and sq_sync returns SQ_ERR_NOMEM (sort it again in the
 * host-driven mode). */
sq_status sq_sync(sq_stream_t stream);

/* Stand-alone SkewTranspose (Section 2.2, Algorithms 2 and 3).
 * keys_in/vals_in hold `cols` columns, column i = elements
 * [min(i*rows, n), min((i+1)*rows, n)), each sorted by the element order.
 * The k-1 sorted pivots (pivot_keys/pivot_vals, device) define k buckets,
 * bucket j = { e : p_{j-1} <= e < p_j } with p_0 = -inf, p_k = +inf.  The
 * call writes to keys_out/vals_out every bucket in turn, each holding its
 * elements column by column and, within a column, in sorted order; and
 * writes the k+1 bucket starts (uint64, device) to bucket_start_out.
 * All buffers are caller-owned device memory; in and out must not overlap. */
typedef struct {
  sq_dtype dtype;
  uint64_t n;
  const void *keys_in;
  const uint32_t *vals_in;
  void *keys_out;
  uint32_t *vals_out;
  const void *pivot_keys;
  const uint32_t *pivot_vals;
  uint64_t k;                  /* buckets; 1 <= k <= p + 1, p = 16384 for SQ_U32, 8192 otherwise */
  uint64_t *bucket_start_out;  /* k+1 entries */
} sq_skew_buf;

/* rows >= 1, cols >= 1, n <= rows*cols, n < 2^32. */
sq_status sq_skew_transpose(const sq_skew_buf *buf, uint64_t rows, uint64_t cols, sq_stream_t stream);

/* sq_skew_transpose without any device allocation.  The paper has no
 * counterpart: this is for callers that cannot allocate device memory where
 * they need the permutation -- a process whose frameworks already hold the
 * whole device in their own caching pools, or a latency-critical path that
 * must not call cudaMalloc / cudaFree (they can synchronise the device or
 * fail under memory pressure).  Same arguments, results, errors and error
 * messages as sq_skew_transpose; all scratch (per-node metadata, work lists,
 * status words) comes from one 64 MiB array in device memory.  The array is
 * reserved on a device by the first call made there (that call loads the
 * part of the library that holds it), and stays reserved until the process
 * exits; so make one call on each device at start-up, before other pools
 * fill it and before any stream capture.  If that first reservation fails
 * the call returns SQ_ERR_CUDA and leaves no CUDA error pending.  Shapes
 * whose scratch exceeds 64 MiB (about 0.078 * k * cols + 2 * (k + cols)
 * 32-bit words, e.g. beyond roughly 14000 x 14000 with k = cols) are refused
 * with SQ_ERR_INVALID and a message naming the size.  Every call uses the
 * same array and leaves the previous call's contents behind (the call
 * initialises what it reads): calls whose GPU work overlaps -- on different
 * streams or from different threads -- race on it and must be serialised by
 * the caller.  Unlike sq_skew_transpose, which allocates a one-byte bucket
 * tag per element for its counting-sort kernel, this form runs the
 * SkewTranspose kernel that searches the pivots itself. */
sq_status sq_skew_transpose_noalloc(const sq_skew_buf *buf, uint64_t rows, uint64_t cols, sq_stream_t stream);

/* One instance of a batched sort: device buffers, sorted in place. */
typedef struct {
  void *keys;
  uint32_t *vals; /* NULL allowed, as in sq_sort */
  uint64_t n;
  sq_dtype dtype;
  uint64_t seed;
} sq_sort_desc;

/* Sort `count` independent instances of any sizes and key types together:
 * every recursion round of every instance runs in the same kernel launches
 * (work items pulled from device lists), instead of one launch sequence per
 * instance.  Each instance's result equals sq_sort of that instance. */
sq_status sq_sort_batch(const sq_sort_desc *descs, uint32_t count, sq_stream_t stream);

/* ------------------------------------------------------------- serving --- */

typedef struct sq_server sq_server;

typedef struct {
  uint32_t max_inflight;  /* requests admitted at once (0 = 4096) */
  uint32_t cutoff;        /* leaf cutoff (0 = tuned default) */
  int device;             /* CUDA device ordinal */
} sq_serve_opts;

/* Create a server whose device memory pool holds at most hbm_budget_bytes
 * (requests' keys, vals and scratch, and the engines' work lists).  One
 * persistent engine per key type runs the recursion rounds of every request
 * of that type in flight, in the same launches; between two rounds it admits
 * the queued requests that fit the pool and its in-flight limits (first
 * come, first served within the key type), whose roots join the next
 * round's work, and it hands back every request whose sort completed in
 * the round just run (continuous batching).  max_inflight bounds the
 * requests in flight per key type.  opts may be NULL. */
sq_status sq_serve_create(sq_server **out, uint64_t hbm_budget_bytes, const sq_serve_opts *opts);

/* Queue one sort.  desc->keys / desc->vals are HOST pointers that must stay
 * valid until sq_serve_poll reports completion; the result is written back
 * to them.  A request whose data needs more than half the budget (or more
 * elements than its key type's engine holds in flight) fails with
 * SQ_ERR_BUDGET.  *ticket identifies the request. */
sq_status sq_serve_submit(sq_server *srv, const sq_sort_desc *desc, uint64_t *ticket);

/* SQ_PENDING while the request runs; SQ_OK once its result is in the
 * caller's buffers (then *result holds the request's own status and
 * *latency_s the time from submit to completion).  Polling a finished ticket
 * again returns SQ_ERR_INVALID. */
sq_status sq_serve_poll(sq_server *srv, uint64_t ticket, sq_status *result, double *latency_s);

/* Stop the server after draining admitted work; frees the pool. */
sq_status sq_serve_destroy(sq_server *srv);

/* ----------------------------------------------------------- utilities --- */

/* Message of the calling thread's last failing call ("" if none). */
const char *sq_last_error(void);

/* Largest n accepted by sq_sort for `dtype`: (p + 1)^2 with p the largest
 * pivot sample of a node -- for SQ_U32 65535, sorted by a cluster of 8 CTAs,
 * capped at 2^32 - 1; 8192 otherwise (one CTA).  An SQ_U32 sort above 2^28
 * has a root with more than 16384 pivots; its bucket count reads them from
 * global memory. */
uint64_t sq_max_n(sq_dtype dtype);

/* Largest leaf sorted directly (the largest allowed cutoff): 65536, by a
 * cluster of CTAs merging through distributed shared memory. */
uint32_t sq_max_leaf(sq_dtype dtype);

/* Default leaf cutoff for `dtype`; while set it also overrides the cutoff
 * table below (0 restores the table and the built-in default, the largest
 * leaf). */
sq_status sq_set_cutoff(sq_dtype dtype, uint32_t cutoff);
uint32_t sq_get_cutoff(sq_dtype dtype);

/* Cutoffs by size (written by the autotuner): entry i applies to sorts with
 * floor(log2 n) == i when non-zero and no cutoff is set with sq_set_cutoff;
 * count <= 64 entries, the rest are cleared.  The cutoff decides where Algorithm 1
 * stops recursing (§4.2 sweeps it); results do not depend on it. */
sq_status sq_set_cutoff_table(sq_dtype dtype, const uint32_t *cutoff_by_log2n, uint32_t count);

/* The cutoff a sort of n keys of `dtype` uses when none is given. */
uint32_t sq_cutoff_for(sq_dtype dtype, uint64_t n);

/* How the recursion's rounds are launched.  Algorithm 1 runs here breadth
 * first: every round sorts the pending leaves and takes every ready node
 * through pivots, counts, SkewTranspose and child creation.
 *  SQ_LAUNCH_HOST : the host launches each round's kernels with grids sized
 *                   to the round's work and reads the next round's work
 *                   counts back (one round trip per round).
 *  SQ_LAUNCH_GRAPH: all rounds run as one CUDA-graph launch whose device-side
 *                   loop ends when every instance is sorted; kernels read
 *                   their work counts on the device.  The graph is built once
 *                   per thread and device and reused by later calls.  Sorts
 *                   on device buffers without a trace are asynchronous (see
 *                   the conventions above and sq_sync).
 *  SQ_LAUNCH_AUTO : (default) currently host rounds everywhere: the graph
 *                   launches every step of a round at a fixed size and was
 *                   measured slower for single, batched and served sorts.
 * Results do not depend on the mode.  While profiling is on
 * (sq_set_profiling) rounds are always host-launched, so that every kernel
 * is timed. */
typedef enum { SQ_LAUNCH_HOST = 0, SQ_LAUNCH_GRAPH = 1, SQ_LAUNCH_AUTO = 2 } sq_launch_mode;
sq_status sq_set_launch_mode(sq_launch_mode mode);
sq_launch_mode sq_get_launch_mode(void);

/* Which base-case sort a leaf gets (Algorithm 1's simple_sort, which the
 * paper leaves open: insertion sort, std::sort below a cutoff, Section 4).
 * Leaves are sorted by size class: class c holds leaves of up to 64 (c = 0),
 * 512 (1), 2048 (2) and (c - 2) * 8192 elements (c = 3..10).  Bit c of
 * `mask` set: leaves of class c with 32-bit key ordinals (SQ_U32, SQ_F32)
 * take the radix base case (a stable LSD radix sort of the key ordinal on
 * one CTA of up to 16K elements, clusters above that, checked against the (key, val) order and merge
 * sorted where it is not); clear: the merge sort.  Only classes 2..10 have a
 * radix kernel (other bits are ignored), and SQ_U64 always merge sorts
 * (sq_set_radix_classes returns SQ_ERR_INVALID for it).  The default mask is
 * every radix class (0x7FC); the binding applies the autotuner's masks.  Results do not depend on the mask; the
 * autotuner measures it.  Process-wide; takes effect at the next call. */
sq_status sq_set_radix_classes(sq_dtype dtype, uint32_t mask);
uint32_t sq_get_radix_classes(sq_dtype dtype);

/* Per-kernel-family counters accumulated by all calls of this process.
 * Families: 0 leaf sort, 1 plan, 2 pivots, 3 count, 4 prefix scan,
 * 5 bucket starts, 6 SkewTranspose, 7 child expansion, 8 auxiliary. */
typedef struct {
  uint64_t launches[9];
  double ms[9];     /* summed kernel durations (only while profiling is on) */
  double bytes[9];  /* algorithmic bytes: leaf 2(w+4)/elem, count (w+4)/elem, skew 2(w+4)/elem */
  uint64_t rounds;  /* recursion rounds (one host read-back each) */
  uint64_t nodes;   /* SquareSort calls with n > cutoff */
  uint64_t sorts;   /* instances sorted */
} sq_stats;

void sq_stats_get(sq_stats *out);
void sq_stats_reset(void);
/* on != 0: time every launch with CUDA events on its stream (adds a little
 * host work per launch). */
void sq_set_profiling(int on);

#ifdef __cplusplus
}
#endif
#endif /* SQUARESORT_H */
