// Host-side interface of the SquareSort engine (one instantiation per key
// type).  Plain C++: no CUDA device code here.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace sq {

// Kernel families, for launch counts, timings and algorithmic bytes.
enum KernelFamily : int {
  KF_LEAF = 0,
  KF_PLAN,
  KF_PIVOTS,
  KF_COUNT,
  KF_SCAN,
  KF_BSTART,
  KF_SKEW,
  KF_EXPAND,
  KF_AUX,
  KF_COUNT_FAMILIES
};

struct EngineStats {
  uint64_t launches[KF_COUNT_FAMILIES];
  double ms[KF_COUNT_FAMILIES];     // summed launch durations (profiling on)
  double bytes[KF_COUNT_FAMILIES];  // algorithmic bytes moved
  uint64_t rounds;
  uint64_t nodes;  // recursing SquareSort calls
  uint64_t sorts;
};

// One sort instance as the engine sees it: device buffers only.
struct InstSpec {
  void *keys;      // A keys (device)
  uint32_t *vals;  // A vals (device)
  void *dkeys;     // D keys scratch (device), same length
  uint32_t *dvals; // D vals scratch (device)
  uint8_t *tags;   // n bytes of scratch (device) for bucket tags; NULL: the SkewTranspose classifies
  // Optional (NULL: keys / vals): where the first pass reads the input and
  // where the last pass writes the result, e.g. mapped pinned host buffers.
  const void *skeys;
  const uint32_t *svals;
  void *fkeys;
  uint32_t *fvals;
  uint64_t n;
  uint64_t seed;
  uint32_t cutoff;  // 0: RunSpec::cutoff
  uint32_t variant; // 0: Algorithm 1; 1: the appendix listing's variant (integer keys, cutoff >= 3)
};

struct TraceOut {
  uint64_t off, n, m, hash;
  uint32_t depth, kind, attempts, index;
};

struct RunSpec {
  const InstSpec *inst;  // host array
  uint32_t ninst;
  uint32_t cutoff;      // default leaf cutoff: leaf iff n <= cutoff (2 <= cutoff <= max_leaf)
  TraceOut *trace;      // host array (optional) receiving per-node records
  uint32_t trace_cap;
  uint32_t *trace_count;  // out
  // stand-alone SkewTranspose (no recursion): instance 0, keys_in = dkeys,
  // keys_out = keys; pivots (k-1) from the caller; bucket starts out.
  int skew_only;
  uint64_t rows, cols, k;
  const void *piv_keys;       // device
  const uint32_t *piv_vals;   // device
  uint64_t *bucket_start;     // device, k+1
  // Optional device allocator for the engine's own scratch (default:
  // cudaMallocAsync / cudaFreeAsync on the stream).
  void *(*dev_alloc)(void *ctx, size_t bytes);
  void (*dev_free)(void *ctx, void *p);
  void *alloc_ctx;
  // Optional host buffer (any memory, >= 512 bytes) for the per-round
  // read-back; default: pinned memory from cudaMallocHost.
  void *host_readback;
  // 1: run all rounds as one CUDA-graph launch (device-side loop) instead
  // of one host round trip per round; ignored while profiling.
  int graph;
  // 1 (with graph, no trace): return once the work is enqueued; the run's
  // status is collected later by engine_sync / engine_poll on the stream.
  int async;
};

// Asynchronous runs still in flight (or finished but not yet collected).
// engine_sync waits for the stream and collects its runs; engine_poll
// collects the stream's runs that have finished, without waiting.  Both
// return 0 or the first run's status code (sq_status values), with its
// message in err.
int engine_sync(cudaStream_t st, char *err, size_t errlen);
int engine_poll(cudaStream_t st, char *err, size_t errlen);

// Device scratch bytes (slab + node record) of a stand-alone SkewTranspose.
uint64_t engine_skew_scratch_bytes(int dtype, uint64_t n, uint64_t cols, uint64_t k);

// Upper bound of the engine's own scratch bytes for a run (admission control).
uint64_t engine_scratch_bytes(int dtype, uint64_t total_n, uint32_t ninst, uint32_t cutoff, uint32_t cutoff_max);

// A persistent engine that instances join between rounds (continuous
// batching): planned once for total_n_cap elements and ninst_cap instances
// in flight.  Scratch from dev_alloc (NULL: cudaMallocAsync on the stream).
struct SessionSpec {
  uint64_t total_n_cap;
  uint32_t ninst_cap;
  uint32_t cutoff_min, cutoff_max;  // the instances' cutoffs lie in this range
  void *(*dev_alloc)(void *ctx, size_t bytes);
  void (*dev_free)(void *ctx, void *p);
  void *alloc_ctx;
};
// Returns 0 or a status code; *out is an opaque session of key type dtype.
int session_open(int dtype, const SessionSpec &sp, cudaStream_t st, void **out, char *err, size_t errlen);
// Starts instance `is` (tags required; n > 0) in slot `slot` at the next round.
int session_admit(int dtype, void *s, const InstSpec &is, uint32_t slot, char *err, size_t errlen);
// Runs one round if anything is in flight; appends the completed slots.
int session_step(int dtype, void *s, std::vector<uint32_t> &completed, char *err, size_t errlen);
bool session_busy(int dtype, void *s);
void session_close(int dtype, void *s);
uint64_t session_scratch_bytes(int dtype, const SessionSpec &sp);

// Returns 0 or a status code (sq_status values); writes a message on error.
int engine_run_u32(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen);
int engine_run_u64(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen);
int engine_run_f32(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen);

// Sets the calling thread's sq_last_error() message.
void api_set_error(const char *msg);

// Largest leaf (and pivot sample) the engine sorts in one group, per key type.
uint32_t engine_max_leaf(int dtype);

// Largest pivot sample (k - 1) that one CTA sorts: bounds the stand-alone
// SkewTranspose's k and the appendix variant's n, (max + 1)^2.
uint32_t engine_max_pivots(int dtype);

// Largest n of a sort (larger pivot samples sorted by a cluster of CTAs where
// the key type has that path).
uint64_t engine_max_n(int dtype);

// Global statistics (all engines, all threads), and kernel timing switch.
void engine_stats_get(EngineStats *out);
void engine_stats_reset();
void engine_set_profiling(int on);

// Leaf classes sorted by the radix base case, per key type (sq_set_radix_classes).
void engine_set_radix_classes(int dtype, uint32_t mask);
uint32_t engine_get_radix_classes(int dtype);

}  // namespace sq
