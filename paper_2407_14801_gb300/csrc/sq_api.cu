// C ABI of the SquareSort library: argument checks, host staging, scratch
// allocation and dispatch to the per-key-type engines.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/squaresort.h"
#include "sq_engine.h"
#include "sq_types.cuh"

namespace {

thread_local char g_err[512];

sq_status fail(sq_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

std::atomic<uint32_t> g_cutoff[3] = {{0}, {0}, {0}};
// Per key type and floor(log2 n): the cutoff an autotuner chose (0 = none).
std::atomic<uint32_t> g_cutoff_table[3][64];

size_t key_bytes(sq_dtype d) { return d == SQ_U64 ? 8 : 4; }
bool dtype_ok(int d) { return d >= 0 && d <= 2; }

uint32_t default_cutoff(sq_dtype d) {
  const uint32_t c = g_cutoff[d].load();
  return c ? c : sq::engine_max_leaf(d);
}

// How recursion rounds are launched (sq_set_launch_mode).
std::atomic<int> g_launch_mode{SQ_LAUNCH_AUTO};

// SQ_LAUNCH_AUTO runs host rounds: graph rounds launch every step of a
// round at a fixed size and measured slower on every workload here.
int graph_for(bool) { return g_launch_mode.load() == SQ_LAUNCH_GRAPH ? 1 : 0; }

// A cutoff set with sq_set_cutoff wins; else the tuned table's entry for
// floor(log2 n); else the largest leaf.
uint32_t cutoff_for(sq_dtype d, uint64_t n) {
  if (g_cutoff[d].load()) return g_cutoff[d].load();
  if (n) {
    const int lg = 63 - __builtin_clzll(n);
    const uint32_t t = g_cutoff_table[d][lg].load();
    if (t) return t;
  }
  return default_cutoff(d);
}

// Scratch comes from the device's default stream-ordered pool.  By default
// that pool hands freed memory back to the driver at every synchronisation,
// so each call would map its scratch afresh; keeping it cached (once per
// device, for this process) makes repeated sorts allocation-cheap.
void keep_pool_cached() {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (done_mask.load() & (1ull << dev)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done_mask.fetch_or(1ull << dev);
}

int run_engine(sq_dtype d, const sq::RunSpec &spec, cudaStream_t st, char *err, size_t len) {
  if (!spec.dev_alloc) keep_pool_cached();
  switch (d) {
    case SQ_U32: return sq::engine_run_u32(spec, st, err, len);
    case SQ_U64: return sq::engine_run_u64(spec, st, err, len);
    default: return sq::engine_run_f32(spec, st, err, len);
  }
}

bool is_host_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// The device address of a page-locked host buffer (mapped into the device's
// address space), else NULL.
void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Where the first pass reads and the last pass writes, when not the sorted
// buffers themselves (NULL members: the buffers).
struct SrcFin {
  const void *skeys;
  const uint32_t *svals;
  void *fkeys;
  uint32_t *fvals;
};

__global__ void k_iota(uint32_t *v, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

struct DevBuf {
  void *p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

// Sorts one instance whose buffers are device memory.
sq_status sort_device(void *keys, uint32_t *vals, uint64_t n, sq_dtype dtype, uint64_t seed, cudaStream_t st,
                      const sq_sort_opts *opts, const SrcFin *io = nullptr) {
  const uint32_t cutoff = (opts && opts->cutoff) ? opts->cutoff : cutoff_for(dtype, n);
  const size_t w = key_bytes(dtype);
  keep_pool_cached();
  DevBuf scratch, iota;
  scratch.st = iota.st = st;
  const size_t dk_bytes = (std::max<size_t>(n, 1) * w + 255) & ~(size_t)255;
  const size_t dv_bytes = (std::max<size_t>(n, 1) * 4 + 255) & ~(size_t)255;
  cudaError_t e = cudaMallocAsync(&scratch.p, dk_bytes + dv_bytes + std::max<size_t>(n, 1), st);
  if (e != cudaSuccess) return fail(SQ_ERR_NOMEM, "scratch allocation of %llu elements failed: %s",
                                    (unsigned long long)n, cudaGetErrorString(e));
  uint32_t *v = vals;
  if (!v) {
    e = cudaMallocAsync(&iota.p, std::max<size_t>(n, 1) * 4, st);
    if (e != cudaSuccess) return fail(SQ_ERR_NOMEM, "payload allocation failed: %s", cudaGetErrorString(e));
    v = (uint32_t *)iota.p;
    k_iota<<<std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, 4096)), 256, 0, st>>>(v, n);
  }
  sq::InstSpec is{};
  is.keys = keys;
  is.vals = v;
  is.dkeys = scratch.p;
  is.dvals = (uint32_t *)((char *)scratch.p + dk_bytes);
  is.tags = (uint8_t *)scratch.p + dk_bytes + dv_bytes;
  if (io) {
    is.skeys = io->skeys;
    is.svals = io->svals;
    is.fkeys = io->fkeys;
    is.fvals = io->fvals;
  }
  is.n = n;
  is.seed = seed;
  is.variant = opts ? opts->variant : 0;
  sq::RunSpec spec;
  memset(&spec, 0, sizeof(spec));
  spec.inst = &is;
  spec.ninst = 1;
  spec.cutoff = cutoff;
  spec.graph = graph_for(false);
  spec.async = !(opts && opts->trace && opts->trace_cap);  // (with graph rounds only)
  std::vector<sq::TraceOut> tr;
  if (opts && opts->trace && opts->trace_cap) {
    tr.resize(opts->trace_cap);
    spec.trace = tr.data();
    spec.trace_cap = opts->trace_cap;
    spec.trace_count = opts->trace_count;
  }
  char err[400] = {0};
  const int rc = run_engine(dtype, spec, st, err, sizeof(err));
  if (rc) return fail((sq_status)rc, "sort: %s", err);
  if (!tr.empty()) {
    const uint32_t got = opts->trace_count ? std::min(*opts->trace_count, opts->trace_cap) : opts->trace_cap;
    for (uint32_t i = 0; i < got; i++) {
      sq_trace_rec &o = opts->trace[i];
      o.off = tr[i].off;
      o.n = tr[i].n;
      o.m = tr[i].m;
      o.hash = tr[i].hash;
      o.depth = tr[i].depth;
      o.kind = tr[i].kind;
      o.attempts = tr[i].attempts;
      o.index = tr[i].index;
    }
  }
  return SQ_OK;
}

}  // namespace

namespace sq {
void api_set_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

// Argument checks of the stand-alone SkewTranspose entry points: clears the
// calling thread's error message, then returns SQ_OK or the first failure
// (with its message set).
sq_status api_check_skew_args(const sq_skew_buf *buf, uint64_t rows, uint64_t cols) {
  g_err[0] = 0;
  if (!buf) return fail(SQ_ERR_INVALID, "buf is NULL");
  if (!dtype_ok(buf->dtype)) return fail(SQ_ERR_INVALID, "bad dtype %d", (int)buf->dtype);
  const uint64_t n = buf->n, k = buf->k;
  if (rows == 0 || cols == 0 || n > rows * cols || n >= (1ull << 32) || rows >= (1ull << 32) ||
      cols >= (1ull << 32))
    return fail(SQ_ERR_INVALID, "bad shape: n=%llu rows=%llu cols=%llu", (unsigned long long)n,
                (unsigned long long)rows, (unsigned long long)cols);
  if (k == 0 || k > (uint64_t)engine_max_pivots(buf->dtype) + 1)
    return fail(SQ_ERR_INVALID, "k = %llu outside [1, %u]", (unsigned long long)k, engine_max_pivots(buf->dtype) + 1);
  if (!buf->bucket_start_out || (n && (!buf->keys_in || !buf->vals_in || !buf->keys_out || !buf->vals_out)) ||
      (k > 1 && (!buf->pivot_keys || !buf->pivot_vals)))
    return fail(SQ_ERR_INVALID, "null buffer");
  return SQ_OK;
}
}  // namespace sq

extern "C" {

const char *sq_last_error(void) { return g_err; }

uint32_t sq_max_leaf(sq_dtype dtype) { return dtype_ok(dtype) ? sq::engine_max_leaf(dtype) : 0; }

uint64_t sq_max_n(sq_dtype dtype) { return dtype_ok(dtype) ? sq::engine_max_n(dtype) : 0; }

sq_status sq_set_cutoff(sq_dtype dtype, uint32_t cutoff) {
  if (!dtype_ok(dtype)) return fail(SQ_ERR_INVALID, "bad dtype %d", (int)dtype);
  if (cutoff != 0 && (cutoff < 2 || cutoff > sq::engine_max_leaf(dtype)))
    return fail(SQ_ERR_INVALID, "cutoff %u outside [2, %u]", cutoff, sq::engine_max_leaf(dtype));
  g_cutoff[dtype].store(cutoff);
  return SQ_OK;
}

uint32_t sq_get_cutoff(sq_dtype dtype) { return dtype_ok(dtype) ? default_cutoff(dtype) : 0; }

sq_status sq_set_cutoff_table(sq_dtype dtype, const uint32_t *cutoff_by_log2n, uint32_t count) {
  if (!dtype_ok(dtype)) return fail(SQ_ERR_INVALID, "bad dtype %d", (int)dtype);
  if (count > 64 || (count && !cutoff_by_log2n)) return fail(SQ_ERR_INVALID, "table of %u entries", count);
  for (uint32_t i = 0; i < count; i++)
    if (cutoff_by_log2n[i] != 0 && (cutoff_by_log2n[i] < 2 || cutoff_by_log2n[i] > sq::engine_max_leaf(dtype)))
      return fail(SQ_ERR_INVALID, "table entry %u: cutoff %u outside [2, %u]", i, cutoff_by_log2n[i],
                  sq::engine_max_leaf(dtype));
  for (uint32_t i = 0; i < 64; i++) g_cutoff_table[dtype][i].store(i < count ? cutoff_by_log2n[i] : 0);
  return SQ_OK;
}

uint32_t sq_cutoff_for(sq_dtype dtype, uint64_t n) { return dtype_ok(dtype) ? cutoff_for(dtype, n) : 0; }

sq_status sq_set_launch_mode(sq_launch_mode mode) {
  if (mode != SQ_LAUNCH_HOST && mode != SQ_LAUNCH_GRAPH && mode != SQ_LAUNCH_AUTO)
    return fail(SQ_ERR_INVALID, "bad launch mode %d", (int)mode);
  g_launch_mode.store(mode);
  return SQ_OK;
}

sq_launch_mode sq_get_launch_mode(void) { return (sq_launch_mode)g_launch_mode.load(); }

sq_status sq_set_radix_classes(sq_dtype dtype, uint32_t mask) {
  g_err[0] = 0;
  if (!dtype_ok(dtype)) return fail(SQ_ERR_INVALID, "bad dtype %d", (int)dtype);
  if (dtype == SQ_U64 && (mask & sq::kRadixClassesAll))
    return fail(SQ_ERR_INVALID, "uint64 keys have no radix base case");
  sq::engine_set_radix_classes(dtype, mask);
  return SQ_OK;
}

uint32_t sq_get_radix_classes(sq_dtype dtype) { return dtype_ok(dtype) ? sq::engine_get_radix_classes(dtype) : 0u; }

sq_status sq_sort_ex(void *keys, uint32_t *vals, uint64_t n, sq_dtype dtype, uint64_t seed, sq_stream_t stream,
                     const sq_sort_opts *opts) {
  g_err[0] = 0;
  if (!dtype_ok(dtype)) return fail(SQ_ERR_INVALID, "bad dtype %d", (int)dtype);
  if (n > sq_max_n(dtype))
    return fail(SQ_ERR_INVALID, "n = %llu exceeds sq_max_n = %llu", (unsigned long long)n,
                (unsigned long long)sq_max_n(dtype));
  if (n && !keys) return fail(SQ_ERR_INVALID, "keys is NULL");
  if (opts && opts->cutoff && (opts->cutoff < 2 || opts->cutoff > sq::engine_max_leaf(dtype)))
    return fail(SQ_ERR_INVALID, "cutoff %u outside [2, %u]", opts->cutoff, sq::engine_max_leaf(dtype));
  if (opts && opts->trace_cap && !opts->trace) return fail(SQ_ERR_INVALID, "trace_cap without trace buffer");
  if (opts && opts->variant > SQ_APPENDIX) return fail(SQ_ERR_INVALID, "unknown variant %u", opts->variant);
  if (opts && opts->variant == SQ_APPENDIX) {
    if (dtype == SQ_F32) return fail(SQ_ERR_INVALID, "the appendix variant sorts integer keys");
    if ((opts->cutoff && opts->cutoff < 8) || (!opts->cutoff && cutoff_for(dtype, n) < 8))
      return fail(SQ_ERR_INVALID, "the appendix variant needs a cutoff of at least 8");
    const uint64_t p = sq::engine_max_pivots(dtype), vmax = (p + 1) * (p + 1);
    if (n >= vmax)
      return fail(SQ_ERR_INVALID, "n = %llu: the appendix variant takes n < %llu", (unsigned long long)n,
                  (unsigned long long)vmax);
  }
  if (opts && opts->trace_count) *opts->trace_count = 0;
  cudaStream_t st = (cudaStream_t)stream;
  {  // an error latched by an earlier asynchronous call on this stream comes first
    char perr[200] = {0};
    const int prc = sq::engine_poll(st, perr, sizeof(perr));
    if (prc) return fail((sq_status)prc, "%s", perr);
  }
  if (n == 0) return SQ_OK;
  const size_t w = key_bytes(dtype);
  const bool hk = is_host_ptr(keys), hv = vals && is_host_ptr(vals);
  if (!hk && !hv) return sort_device(keys, vals, n, dtype, seed, st, opts);
  cudaError_t e;
  void *mk = hk ? mapped_host(keys) : nullptr;
  uint32_t *mv = hv ? (uint32_t *)mapped_host(vals) : nullptr;
  if (hk && mk && (!vals || mv)) {
    // page-locked host buffers: the first pass (the root's column sorts, or
    // a single leaf) reads them and the last pass (the final leaves) writes
    // them, through the mapping; device memory holds only the rounds between
    DevBuf ak, av;
    ak.st = av.st = st;
    if ((e = cudaMallocAsync(&ak.p, n * w, st)) != cudaSuccess)
      return fail(SQ_ERR_NOMEM, "device keys: %s", cudaGetErrorString(e));
    if (vals && (e = cudaMallocAsync(&av.p, n * 4, st)) != cudaSuccess)
      return fail(SQ_ERR_NOMEM, "device vals: %s", cudaGetErrorString(e));
    const SrcFin io{mk, mv, mk, mv};
    const sq_status s = sort_device(ak.p, vals ? (uint32_t *)av.p : nullptr, n, dtype, seed, st, opts, &io);
    if (s != SQ_OK) return s;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(SQ_ERR_CUDA, "%s", cudaGetErrorString(e));
    return SQ_OK;
  }
  // other host buffers: staged through device memory
  DevBuf dk, dv;
  dk.st = dv.st = st;
  void *k = keys;
  uint32_t *v = vals;
  if (hk) {
    if ((e = cudaMallocAsync(&dk.p, n * w, st)) != cudaSuccess)
      return fail(SQ_ERR_NOMEM, "staging keys: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(dk.p, keys, n * w, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return fail(SQ_ERR_CUDA, "copy keys in: %s", cudaGetErrorString(e));
    k = dk.p;
  }
  if (hv) {
    if ((e = cudaMallocAsync(&dv.p, n * 4, st)) != cudaSuccess)
      return fail(SQ_ERR_NOMEM, "staging vals: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(dv.p, vals, n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return fail(SQ_ERR_CUDA, "copy vals in: %s", cudaGetErrorString(e));
    v = (uint32_t *)dv.p;
  }
  const sq_status s = sort_device(k, v, n, dtype, seed, st, opts);
  if (s != SQ_OK) return s;
  if (hk && (e = cudaMemcpyAsync(keys, dk.p, n * w, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(SQ_ERR_CUDA, "copy keys out: %s", cudaGetErrorString(e));
  if (hv && (e = cudaMemcpyAsync(vals, dv.p, n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail(SQ_ERR_CUDA, "copy vals out: %s", cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(SQ_ERR_CUDA, "%s", cudaGetErrorString(e));
  return SQ_OK;
}

sq_status sq_sync(sq_stream_t stream) {
  g_err[0] = 0;
  char err[200] = {0};
  const int rc = sq::engine_sync((cudaStream_t)stream, err, sizeof(err));
  if (rc) return fail((sq_status)rc, "%s", err);
  return SQ_OK;
}

sq_status sq_sort(void *keys, uint32_t *vals, uint64_t n, sq_dtype dtype, uint64_t seed, sq_stream_t stream) {
  return sq_sort_ex(keys, vals, n, dtype, seed, stream, nullptr);
}

sq_status sq_skew_transpose(const sq_skew_buf *buf, uint64_t rows, uint64_t cols, sq_stream_t stream) {
  const sq_status chk = sq::api_check_skew_args(buf, rows, cols);
  if (chk != SQ_OK) return chk;
  const uint64_t n = buf->n, k = buf->k;
  sq::InstSpec is{};
  is.keys = buf->keys_out;
  is.vals = buf->vals_out;
  is.dkeys = const_cast<void *>(buf->keys_in);
  is.dvals = const_cast<uint32_t *>(buf->vals_in);
  is.n = n;
  is.seed = 0;
  DevBuf tags;  // the count's bucket of every element, read by the SkewTranspose
  tags.st = (cudaStream_t)stream;
  keep_pool_cached();
  if (cudaMallocAsync(&tags.p, std::max<uint64_t>(n, 1), (cudaStream_t)stream) != cudaSuccess)
    return fail(SQ_ERR_NOMEM, "tag scratch of %llu bytes", (unsigned long long)n);
  is.tags = (uint8_t *)tags.p;
  sq::RunSpec spec;
  memset(&spec, 0, sizeof(spec));
  spec.inst = &is;
  spec.ninst = 1;
  spec.cutoff = 2;
  spec.skew_only = 1;
  spec.rows = rows;
  spec.cols = cols;
  spec.k = k;
  spec.piv_keys = buf->pivot_keys;
  spec.piv_vals = buf->pivot_vals;
  spec.bucket_start = buf->bucket_start_out;
  char err[400] = {0};
  const int rc = run_engine(buf->dtype, spec, (cudaStream_t)stream, err, sizeof(err));
  if (rc) return fail((sq_status)rc, "skew_transpose: %s", err);
  return SQ_OK;
}

sq_status sq_sort_batch(const sq_sort_desc *descs, uint32_t count, sq_stream_t stream) {
  g_err[0] = 0;
  if (count && !descs) return fail(SQ_ERR_INVALID, "descs is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  {  // an error latched by an earlier asynchronous call on this stream comes first
    char perr[200] = {0};
    const int prc = sq::engine_poll(st, perr, sizeof(perr));
    if (prc) return fail((sq_status)prc, "%s", perr);
  }
  for (uint32_t i = 0; i < count; i++) {
    if (!dtype_ok(descs[i].dtype)) return fail(SQ_ERR_INVALID, "desc %u: bad dtype", i);
    if (descs[i].n > sq_max_n(descs[i].dtype)) return fail(SQ_ERR_INVALID, "desc %u: n too large", i);
    if (descs[i].n && !descs[i].keys) return fail(SQ_ERR_INVALID, "desc %u: keys is NULL", i);
    if (descs[i].n && (is_host_ptr(descs[i].keys) || (descs[i].vals && is_host_ptr(descs[i].vals))))
      return fail(SQ_ERR_INVALID, "desc %u: sq_sort_batch takes device buffers", i);
  }
  for (int d = 0; d < 3; d++) {
    std::vector<uint32_t> ids;
    uint64_t total = 0, nnull = 0;
    for (uint32_t i = 0; i < count; i++)
      if (descs[i].dtype == d) {
        ids.push_back(i);
        total += descs[i].n;
        if (!descs[i].vals) nnull += descs[i].n;
      }
    if (ids.empty()) continue;
    const size_t w = key_bytes((sq_dtype)d);
    // scratch D for every instance in one allocation, plus payloads for NULL vals
    std::vector<size_t> koff(ids.size()), voff(ids.size()), ioff(ids.size());
    size_t off = 0;
    auto carve = [&](size_t b) {
      const size_t o = off;
      off += (b + 255) & ~(size_t)255;
      return o;
    };
    std::vector<size_t> toff(ids.size());
    for (size_t q = 0; q < ids.size(); q++) {
      const uint64_t n = descs[ids[q]].n;
      koff[q] = carve(n * w);
      voff[q] = carve(n * 4);
      ioff[q] = descs[ids[q]].vals ? 0 : carve(n * 4);
      toff[q] = carve(n);
    }
    DevBuf slab;
    slab.st = st;
    keep_pool_cached();
    cudaError_t e = cudaMallocAsync(&slab.p, std::max<size_t>(off, 256), st);
    if (e != cudaSuccess) return fail(SQ_ERR_NOMEM, "batch scratch: %s", cudaGetErrorString(e));
    std::vector<sq::InstSpec> is(ids.size());
    for (size_t q = 0; q < ids.size(); q++) {
      const sq_sort_desc &ds = descs[ids[q]];
      is[q].keys = ds.keys;
      is[q].vals = ds.vals;
      if (!ds.vals) {
        is[q].vals = (uint32_t *)((char *)slab.p + ioff[q]);
        if (ds.n) k_iota<<<std::max<uint64_t>(1, std::min<uint64_t>((ds.n + 255) / 256, 4096)), 256, 0, st>>>(
            is[q].vals, ds.n);
      }
      is[q].dkeys = (char *)slab.p + koff[q];
      is[q].dvals = (uint32_t *)((char *)slab.p + voff[q]);
      is[q].tags = (uint8_t *)slab.p + toff[q];
      is[q].n = ds.n;
      is[q].seed = ds.seed;
      is[q].cutoff = cutoff_for((sq_dtype)d, ds.n);
    }
    sq::RunSpec spec;
    memset(&spec, 0, sizeof(spec));
    spec.inst = is.data();
    spec.ninst = (uint32_t)is.size();
    spec.cutoff = default_cutoff((sq_dtype)d);
    spec.graph = graph_for(true);
    spec.async = 1;  // (with graph rounds only)
    char err[400] = {0};
    const int rc = run_engine((sq_dtype)d, spec, st, err, sizeof(err));
    if (rc) return fail((sq_status)rc, "batch: %s", err);
    (void)nnull;
    (void)total;
  }
  return SQ_OK;
}

void sq_stats_get(sq_stats *out) {
  if (!out) return;
  sq::EngineStats s;
  sq::engine_stats_get(&s);
  for (int f = 0; f < 9; f++) {
    out->launches[f] = s.launches[f];
    out->ms[f] = s.ms[f];
    out->bytes[f] = s.bytes[f];
  }
  out->rounds = s.rounds;
  out->nodes = s.nodes;
  out->sorts = s.sorts;
}

void sq_stats_reset(void) { sq::engine_stats_reset(); }

void sq_set_profiling(int on) { sq::engine_set_profiling(on); }

}  // extern "C"
