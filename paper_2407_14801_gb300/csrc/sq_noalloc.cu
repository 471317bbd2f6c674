// SkewTranspose that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a
// SkewTranspose: a process whose frameworks have already reserved the whole
// device for their own caching pools, or a latency-critical path that must
// not call cudaMalloc / cudaFree (which can synchronise the device, or fail
// under memory pressure at an arbitrary moment).  This entry point does the
// same work as sq_skew_transpose but takes all its scratch (the per-node
// metadata, work lists and status words) from one statically sized device
// array that the library carries from the moment it is loaded.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/squaresort.h"
#include "sq_engine.h"

namespace {

// Scratch shared by every call on a device.  Every GPU that loads this
// library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device (host code only
// sees a host-side stand-in under the array's name).
std::mutex g_mu;
void *g_scratch_ptr[128] = {};

struct Bump {
  char *base;
  size_t size, used;
};

void *bump_alloc(void *ctx, size_t bytes) {
  Bump *b = static_cast<Bump *>(ctx);
  const size_t need = (bytes + 255) & ~(size_t)255;
  if (b->used + need > b->size) return nullptr;
  void *p = b->base + b->used;
  b->used += need;
  return p;
}
void bump_free(void *, void *) {}

sq_status nfail(sq_status s, const char *msg) {
  sq::api_set_error(msg);
  return s;
}

}  // namespace

extern "C" sq_status sq_skew_transpose_noalloc(const sq_skew_buf *buf, uint64_t rows, uint64_t cols,
                                                sq_stream_t stream) {
  char msg[256];
  if (!buf) return nfail(SQ_ERR_INVALID, "buf is NULL");
  if (buf->dtype < 0 || buf->dtype > 2) return nfail(SQ_ERR_INVALID, "bad dtype");
  const uint64_t n = buf->n, k = buf->k;
  if (rows == 0 || cols == 0 || n > rows * cols || n >= (1ull << 32) || rows >= (1ull << 32) ||
      cols >= (1ull << 32))
    return nfail(SQ_ERR_INVALID, "bad shape");
  if (k == 0 || k > (uint64_t)sq::engine_max_pivots(buf->dtype) + 1) return nfail(SQ_ERR_INVALID, "bad k");
  if (!buf->bucket_start_out || (n && (!buf->keys_in || !buf->vals_in || !buf->keys_out || !buf->vals_out)) ||
      (k > 1 && (!buf->pivot_keys || !buf->pivot_vals)))
    return nfail(SQ_ERR_INVALID, "null buffer");
  const uint64_t need = sq::engine_skew_scratch_bytes(buf->dtype, n, cols, k);
  if (need > kNoAllocScratchBytes) {
    snprintf(msg, sizeof(msg),
             "this shape needs %llu bytes of scratch; sq_skew_transpose_noalloc holds %llu "
             "(use sq_skew_transpose)",
             (unsigned long long)need, (unsigned long long)kNoAllocScratchBytes);
    return nfail(SQ_ERR_INVALID, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) return nfail(SQ_ERR_CUDA, "cudaGetDevice failed");
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {  // first call on this device (current device)
      e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        snprintf(msg, sizeof(msg), "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return nfail(SQ_ERR_CUDA, msg);
      }
    }
    base = g_scratch_ptr[dev];
  }
  Bump bump{static_cast<char *>(base), kNoAllocScratchBytes, 0};
  alignas(64) unsigned char readback[512];
  sq::InstSpec is{};
  is.keys = buf->keys_out;
  is.vals = buf->vals_out;
  is.dkeys = const_cast<void *>(buf->keys_in);
  is.dvals = const_cast<uint32_t *>(buf->vals_in);
  is.n = n;
  is.seed = 0;
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
  spec.dev_alloc = bump_alloc;
  spec.dev_free = bump_free;
  spec.alloc_ctx = &bump;
  spec.host_readback = readback;
  char err[256] = {0};
  int rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (buf->dtype) {
    case SQ_U32: rc = sq::engine_run_u32(spec, st, err, sizeof(err)); break;
    case SQ_U64: rc = sq::engine_run_u64(spec, st, err, sizeof(err)); break;
    default: rc = sq::engine_run_f32(spec, st, err, sizeof(err)); break;
  }
  if (rc) {
    snprintf(msg, sizeof(msg), "skew_transpose_noalloc: %s", err);
    return nfail((sq_status)rc, msg);
  }
  return SQ_OK;
}
