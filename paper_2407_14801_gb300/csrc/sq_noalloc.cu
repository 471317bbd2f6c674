// SkewTranspose that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a
// SkewTranspose: a process whose frameworks have already reserved the whole
// device for their own caching pools, or a latency-critical path that must
// not call cudaMalloc / cudaFree (which can synchronise the device, or fail
// under memory pressure at an arbitrary moment).  This entry point does the
// same work as sq_skew_transpose but takes all its scratch (the per-node
// metadata, work lists and status words) from one statically sized device
// array.  The array belongs to this file's module, which the CUDA runtime
// loads (and so reserves the array) on the first call on each device.
#include <cstdio>
#include <cstring>

#include "../../include/squaresort.h"
#include "sq_engine.h"

namespace {

// Scratch shared by every call on a device.  Reserved on a device by the
// first call there; held until the process exits.
constexpr size_t kNoAllocScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

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

namespace sq {
sq_status api_check_skew_args(const sq_skew_buf *buf, uint64_t rows, uint64_t cols);  // (sq_api.cu)
}

extern "C" sq_status sq_skew_transpose_noalloc(const sq_skew_buf *buf, uint64_t rows, uint64_t cols,
                                                sq_stream_t stream) {
  char msg[256];
  const sq_status chk = sq::api_check_skew_args(buf, rows, cols);  // the regular call's checks and messages
  if (chk != SQ_OK) return chk;
  const uint64_t n = buf->n, k = buf->k;
  const uint64_t need = sq::engine_skew_scratch_bytes(buf->dtype, n, cols, k);
  if (need > kNoAllocScratchBytes) {
    snprintf(msg, sizeof(msg),
             "this shape needs %llu bytes of scratch; sq_skew_transpose_noalloc holds %llu "
             "(use sq_skew_transpose)",
             (unsigned long long)need, (unsigned long long)kNoAllocScratchBytes);
    return nfail(SQ_ERR_INVALID, msg);
  }
  // The array's device address in the current device's context.  Host code
  // sees only a host-side stand-in under the array's name, so the address is
  // asked for on every call (cheap once the module is loaded; no address is
  // kept across a device reset or a context change).  On a device's first
  // call this loads the module, which is where the array is reserved.
  void *base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess || !base) {
    cudaGetLastError();  // leave no stale error for the next, unrelated runtime check
    snprintf(msg, sizeof(msg), "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return nfail(SQ_ERR_CUDA, msg);
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
