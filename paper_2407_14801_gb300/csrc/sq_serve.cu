// Serving loop: a FIFO of sort requests, a device memory pool bounded by an
// HBM budget, and several sessions (host thread + CUDA stream each).  A free
// session admits every queued request that fits the pool (first come, first
// served) and runs them as one batch through the engine; the other sessions
// keep running theirs, so requests that arrive while others are on the GPU
// start as soon as a session and memory free up, and their kernels overlap
// on the device with the batches already running.
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/squaresort.h"
#include "sq_engine.h"
#include "sq_pool.h"

namespace {

sq_status sfail(sq_status s, const char *fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  sq::api_set_error(buf);
  return s;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t kbytes(sq_dtype d) { return d == SQ_U64 ? 8 : 4; }
uint64_t al(uint64_t b) { return (b + 255) & ~255ull; }

struct Req {
  uint64_t ticket;
  sq_sort_desc d;
  double t0 = 0, latency = 0;
  sq_status result = SQ_OK;
  bool done = false;
  uint64_t off = 0;  // data range in the pool: keys | vals | D keys | D vals
  uint64_t data = 0;
};

uint64_t data_bytes(const sq_sort_desc &d) {
  const uint64_t n = d.n, w = kbytes(d.dtype);
  return al(n * w) + al(n * 4) + al(n * w) + al(n * 4) + al(n) + 256;
}

}  // namespace

struct sq_server {
  int device = 0;
  uint32_t max_inflight = 4096, cutoff = 0;
  uint64_t budget = 0;
  char *slab = nullptr;
  sq::RangePool pool;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req *> queue;
  std::unordered_map<uint64_t, Req *> reqs;
  uint64_t next_ticket = 1;
  uint32_t inflight = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
};

namespace {

uint64_t scratch_need(sq_server *s, const std::vector<Req *> &b, int dtype) {
  uint64_t tot = 0;
  uint32_t cnt = 0, c = s->cutoff ? s->cutoff : sq_get_cutoff((sq_dtype)dtype), cmax = c;
  for (Req *r : b)
    if (r->d.dtype == dtype) {
      tot += r->d.n;
      cnt++;
      // work lists are sized for the smallest cutoff, leaf classes for the largest
      if (!s->cutoff) {
        const uint32_t ci = sq_cutoff_for((sq_dtype)dtype, r->d.n);
        c = std::min(c, ci);
        cmax = std::max(cmax, ci);
      }
    }
  if (!cnt) return 0;
  return sq::engine_scratch_bytes(dtype, tot, cnt, c, cmax) + 4096;
}

uint64_t batch_scratch(sq_server *s, const std::vector<Req *> &b) {
  uint64_t m = 0;  // dtype groups run one after another: the largest need
  for (int d = 0; d < 3; d++) m = std::max(m, scratch_need(s, b, d));
  return m;
}

struct Bump {
  char *base;
  uint64_t size, used;
};
void *bump_alloc(void *ctx, size_t bytes) {
  Bump *b = (Bump *)ctx;
  const uint64_t need = al(bytes);
  if (b->used + need > b->size) return nullptr;
  void *p = b->base + b->used;
  b->used += need;
  return p;
}
void bump_free(void *, void *) {}

void run_batch(sq_server *s, cudaStream_t st, std::vector<Req *> &batch, uint64_t soff, uint64_t ssize) {
  cudaError_t e = cudaSuccess;
  for (Req *r : batch) {  // copy in
    const uint64_t n = r->d.n, w = kbytes(r->d.dtype);
    char *base = s->slab + r->off;
    if (n && e == cudaSuccess) e = cudaMemcpyAsync(base, r->d.keys, n * w, cudaMemcpyHostToDevice, st);
    if (n && e == cudaSuccess && r->d.vals)
      e = cudaMemcpyAsync(base + al(n * w), r->d.vals, n * 4, cudaMemcpyHostToDevice, st);
  }
  std::vector<sq_status> st_of(batch.size(), e == cudaSuccess ? SQ_OK : SQ_ERR_CUDA);
  for (int d = 0; d < 3 && e == cudaSuccess; d++) {
    std::vector<sq::InstSpec> is;
    std::vector<size_t> who;
    for (size_t q = 0; q < batch.size(); q++) {
      Req *r = batch[q];
      if (r->d.dtype != d || r->d.n == 0) continue;
      const uint64_t n = r->d.n, w = kbytes(r->d.dtype);
      char *base = s->slab + r->off;
      sq::InstSpec x{};
      x.keys = base;
      x.vals = (uint32_t *)(base + al(n * w));
      x.dkeys = base + al(n * w) + al(n * 4);
      x.dvals = (uint32_t *)(base + al(n * w) + al(n * 4) + al(n * w));
      x.tags = (uint8_t *)(base + al(n * w) + al(n * 4) + al(n * w) + al(n * 4));
      x.n = n;
      x.seed = r->d.seed;
      x.cutoff = s->cutoff ? s->cutoff : sq_cutoff_for((sq_dtype)d, n);
      is.push_back(x);
      who.push_back(q);
    }
    if (is.empty()) continue;
    // payloads for requests without vals: the original index
    for (size_t q = 0; q < who.size(); q++)
      if (!batch[who[q]]->d.vals) {
        std::vector<uint32_t> iota(is[q].n);
        for (uint64_t i = 0; i < is[q].n; i++) iota[i] = (uint32_t)i;
        cudaMemcpyAsync(is[q].vals, iota.data(), 4 * is[q].n, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
      }
    Bump bump{s->slab + soff, ssize, 0};
    sq::RunSpec spec;
    memset(&spec, 0, sizeof(spec));
    spec.inst = is.data();
    spec.ninst = (uint32_t)is.size();
    spec.cutoff = s->cutoff ? s->cutoff : sq_get_cutoff((sq_dtype)d);
    spec.graph = sq_get_launch_mode() == SQ_LAUNCH_GRAPH;
    spec.dev_alloc = bump_alloc;
    spec.dev_free = bump_free;
    spec.alloc_ctx = &bump;
    char err[256] = {0};
    int rc = 0;
    switch (d) {
      case SQ_U32: rc = sq::engine_run_u32(spec, st, err, sizeof(err)); break;
      case SQ_U64: rc = sq::engine_run_u64(spec, st, err, sizeof(err)); break;
      default: rc = sq::engine_run_f32(spec, st, err, sizeof(err)); break;
    }
    if (rc)
      for (size_t q : who) st_of[q] = (sq_status)rc;
  }
  for (size_t q = 0; q < batch.size(); q++) {  // copy out
    Req *r = batch[q];
    const uint64_t n = r->d.n, w = kbytes(r->d.dtype);
    if (!n || st_of[q] != SQ_OK) continue;
    char *base = s->slab + r->off;
    if (cudaMemcpyAsync(r->d.keys, base, n * w, cudaMemcpyDeviceToHost, st) != cudaSuccess) st_of[q] = SQ_ERR_CUDA;
    if (r->d.vals && cudaMemcpyAsync(r->d.vals, base + al(n * w), n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      st_of[q] = SQ_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess)
    for (auto &x : st_of) x = SQ_ERR_CUDA;
  const double t1 = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  s->pool.release(soff);
  for (size_t q = 0; q < batch.size(); q++) {
    Req *r = batch[q];
    s->pool.release(r->off);
    r->result = st_of[q];
    r->latency = t1 - r->t0;
    r->done = true;
  }
  s->inflight -= (uint32_t)batch.size();
  s->cv.notify_all();
}

void worker(sq_server *s) {
  cudaSetDevice(s->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Req *> batch;
    uint64_t soff = 0, ssize = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->stopping) return true;
        if (s->queue.empty() || s->inflight >= s->max_inflight) return false;
        Req *f = s->queue.front();
        return s->pool.fits(f->data) && s->pool.largest_free() >= f->data + scratch_need(s, {f}, f->d.dtype);
      });
      if (s->stopping && s->queue.empty()) break;
      while (!s->queue.empty() && s->inflight + batch.size() < s->max_inflight) {
        Req *r = s->queue.front();
        if (!s->pool.alloc(r->data, &r->off)) break;
        batch.push_back(r);
        s->queue.pop_front();
      }
      // scratch for the batch; give back the newest requests until it fits
      while (!batch.empty()) {
        ssize = batch_scratch(s, batch);
        if (s->pool.alloc(ssize, &soff)) break;
        Req *r = batch.back();
        batch.pop_back();
        s->pool.release(r->off);
        s->queue.push_front(r);
      }
      s->inflight += (uint32_t)batch.size();
    }
    if (!batch.empty()) run_batch(s, st, batch, soff, ssize);
  }
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

sq_status sq_serve_create(sq_server **out, uint64_t hbm_budget_bytes, const sq_serve_opts *opts) {
  if (!out) return sfail(SQ_ERR_INVALID, "out is NULL");
  if (hbm_budget_bytes < (1ull << 20)) return sfail(SQ_ERR_INVALID, "budget below 1 MiB");
  sq_server *s = new sq_server();
  s->budget = hbm_budget_bytes;
  if (opts) {
    s->device = opts->device;
    if (opts->max_inflight) s->max_inflight = opts->max_inflight;
    s->cutoff = opts->cutoff;
  }
  cudaError_t e = cudaSetDevice(s->device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&s->slab, hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    return sfail(SQ_ERR_NOMEM, "pool of %llu bytes: %s", (unsigned long long)hbm_budget_bytes,
                 cudaGetErrorString(e));
  }
  s->pool.reset(hbm_budget_bytes);
  const int sessions = 4;
  for (int i = 0; i < sessions; i++) s->workers.emplace_back(worker, s);
  *out = s;
  return SQ_OK;
}

sq_status sq_serve_submit(sq_server *s, const sq_sort_desc *desc, uint64_t *ticket) {
  if (!s || !desc || !ticket) return sfail(SQ_ERR_INVALID, "null argument");
  if (desc->dtype < 0 || desc->dtype > 2) return sfail(SQ_ERR_INVALID, "bad dtype");
  if (desc->n > sq_max_n(desc->dtype)) return sfail(SQ_ERR_INVALID, "n too large");
  if (desc->n && !desc->keys) return sfail(SQ_ERR_INVALID, "keys is NULL");
  Req *r = new Req();
  r->d = *desc;
  r->data = data_bytes(*desc);
  r->t0 = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  const uint64_t need = r->data + scratch_need(s, {r}, desc->dtype) + 256;
  if (need > s->pool.capacity()) {
    delete r;
    return sfail(SQ_ERR_BUDGET, "request needs %llu bytes, budget is %llu", (unsigned long long)need,
                 (unsigned long long)s->pool.capacity());
  }
  if (s->stopping) {
    delete r;
    return sfail(SQ_ERR_INVALID, "server is stopping");
  }
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv.notify_all();
  return SQ_OK;
}

sq_status sq_serve_poll(sq_server *s, uint64_t ticket, sq_status *result, double *latency_s) {
  if (!s) return sfail(SQ_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(SQ_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  Req *r = it->second;
  if (!r->done) return SQ_PENDING;
  if (result) *result = r->result;
  if (latency_s) *latency_s = r->latency;
  s->reqs.erase(it);
  delete r;
  return SQ_OK;
}

sq_status sq_serve_destroy(sq_server *s) {
  if (!s) return sfail(SQ_ERR_INVALID, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv.notify_all();
  }
  for (auto &t : s->workers) t.join();
  for (auto &kv : s->reqs) delete kv.second;
  if (s->slab) cudaFree(s->slab);
  delete s;
  return SQ_OK;
}

}  // extern "C"
