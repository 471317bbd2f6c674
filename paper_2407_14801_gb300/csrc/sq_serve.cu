// Serving loop: a FIFO of sort requests, a device memory pool bounded by an
// HBM budget, and one persistent engine session per key type, each with a
// copy-in and a copy-out stage (host thread + CUDA stream each).  Between any two recursion rounds a session admits the
// queued requests of its key type that fit (first come, first served within
// the type): their roots join the next round's work lists, so a request
// that arrives while others are on the GPU starts at the next round
// boundary and its kernels are the same launches as theirs (continuous
// batching).  A request leaves the session, and its result is copied back,
// as soon as the round in which its last leaf finished ends.
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
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
  bool stopping = false;
  std::vector<std::thread> workers;
  // one engine session per key type (a request joins its type's session)
  uint64_t total_n_cap[3] = {0, 0, 0};
  uint64_t inflight_n[3] = {0, 0, 0};
  uint32_t reserved[3] = {0, 0, 0};  // requests copied in or in flight
  std::deque<Req *> joinq[3];        // copied in, waiting for the next round boundary
  std::deque<Req *> outq[3];         // sorted, waiting to be copied out
  std::string open_error[3];
  bool open_failed[3] = {false, false, false};
  bool session_gone[3] = {false, false, false};
};

namespace {

// Engine scratch (node pool growth included) comes from the same pool as
// the requests' data.
void *pool_alloc(void *ctx, size_t bytes) {
  sq_server *s = (sq_server *)ctx;
  std::lock_guard<std::mutex> lk(s->mu);
  uint64_t off = 0;
  if (!s->pool.alloc(al(bytes), &off)) return nullptr;
  return s->slab + off;
}
void pool_free(void *ctx, void *p) {
  sq_server *s = (sq_server *)ctx;
  std::lock_guard<std::mutex> lk(s->mu);
  s->pool.release((uint64_t)((char *)p - s->slab));
}

__global__ void k_serve_iota(uint32_t *v, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

// The key type's cutoffs: the server's, or the range of the tuned table.
void cutoff_range(sq_server *s, int d, uint32_t &lo, uint32_t &hi) {
  if (s->cutoff) {
    lo = hi = s->cutoff;
    return;
  }
  lo = hi = sq_get_cutoff((sq_dtype)d);
  for (int lg = 0; lg < 63; lg++) {
    const uint32_t c = sq_cutoff_for((sq_dtype)d, 1ull << lg);
    lo = std::min(lo, c);
    hi = std::max(hi, c);
  }
}

void finish(sq_server *s, Req *r, sq_status st) {
  // caller holds s->mu
  r->result = st;
  r->latency = now_s() - r->t0;
  r->done = true;
  s->pool.release(r->off);
  s->inflight_n[r->d.dtype] -= r->d.n;
  s->reserved[r->d.dtype]--;
}

// The InstSpec of a request's pool range: keys | vals | D keys | D vals | tags.
sq::InstSpec layout(sq_server *s, Req *r) {
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
  x.cutoff = s->cutoff ? s->cutoff : sq_cutoff_for(r->d.dtype, n);
  return x;
}

// Copy-in stage of one key type: takes queued requests of the type in order
// while a pool range, an engine slot and room under the type's in-flight
// limit are free, copies them in on its own stream and hands them to the
// session thread, which admits them at its next round boundary.
void copier_in(sq_server *s, int d) {
  cudaSetDevice(s->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  const uint64_t w = kbytes((sq_dtype)d);
  for (;;) {
    Req *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto head = [&]() -> Req * {
        for (Req *q : s->queue)
          if (q->d.dtype == d) return q;
        return nullptr;
      };
      auto can_take = [&](Req *q) {
        return q && (s->session_gone[d] ||
                     (s->reserved[d] < s->max_inflight && s->inflight_n[d] + q->d.n <= s->total_n_cap[d] &&
                      s->pool.fits(q->data)));
      };
      s->cv.wait(lk, [&] { return (s->stopping && !head()) || can_take(head()); });
      r = head();
      if (!r) break;  // stopping, nothing of this type queued
      for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == r) {
          s->queue.erase(it);
          break;
        }
      if (s->session_gone[d]) {
        r->result = SQ_ERR_NOMEM;
        r->latency = now_s() - r->t0;
        r->done = true;
        continue;
      }
      if (!s->pool.alloc(r->data, &r->off)) {  // raced with another allocation: queue head again
        s->queue.push_front(r);
        continue;
      }
      s->inflight_n[d] += r->d.n;
      s->reserved[d]++;
    }
    const sq::InstSpec x = layout(s, r);
    const uint64_t n = r->d.n;
    cudaError_t e = cudaMemcpyAsync(x.keys, r->d.keys, n * w, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      if (r->d.vals)
        e = cudaMemcpyAsync(x.vals, r->d.vals, n * 4, cudaMemcpyHostToDevice, st);
      else
        k_serve_iota<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 4096), 256, 0, st>>>(x.vals, n);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::lock_guard<std::mutex> lk(s->mu);
    if (e != cudaSuccess)
      finish(s, r, SQ_ERR_CUDA);
    else
      s->joinq[d].push_back(r);
    s->cv.notify_all();
  }
  cudaStreamDestroy(st);
}

// Copy-out stage: results of the requests the session finished.
void copier_out(sq_server *s, int d) {
  cudaSetDevice(s->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  const uint64_t w = kbytes((sq_dtype)d);
  for (;;) {
    std::vector<Req *> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return !s->outq[d].empty() || (s->stopping && s->reserved[d] == 0); });
      if (s->outq[d].empty()) break;
      batch.assign(s->outq[d].begin(), s->outq[d].end());
      s->outq[d].clear();
    }
    std::vector<sq_status> res(batch.size(), SQ_OK);
    for (size_t i = 0; i < batch.size(); i++) {
      Req *r = batch[i];
      const uint64_t n = r->d.n;
      char *base = s->slab + r->off;
      if (cudaMemcpyAsync(r->d.keys, base, n * w, cudaMemcpyDeviceToHost, st) != cudaSuccess) res[i] = SQ_ERR_CUDA;
      if (r->d.vals && cudaMemcpyAsync(r->d.vals, base + al(n * w), n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        res[i] = SQ_ERR_CUDA;
    }
    const bool ok = cudaStreamSynchronize(st) == cudaSuccess;
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < batch.size(); i++) finish(s, batch[i], ok ? res[i] : SQ_ERR_CUDA);
    s->cv.notify_all();
  }
  cudaStreamDestroy(st);
}

// Session stage of one key type: between rounds, admit what the copy-in
// stage finished (each takes a free slot); run one round; pass the requests
// that completed in it to the copy-out stage.
void worker(sq_server *s, int d) {
  cudaSetDevice(s->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  sq::SessionSpec sp;
  memset(&sp, 0, sizeof(sp));
  sp.total_n_cap = s->total_n_cap[d];
  sp.ninst_cap = s->max_inflight;
  cutoff_range(s, d, sp.cutoff_min, sp.cutoff_max);
  sp.dev_alloc = pool_alloc;
  sp.dev_free = pool_free;
  sp.alloc_ctx = s;
  void *sess = nullptr;
  char err[256] = {0};
  if (sq::session_open(d, sp, st, &sess, err, sizeof(err)) != 0) sess = nullptr;
  if (!sess) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->open_failed[d] = true;
    s->session_gone[d] = true;
    s->open_error[d] = err;
    for (Req *r : s->joinq[d]) finish(s, r, SQ_ERR_NOMEM);
    s->joinq[d].clear();
    s->cv.notify_all();
  }
  std::vector<Req *> slot_req(s->max_inflight, nullptr);
  std::vector<uint32_t> free_slots;
  for (uint32_t i = s->max_inflight; i-- > 0;) free_slots.push_back(i);
  while (sess) {
    std::vector<Req *> join;
    const bool busy = sq::session_busy(d, sess);
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (!busy)
        s->cv.wait(lk, [&] { return !s->joinq[d].empty() || (s->stopping && s->reserved[d] == 0); });
      if (!busy && s->joinq[d].empty()) break;  // stopping and drained
      while (!s->joinq[d].empty() && !free_slots.empty()) {
        join.push_back(s->joinq[d].front());
        s->joinq[d].pop_front();
      }
    }
    for (Req *r : join) {
      const uint32_t slot = free_slots.back();
      free_slots.pop_back();
      const int rc = sq::session_admit(d, sess, layout(s, r), slot, err, sizeof(err));
      if (rc) {
        std::lock_guard<std::mutex> lk(s->mu);
        finish(s, r, (sq_status)rc);
        free_slots.push_back(slot);
        s->cv.notify_all();
      } else {
        slot_req[slot] = r;
      }
    }
    if (!sq::session_busy(d, sess)) continue;
    std::vector<uint32_t> done;
    const int rc = sq::session_step(d, sess, done, err, sizeof(err));
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc) {  // the session's state is lost: fail what it holds and start afresh
      for (uint32_t i = 0; i < s->max_inflight; i++)
        if (slot_req[i]) {
          finish(s, slot_req[i], (sq_status)rc);
          slot_req[i] = nullptr;
        }
      free_slots.clear();
      for (uint32_t i = s->max_inflight; i-- > 0;) free_slots.push_back(i);
      sq::session_close(d, sess);
      sess = nullptr;
      if (sq::session_open(d, sp, st, &sess, err, sizeof(err)) != 0) {
        sess = nullptr;
        s->session_gone[d] = true;
        for (Req *r : s->joinq[d]) finish(s, r, SQ_ERR_NOMEM);
        s->joinq[d].clear();
      }
      s->cv.notify_all();
      continue;
    }
    for (uint32_t slot : done) {
      Req *r = slot < slot_req.size() ? slot_req[slot] : nullptr;
      if (!r) continue;
      slot_req[slot] = nullptr;
      free_slots.push_back(slot);
      s->outq[d].push_back(r);
    }
    if (!done.empty()) s->cv.notify_all();
  }
  if (sess) sq::session_close(d, sess);
  cudaStreamSynchronize(st);
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
  // every key type may hold up to half the budget's worth of elements in
  // flight (data of 2(w+4)+1 bytes an element), as long as its session's
  // work lists -- planned for that many -- take at most a tenth of the budget
  for (int d = 0; d < 3; d++) {
    sq::SessionSpec sp;
    memset(&sp, 0, sizeof(sp));
    sp.ninst_cap = s->max_inflight;
    cutoff_range(s, d, sp.cutoff_min, sp.cutoff_max);
    sp.total_n_cap = hbm_budget_bytes / 2 / (2 * (kbytes((sq_dtype)d) + 4) + 3);
    while (sp.total_n_cap > 4096 && sq::session_scratch_bytes(d, sp) > hbm_budget_bytes / 10) sp.total_n_cap /= 2;
    s->total_n_cap[d] = sp.total_n_cap;
  }
  for (int d = 0; d < 3; d++) {  // copies from and to pageable host memory: two threads a direction
    s->workers.emplace_back(worker, s, d);
    for (int c = 0; c < 2; c++) {
      s->workers.emplace_back(copier_in, s, d);
      s->workers.emplace_back(copier_out, s, d);
    }
  }
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
  if (r->data > s->pool.capacity() / 2 || desc->n > s->total_n_cap[desc->dtype]) {
    delete r;
    return sfail(SQ_ERR_BUDGET, "request needs %llu bytes, at most half the budget (%llu) is available to one request",
                 (unsigned long long)al(data_bytes(*desc)), (unsigned long long)s->pool.capacity());
  }
  if (s->open_failed[desc->dtype]) {
    delete r;
    return sfail(SQ_ERR_NOMEM, "no engine for this key type: %s", s->open_error[desc->dtype].c_str());
  }
  if (s->stopping) {
    delete r;
    return sfail(SQ_ERR_INVALID, "server is stopping");
  }
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  *ticket = r->ticket;
  if (desc->n == 0) {  // nothing to sort
    r->done = true;
    return SQ_OK;
  }
  s->queue.push_back(r);
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
