// uint32 engine instantiation, plus the process-wide statistics.
#include "sq_engine.cuh"

namespace sq {

StatsBox &stats_box() {
  static StatsBox box;
  return box;
}

void engine_stats_get(EngineStats *out) {
  std::lock_guard<std::mutex> g(stats_box().mu);
  *out = stats_box().s;
}

void engine_stats_reset() {
  std::lock_guard<std::mutex> g(stats_box().mu);
  memset(&stats_box().s, 0, sizeof(EngineStats));
}

void engine_set_profiling(int on) { stats_box().profiling.store(on ? 1 : 0); }

// ---- asynchronous runs ------------------------------------------------------
// A fixed table of records in page-locked memory; each committed record has
// the event recorded after its copies.  A record's errors, once collected,
// wait in a per-stream latch for the stream's next poll or sync.
namespace {
constexpr int kPending = 256;
struct PendingMeta {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool used = false, committed = false;
  double key_bytes = 0;
  EngineStats per_round{};
  uint32_t ninst = 0;
  uint64_t seq = 0;
};
struct Latched {
  cudaStream_t st;
  int rc;
  char msg[160];
};
struct PendingBox {
  std::mutex mu;
  PendingRun *runs = nullptr;
  PendingMeta meta[kPending];
  uint64_t seq = 0;
  std::vector<Latched> latched;
};
PendingBox &pbox() {
  static PendingBox b;
  return b;
}

// Turns record i (its event complete) into statistics and, on error, a latch.
void collect_locked(PendingBox &b, int i) {
  PendingMeta &m = b.meta[i];
  const PendingRun &r = b.runs[i];
  int rc = 0;
  char msg[160] = {0};
  const uint32_t e = r.status.error & ~ERRB_TRACE;
  if (e) {
    snprintf(msg, sizeof(msg), "asynchronous sort: engine error bits 0x%x (1 pivot attempts, 2 nodes, 4 list, 8 arena, "
             "16 sizes)", r.status.error);
    rc = (e & ERRB_ATTEMPTS) ? 7 : ((e & ERRB_SIZES) ? 8 : 2);
  } else if (r.status.done < m.ninst) {
    snprintf(msg, sizeof(msg), "asynchronous sort did not finish (%s)",
             r.gs.grow ? "its node pool was too small: sort it with host-driven rounds" : "round limit");
    rc = r.gs.grow ? 2 : 8;
  }
  {
    std::lock_guard<std::mutex> g(stats_box().mu);
    EngineStats &S = stats_box().s;
    S.rounds += r.gs.rounds;
    S.nodes += r.gs.nodes;
    S.sorts += m.ninst;
    S.bytes[KF_LEAF] += 2.0 * (m.key_bytes + 4) * (double)r.gs.leaf_elems;
    S.bytes[KF_COUNT] += (m.key_bytes + 4) * (double)r.gs.ready_elems;
    S.bytes[KF_SKEW] += 2.0 * (m.key_bytes + 4) * (double)r.gs.ready_elems;
    for (int f = 0; f < KF_COUNT_FAMILIES; f++) S.launches[f] += r.gs.rounds * m.per_round.launches[f];
  }
  if (rc) {
    bool have = false;
    for (const Latched &l : b.latched) have = have || l.st == m.st;
    if (!have) {
      Latched l;
      l.st = m.st;
      l.rc = rc;
      snprintf(l.msg, sizeof(l.msg), "%s", msg);
      b.latched.push_back(l);
    }
  }
  if (m.ev) cudaEventDestroy(m.ev);
  m = PendingMeta();
}

// Collects the stream's finished records (all of them when wait); returns
// its latched error, if any.
int poll_locked(PendingBox &b, cudaStream_t st, bool wait, char *err, size_t errlen) {
  for (int i = 0; i < kPending; i++) {
    PendingMeta &m = b.meta[i];
    if (!m.used || !m.committed || m.st != st) continue;
    const cudaError_t q = wait ? cudaEventSynchronize(m.ev) : cudaEventQuery(m.ev);
    if (q == cudaSuccess)
      collect_locked(b, i);
    else if (q != cudaErrorNotReady) {
      snprintf(err, errlen, "asynchronous sort: %s", cudaGetErrorString(q));
      return 5;
    }
  }
  for (size_t j = 0; j < b.latched.size(); j++)
    if (b.latched[j].st == st) {
      const int rc = b.latched[j].rc;
      snprintf(err, errlen, "%s", b.latched[j].msg);
      b.latched.erase(b.latched.begin() + (long)j);
      return rc;
    }
  return 0;
}
}  // namespace

PendingRun *pending_take(cudaStream_t st, double key_bytes, const EngineStats &per_round, uint32_t ninst,
                         char *err, size_t errlen, int *rc) {
  PendingBox &b = pbox();
  std::lock_guard<std::mutex> g(b.mu);
  *rc = 0;
  if (!b.runs) {
    void *p = nullptr;
    const cudaError_t e = cudaMallocHost(&p, sizeof(PendingRun) * kPending);
    if (e != cudaSuccess) {
      snprintf(err, errlen, "page-locked status records: %s", cudaGetErrorString(e));
      *rc = 5;
      return nullptr;
    }
    b.runs = static_cast<PendingRun *>(p);
  }
  int slot = -1;
  for (int i = 0; i < kPending && slot < 0; i++)
    if (!b.meta[i].used) slot = i;
  if (slot < 0) {  // all in flight: wait for the oldest and collect it
    int old = 0;
    for (int i = 1; i < kPending; i++)
      if (b.meta[i].seq < b.meta[old].seq) old = i;
    const cudaError_t e = cudaEventSynchronize(b.meta[old].ev);
    if (e != cudaSuccess) {
      snprintf(err, errlen, "asynchronous sort: %s", cudaGetErrorString(e));
      *rc = 5;
      return nullptr;
    }
    collect_locked(b, old);
    slot = old;
  }
  PendingMeta &m = b.meta[slot];
  m.used = true;
  m.committed = false;
  m.st = st;
  m.key_bytes = key_bytes;
  m.per_round = per_round;
  m.ninst = ninst;
  memset(&b.runs[slot], 0, sizeof(PendingRun));
  return &b.runs[slot];
}

int pending_commit(PendingRun *r, cudaStream_t st, char *err, size_t errlen) {
  PendingBox &b = pbox();
  std::lock_guard<std::mutex> g(b.mu);
  PendingMeta &m = b.meta[r - b.runs];
  cudaError_t e = cudaEventCreateWithFlags(&m.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(m.ev, st);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "asynchronous sort: %s", cudaGetErrorString(e));
    if (m.ev) cudaEventDestroy(m.ev);
    m = PendingMeta();
    return 5;
  }
  m.committed = true;
  m.seq = ++b.seq;
  return 0;
}

int engine_poll(cudaStream_t st, char *err, size_t errlen) {
  PendingBox &b = pbox();
  std::lock_guard<std::mutex> g(b.mu);
  return poll_locked(b, st, false, err, errlen);
}

int engine_sync(cudaStream_t st, char *err, size_t errlen) {
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "%s", cudaGetErrorString(e));
    return 5;
  }
  PendingBox &b = pbox();
  std::lock_guard<std::mutex> g(b.mu);
  return poll_locked(b, st, true, err, errlen);
}

void engine_set_radix_classes(int dtype, uint32_t mask) { stats_box().radix_classes[dtype].store(mask & kRadixClassesAll); }
uint32_t engine_get_radix_classes(int dtype) { return stats_box().radix_classes[dtype].load(); }

uint32_t engine_max_pivots(int dtype) {
  return dtype == DT_U32 ? Engine<DT_U32>::max_pivots()
                         : (dtype == DT_U64 ? Engine<DT_U64>::max_pivots() : Engine<DT_F32>::max_pivots());
}

uint64_t engine_max_n(int dtype) {
  return dtype == DT_U32 ? Engine<DT_U32>::max_n()
                         : (dtype == DT_U64 ? Engine<DT_U64>::max_n() : Engine<DT_F32>::max_n());
}

uint32_t engine_max_leaf(int dtype) {
  return dtype == DT_U32 ? Engine<DT_U32>::max_leaf()
                         : (dtype == DT_U64 ? Engine<DT_U64>::max_leaf() : Engine<DT_F32>::max_leaf());
}

uint64_t engine_scratch_bytes_u64(uint64_t, uint32_t, uint32_t, uint32_t);
uint64_t engine_scratch_bytes_f32(uint64_t, uint32_t, uint32_t, uint32_t);

uint64_t engine_skew_scratch_bytes(int dtype, uint64_t n, uint64_t cols, uint64_t k) {
  if (dtype == DT_U64) return Engine<DT_U64>::skew_scratch_bytes(n, (u32)cols, (u32)k);
  if (dtype == DT_F32) return Engine<DT_F32>::skew_scratch_bytes(n, (u32)cols, (u32)k);
  return Engine<DT_U32>::skew_scratch_bytes(n, (u32)cols, (u32)k);
}

uint64_t engine_scratch_bytes(int dtype, uint64_t total_n, uint32_t ninst, uint32_t cutoff, uint32_t cutoff_max) {
  if (dtype == DT_U64) return engine_scratch_bytes_u64(total_n, ninst, cutoff, cutoff_max);
  if (dtype == DT_F32) return engine_scratch_bytes_f32(total_n, ninst, cutoff, cutoff_max);
  return Engine<DT_U32>::scratch_bytes(total_n, ninst, cutoff, cutoff_max);
}

#define SQ_SESSION_DECL(SUFFIX)                                                                          \
  int session_open_##SUFFIX(const SessionSpec &, cudaStream_t, void **, char *, size_t);                 \
  int session_admit_##SUFFIX(void *, const InstSpec &, uint32_t, char *, size_t);                        \
  int session_step_##SUFFIX(void *, std::vector<uint32_t> &, char *, size_t);                            \
  bool session_busy_##SUFFIX(void *);                                                                     \
  void session_close_##SUFFIX(void *);                                                                    \
  uint64_t session_scratch_bytes_##SUFFIX(const SessionSpec &);
SQ_SESSION_DECL(u32)
SQ_SESSION_DECL(u64)
SQ_SESSION_DECL(f32)

#define SQ_BY_DTYPE(dtype, CALL) \
  ((dtype) == DT_U64 ? CALL(u64) : (dtype) == DT_F32 ? CALL(f32) : CALL(u32))

int session_open(int dtype, const SessionSpec &sp, cudaStream_t st, void **out, char *err, size_t errlen) {
#define C(S) session_open_##S(sp, st, out, err, errlen)
  return SQ_BY_DTYPE(dtype, C);
#undef C
}
int session_admit(int dtype, void *s, const InstSpec &is, uint32_t slot, char *err, size_t errlen) {
#define C(S) session_admit_##S(s, is, slot, err, errlen)
  return SQ_BY_DTYPE(dtype, C);
#undef C
}
int session_step(int dtype, void *s, std::vector<uint32_t> &done, char *err, size_t errlen) {
#define C(S) session_step_##S(s, done, err, errlen)
  return SQ_BY_DTYPE(dtype, C);
#undef C
}
bool session_busy(int dtype, void *s) {
#define C(S) session_busy_##S(s)
  return SQ_BY_DTYPE(dtype, C);
#undef C
}
void session_close(int dtype, void *s) {
  if (dtype == DT_U64)
    session_close_u64(s);
  else if (dtype == DT_F32)
    session_close_f32(s);
  else
    session_close_u32(s);
}
uint64_t session_scratch_bytes(int dtype, const SessionSpec &sp) {
#define C(S) session_scratch_bytes_##S(sp)
  return SQ_BY_DTYPE(dtype, C);
#undef C
}

int engine_run_u32(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen) {
  return Engine<DT_U32>::run(spec, st, err, errlen);
}

SQ_SESSION_FUNCS(u32, DT_U32)

}  // namespace sq
