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

void engine_set_radix_classes(int dtype, uint32_t mask) { stats_box().radix_classes[dtype].store(mask & kRadixClassesAll); }
uint32_t engine_get_radix_classes(int dtype) { return stats_box().radix_classes[dtype].load(); }

uint32_t engine_max_pivots(int dtype) {
  return dtype == DT_U32 ? Engine<DT_U32>::max_pivots()
                         : (dtype == DT_U64 ? Engine<DT_U64>::max_pivots() : Engine<DT_F32>::max_pivots());
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
