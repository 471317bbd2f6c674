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

int engine_run_u32(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen) {
  return Engine<DT_U32>::run(spec, st, err, errlen);
}

}  // namespace sq
