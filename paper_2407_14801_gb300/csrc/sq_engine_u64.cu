// u64 engine instantiation.
#include "sq_engine.cuh"

namespace sq {

uint64_t engine_scratch_bytes_u64(uint64_t total_n, uint32_t ninst, uint32_t cutoff, uint32_t cutoff_max) {
  return Engine<DT_U64>::scratch_bytes(total_n, ninst, cutoff, cutoff_max);
}

int engine_run_u64(const RunSpec &spec, cudaStream_t st, char *err, size_t errlen) {
  return Engine<DT_U64>::run(spec, st, err, errlen);
}

SQ_SESSION_FUNCS(u64, DT_U64)

}  // namespace sq
