// S7 growth and division (Table D.1 GrowthDivision).
#include "kernels.cuh"

namespace bdm {

size_t growth_scratch_bytes(int64_t total_slots, int n_sims) {
  return (size_t)(total_slots > 0 ? total_slots : 1) * 16 + (size_t)n_sims * 64;
}

void launch_growth(const DevCtx &C, cudaStream_t st, void *scratch, size_t scratch_bytes) {
  (void)C; (void)st; (void)scratch; (void)scratch_bytes;
}

}  // namespace bdm
