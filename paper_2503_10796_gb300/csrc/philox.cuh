// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): the counter-based generator proposed in
// §7.1.4 for reproducible agent-based simulation.  Every draw is a function
// of (key, counter) alone, so no order of processing changes a result.
#pragma once

namespace bdm {

__device__ __forceinline__ void philox4x64_10(const unsigned long long ctr[4], const unsigned long long key[2],
                                              unsigned long long out[4]) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  unsigned long long c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  unsigned long long k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const unsigned long long lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    const unsigned long long lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    const unsigned long long n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// A uniform in [0, 1) from the top 53 bits of a word (exact in FP64).
__device__ __forceinline__ double unit53(unsigned long long w) { return __dmul_rn((double)(w >> 11), 0x1.0p-53); }

}  // namespace bdm
