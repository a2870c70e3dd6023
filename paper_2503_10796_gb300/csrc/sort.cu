// S3 Morton re-sort of the agent storage (§5.4.2, Fig 5.4).
//
// Runs inside an iteration, right after the box count (S1), when a
// re-sort is due.  Keys are the Morton codes of the agents' boxes of the
// current grid (bits of c_x, c_y, c_z interleaved with x least significant,
// as in Fig 5.4C), prefixed by the simulation's rank in slot-region order.
// A least-significant-digit radix sort (8-bit digits, stable) orders the
// (key, slot) pairs; then every per-slot array is permuted, so that the
// prefix sum over box leaders that follows places boxes, and therefore
// cells, in Morton order.  The thesis obtains the same order without a sort
// by its gap algorithm over a dense box enumeration; on the GPU a radix sort
// over the agents is O(#agents) also when the grid is sparse.
#include "kernels.cuh"

namespace bdm {

constexpr int kSortThreads = 256;
constexpr int kDigits = 256;

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  // bit b of v -> bit 3b (v < 2^21)
  v &= 0x1FFFFFull;
  v = (v | (v << 32)) & 0x1F00000000FFFFull;
  v = (v | (v << 16)) & 0x1F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__device__ __forceinline__ uint64_t morton3(uint64_t pk) {
  return spread3(pk & kCoordMask) | (spread3((pk >> kCoordBits) & kCoordMask) << 1) |
         (spread3((pk >> (2 * kCoordBits)) & kCoordMask) << 2);
}

struct SortBufs {
  uint64_t *ka, *kb;
  int32_t *va, *vb;
  uint32_t *hist;   // kDigits x G counts, digit-major
  uint32_t *dbase;  // kDigits: first output position of each digit
  uint32_t *flag;   // [0] = sort due this iteration
  // permutation scratch
  double *x, *y, *z, *d, *v;
  int32_t *id;
  uint64_t *pkey;
  uint32_t *rank;
  uint8_t *flags, *nnz;
};

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

static SortBufs carve(void *scratch, int64_t M) {
  SortBufs b;
  char *p = (char *)scratch;
  auto take = [&](size_t bytes) {
    char *r = p;
    p += align256(bytes);
    return (void *)r;
  };
  b.ka = (uint64_t *)take(8 * M);
  b.kb = (uint64_t *)take(8 * M);
  b.va = (int32_t *)take(4 * M);
  b.vb = (int32_t *)take(4 * M);
  b.hist = (uint32_t *)take(4 * (size_t)kDigits * 2048);
  b.dbase = (uint32_t *)take(4 * (size_t)kDigits);
  b.flag = (uint32_t *)take(16);
  b.x = (double *)take(8 * M);
  b.y = (double *)take(8 * M);
  b.z = (double *)take(8 * M);
  b.d = (double *)take(8 * M);
  b.v = (double *)take(8 * M);
  b.id = (int32_t *)take(4 * M);
  b.pkey = (uint64_t *)take(8 * M);
  b.rank = (uint32_t *)take(4 * M);
  b.flags = (uint8_t *)take(M);
  b.nnz = (uint8_t *)take(M);
  return b;
}

size_t morton_scratch_bytes(int64_t total_slots) {
  size_t M = (size_t)(total_slots > 0 ? total_slots : 1);
  size_t b = 0;
  for (size_t s : {8 * M, 8 * M, 4 * M, 4 * M, (size_t)4 * kDigits * 2048, (size_t)4 * kDigits, (size_t)16, 8 * M,
                   8 * M, 8 * M,
                   8 * M, 8 * M, 4 * M, 8 * M, 4 * M, M, M})
    b += align256(s);
  return b;
}

// Decide whether the re-sort is due (some simulation with an interval whose
// current iteration is a multiple of it) and build the keys.
// curve 0: Morton code of the box (§5.4.2); curve 1: row-major box index
// (x fastest), the order in which a warp's lanes read neighbouring table
// words and records contiguously.
__global__ void k_sort_keys(DevCtx C, SortBufs B, int mbits, int curve) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ int due;
  if (threadIdx.x == 0) {
    int d = 0;
    for (int q = 0; q < C.n_sims; ++q) {
      int s = C.order[q];
      if (s < 0) break;
      int iv = C.sc[s].sort_interval;
      if (iv > 0 && C.ss[s].valid && C.ss[s].it % iv == 0) d = 1;
    }
    due = d;
    if (blockIdx.x == 0) B.flag[0] = (uint32_t)d;
  }
  __syncthreads();
  if (!due) return;
  int64_t n = C.g->n_cells;
  if (k >= n) return;
  // simulation of compacted index k (regions in order; cell_base prefix)
  int lo = 0, hi = C.n_sims - 1;
  while (hi > 0 && C.order[hi] < 0) --hi;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (C.ss[C.order[mid]].cell_base <= k) lo = mid; else hi = mid - 1;
  }
  int s = C.order[lo];
  int64_t slot = C.sc[s].base + (k - C.ss[s].cell_base);
  const uint64_t pk = C.a.pkey[slot];
  uint64_t code;
  if (curve == 1) {
    int64_t bx, by, bz;
    unpack_coords(pk, bx, by, bz);
    code = (uint64_t)linear_box(C.ss[s], bx, by, bz);
  } else {
    code = morton3(pk);
  }
  uint64_t key = ((uint64_t)lo << mbits) | code;
  B.ka[k] = key;
  B.va[k] = (int32_t)slot;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(DevCtx C, SortBufs B, const uint64_t *keys, int shift,
                                                            int64_t chunk) {
  if (!B.flag[0]) return;
  __shared__ uint32_t h[kDigits];
  for (int i = threadIdx.x; i < kDigits; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int64_t n = C.g->n_cells;
  int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kDigits; i += blockDim.x) B.hist[(size_t)i * gridDim.x + blockIdx.x] = h[i];
}

// Exclusive scan of the digit-major histogram: one block per digit scans
// that digit's G block counts in place (and writes the digit total to
// dbase); a second small kernel turns the totals into digit bases.
__global__ void __launch_bounds__(1024) k_sort_scan_digit(SortBufs B, int G) {
  if (!B.flag[0]) return;
  __shared__ uint32_t wsum[33];
  const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *h = B.hist + (size_t)d * G;
  const int per = (G + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b = threadIdx.x * per, e = b + per < G ? b + per : G;
  uint32_t tsum = 0;
  for (int i = b; i < e; ++i) tsum += h[i];
  uint32_t inc = tsum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const uint32_t t = wsum[w];
      wsum[w] = run;
      run += t;
    }
    wsum[32] = run;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + inc - tsum;
  for (int i = b; i < e; ++i) {
    const uint32_t v = h[i];
    h[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) B.dbase[d] = wsum[32];
}

__global__ void k_sort_scan_base(SortBufs B) {
  if (!B.flag[0]) return;
  if (threadIdx.x != 0) return;
  uint32_t run = 0;
  for (int d = 0; d < kDigits; ++d) {
    const uint32_t t = B.dbase[d];
    B.dbase[d] = run;
    run += t;
  }
}

// Stable scatter: a block walks its chunk in order, 256 elements at a time;
// ranks inside a warp from match_any, across warps from per-warp digit
// counts, across rounds from a running per-digit count.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(DevCtx C, SortBufs B, const uint64_t *kin,
                                                               const int32_t *vin, uint64_t *kout, int32_t *vout,
                                                               int shift, int64_t chunk) {
  if (!B.flag[0]) return;
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t base[kDigits];
  __shared__ uint32_t wcnt[W][kDigits];
  for (int i = threadIdx.x; i < kDigits; i += blockDim.x)
    base[i] = B.hist[(size_t)i * gridDim.x + blockIdx.x] + B.dbase[i];
  int64_t n = C.g->n_cells;
  int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t0 = b; t0 < e; t0 += blockDim.x) {
    for (int i = threadIdx.x; i < W * kDigits; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    int64_t i = t0 + threadIdx.x;
    bool act = i < e;
    uint64_t key = act ? kin[i] : 0ull;
    int32_t val = act ? vin[i] : 0;
    uint32_t dg = act ? (uint32_t)((key >> shift) & 0xFF) : 0xFFFFFFFFu;
    // lanes holding the same digit: one ballot per digit bit (and one for
    // the active lanes), which is cheaper than a match instruction
    const unsigned int am = __ballot_sync(0xffffffffu, act);
    unsigned int peers = act ? am : ~am;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const unsigned int B = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
      peers &= ((dg >> b) & 1u) ? B : ~B;
    }
    unsigned int lt = (1u << lane) - 1u;
    uint32_t r_in_warp = __popc(peers & lt);
    if (act && r_in_warp == 0) wcnt[warp][dg] = __popc(peers);
    __syncthreads();
    if (act) {
      uint32_t r = base[dg] + r_in_warp;
      for (int w = 0; w < warp; ++w) r += wcnt[w][dg];
      kout[r] = key;
      vout[r] = val;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) {
      uint32_t s = 0;
      for (int w = 0; w < W; ++w) s += wcnt[w][d];
      base[d] += s;
    }
    __syncthreads();
  }
}

// Permutation: gather every per-slot array in sorted order into scratch,
// then copy back.  Sorted position k of simulation s lands in slot
// base_s + (k - cell_base_s).
__global__ void k_sort_gather(DevCtx C, SortBufs B, const int32_t *perm) {
  if (!B.flag[0]) return;
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= C.g->n_cells) return;
  int32_t src = perm[k];
  B.x[k] = C.a.x[src];
  B.y[k] = C.a.y[src];
  B.z[k] = C.a.z[src];
  B.d[k] = C.a.d[src];
  B.v[k] = C.a.v[src];
  B.id[k] = C.a.id[src];
  B.pkey[k] = C.a.pkey[src];
  B.rank[k] = C.a.rank[src];
  B.flags[k] = C.a.flags[src];
  B.nnz[k] = C.a.nnz[src];
}

// cells: the permutation is the cell order (perm = the cells' slots), and
// each cell's slot becomes its new one.
__global__ void k_sort_writeback(DevCtx C, SortBufs B, const int32_t *perm, int cells) {
  if (!B.flag[0]) return;
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= C.g->n_cells) return;
  int s = C.a.sim[perm[k]];
  int64_t dst = C.sc[s].base + (k - C.ss[s].cell_base);
  if (cells) C.c.slot[k] = (int32_t)dst;
  C.a.x[dst] = B.x[k];
  C.a.y[dst] = B.y[k];
  C.a.z[dst] = B.z[k];
  C.a.d[dst] = B.d[k];
  C.a.v[dst] = B.v[k];
  C.a.id[dst] = B.id[k];
  C.a.pkey[dst] = B.pkey[k];
  C.a.rank[dst] = B.rank[k];
  C.a.flags[dst] = B.flags[k];
  C.a.nnz[dst] = B.nnz[k];
}

void launch_morton(const DevCtx &C, cudaStream_t st, void *scratch, size_t scratch_bytes, int key_bits,
                   int curve) {
  (void)scratch_bytes;
  int64_t M = C.total_slots;
  if (M <= 0) return;
  SortBufs B = carve(scratch, M);
  // key_bits: simulation-rank bits + 3 x bits per axis, passed by the host
  int sim_bits = 0;
  while ((1 << sim_bits) < C.n_sims) ++sim_bits;
  int mbits = key_bits - sim_bits;
  if (mbits < 3) mbits = 3;
  int total_bits = mbits + sim_bits;
  int passes = (total_bits + 7) / 8;
  unsigned int nb = (unsigned int)((M + kSortThreads - 1) / kSortThreads);
  k_sort_keys<<<nb, kSortThreads, 0, st>>>(C, B, mbits, curve);
  int64_t G = (M + 8191) / 8192;
  if (G > 2048) G = 2048;
  if (G < 1) G = 1;
  int64_t chunk = (M + G - 1) / G;
  chunk = (chunk + kSortThreads - 1) / kSortThreads * kSortThreads;
  G = (M + chunk - 1) / chunk;
  if (G < 1) G = 1;
  uint64_t *kin = B.ka, *kout = B.kb;
  int32_t *vin = B.va, *vout = B.vb;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_sort_hist<<<(unsigned int)G, kSortThreads, 0, st>>>(C, B, kin, shift, chunk);
    k_sort_scan_digit<<<kDigits, 1024, 0, st>>>(B, (int)G);
    k_sort_scan_base<<<1, 32, 0, st>>>(B);
    k_sort_scatter<<<(unsigned int)G, kSortThreads, 0, st>>>(C, B, kin, vin, kout, vout, shift, chunk);
    uint64_t *tk = kin; kin = kout; kout = tk;
    int32_t *tv = vin; vin = vout; vout = tv;
  }
  k_sort_gather<<<nb, kSortThreads, 0, st>>>(C, B, vin);
  k_sort_writeback<<<nb, kSortThreads, 0, st>>>(C, B, vin, 0);
}

// Re-sort without a sort: the cells of the iteration just computed list
// every box's agents together, boxes in the storage order of their first
// agent (the order of the last sort, kept as agents move); permuting the
// storage into cell order keeps boxes contiguous and that order.  Runs at
// the end of an iteration (after displacement and division), when the cells
// still map onto the storage.
void launch_cell_order(const DevCtx &C, cudaStream_t st, void *scratch) {
  int64_t M = C.total_slots;
  if (M <= 0) return;
  SortBufs B = carve(scratch, M);
  cudaMemsetAsync(B.flag, 1, sizeof(uint32_t), st);  // non-zero: due (a memset node in a graph)
  unsigned int nb = (unsigned int)((M + kSortThreads - 1) / kSortThreads);
  k_sort_gather<<<nb, kSortThreads, 0, st>>>(C, B, C.c.slot);
  k_sort_writeback<<<nb, kSortThreads, 0, st>>>(C, B, C.c.slot, 1);
}

}  // namespace bdm
