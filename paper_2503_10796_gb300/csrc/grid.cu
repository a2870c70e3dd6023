// Grid build on the device (S0 bounding box, S1 box index, S2 count /
// prefix sum / placement), after §4.4.3 and §5.3.1 of the thesis: boxes of
// equal size L, an agent's box from its center, per-box timestamps so that
// empty boxes never have to be cleared, and boxes that store only a start
// index and a count.
#include "kernels.cuh"

namespace bdm {

// ---------------------------------------------------------------------------
// S0: per-simulation bounding box and largest diameter.
//
// Blocks walk contiguous chunks of slots.  A thread keeps running minima and
// maxima for the simulation it is in; whenever the simulation of a tile is
// not the one accumulated so far, the block reduces and flushes with one
// atomic per quantity.  FP64 min/max are exact, so the result does not
// depend on the order, and order-preserving 64-bit keys let plain integer
// atomics do the reduction.
// ---------------------------------------------------------------------------
struct BoxAcc {
  unsigned long long mn[3], mx[3], dm;
  __device__ void reset() {
    for (int a = 0; a < 3; ++a) { mn[a] = ~0ull; mx[a] = 0ull; }
    dm = 0ull;
  }
};

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  for (int o = 16; o; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ void flush_box(const DevCtx &C, int sim, BoxAcc &acc, unsigned long long (*sh)[7]) {
  // Block-wide reduction of the 7 keys, then 7 atomics.
  unsigned long long v[7] = {acc.mn[0], acc.mn[1], acc.mn[2], acc.mx[0], acc.mx[1], acc.mx[2], acc.dm};
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 3; ++q) v[q] = warp_min_u64(v[q]);
  for (int q = 3; q < 7; ++q) v[q] = warp_max_u64(v[q]);
  if (lane == 0)
    for (int q = 0; q < 7; ++q) sh[warp][q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    for (int w = 1; w < nw; ++w) {
      for (int q = 0; q < 3; ++q) v[q] = sh[w][q] < v[q] ? sh[w][q] : v[q];
      for (int q = 3; q < 7; ++q) v[q] = sh[w][q] > v[q] ? sh[w][q] : v[q];
    }
    SimState &s = C.ss[sim];
    if (v[0] != ~0ull) {
      for (int a = 0; a < 3; ++a) {
        atomicMin(&s.bmin[a], v[a]);
        atomicMax(&s.bmax[a], v[3 + a]);
      }
      atomicMax(&s.dmax, v[6]);
    }
  }
  __syncthreads();
  acc.reset();
}

__global__ void __launch_bounds__(kThreads) k_bbox(DevCtx C, int64_t chunk) {
  __shared__ unsigned long long sh[kThreads / 32][7];
  __shared__ int tile_sim[2];
  BoxAcc acc;
  acc.reset();
  int cur = -1;  // simulation accumulated by the block
  int64_t begin = (int64_t)blockIdx.x * chunk;
  int64_t end = begin + chunk < C.total_slots ? begin + chunk : C.total_slots;
  if (begin >= end) return;
  {
    // Regions are contiguous: a chunk whose ends lie in one simulation lies
    // in it entirely, and needs no per-tile checks.
    const int s0 = C.a.sim[begin], s1 = C.a.sim[end - 1];
    if (s0 == s1 && s0 >= 0) {
      const int64_t last = C.sc[s0].base + C.ss[s0].n;
      for (int64_t slot = begin + threadIdx.x; slot < end && slot < last; slot += blockDim.x) {
        const unsigned long long kx = ord_key(C.a.x[slot]), ky = ord_key(C.a.y[slot]), kz = ord_key(C.a.z[slot]);
        const unsigned long long kd = ord_key(C.a.d[slot]);
        acc.mn[0] = kx < acc.mn[0] ? kx : acc.mn[0];
        acc.mn[1] = ky < acc.mn[1] ? ky : acc.mn[1];
        acc.mn[2] = kz < acc.mn[2] ? kz : acc.mn[2];
        acc.mx[0] = kx > acc.mx[0] ? kx : acc.mx[0];
        acc.mx[1] = ky > acc.mx[1] ? ky : acc.mx[1];
        acc.mx[2] = kz > acc.mx[2] ? kz : acc.mx[2];
        acc.dm = kd > acc.dm ? kd : acc.dm;
      }
      flush_box(C, s0, acc, sh);
      return;
    }
  }
  for (int64_t t0 = begin; t0 < end; t0 += blockDim.x) {
    int64_t slot = t0 + threadIdx.x;
    int sim = slot < end ? C.a.sim[slot] : -1;
    if (threadIdx.x == 0) { tile_sim[0] = 0x7fffffff; tile_sim[1] = -1; }
    __syncthreads();
    if (sim >= 0) { atomicMin(&tile_sim[0], sim); atomicMax(&tile_sim[1], sim); }
    __syncthreads();
    int lo = tile_sim[0], hi = tile_sim[1];
    __syncthreads();
    if (hi < 0) continue;
    bool uniform = (lo == hi);
    if (uniform && lo != cur) {
      if (cur >= 0) flush_box(C, cur, acc, sh);
      cur = lo;
    }
    bool active = false;
    double x = 0, y = 0, z = 0, d = 0;
    if (sim >= 0 && slot - C.sc[sim].base < C.ss[sim].n) {
      active = true;
      x = C.a.x[slot]; y = C.a.y[slot]; z = C.a.z[slot]; d = C.a.d[slot];
    }
    if (!active) continue;
    unsigned long long kx = ord_key(x), ky = ord_key(y), kz = ord_key(z), kd = ord_key(d);
    if (uniform) {
      acc.mn[0] = kx < acc.mn[0] ? kx : acc.mn[0];
      acc.mn[1] = ky < acc.mn[1] ? ky : acc.mn[1];
      acc.mn[2] = kz < acc.mn[2] ? kz : acc.mn[2];
      acc.mx[0] = kx > acc.mx[0] ? kx : acc.mx[0];
      acc.mx[1] = ky > acc.mx[1] ? ky : acc.mx[1];
      acc.mx[2] = kz > acc.mx[2] ? kz : acc.mx[2];
      acc.dm = kd > acc.dm ? kd : acc.dm;
    } else {
      SimState &s = C.ss[sim];
      atomicMin(&s.bmin[0], kx); atomicMin(&s.bmin[1], ky); atomicMin(&s.bmin[2], kz);
      atomicMax(&s.bmax[0], kx); atomicMax(&s.bmax[1], ky); atomicMax(&s.bmax[2], kz);
      atomicMax(&s.dmax, kd);
    }
  }
  if (cur >= 0) flush_box(C, cur, acc, sh);
}

// ---------------------------------------------------------------------------
// Grid parameters of every simulation: origin, box length, boxes per axis
// (floor((max - o) / L) + 1 in IEEE FP64), table fit, the float-float
// constants of the FP32 path and the cell ranges.
// ---------------------------------------------------------------------------
__device__ void split_pos(double v, float &h, float &l) { split_ff(v, h, l); }

// One thread per simulation; thread 0 then lays out the cell ranges.
__global__ void k_params(DevCtx C, int32_t step) {
  Globals *g = C.g;
  for (int k = threadIdx.x; k < C.n_sims; k += blockDim.x) {
    int s = C.order[k];
    if (s < 0) continue;
    const SimConst &sc = C.sc[s];
    SimState &st = C.ss[s];
    st.ncell = st.n;
    st.valid = 0;
    st.same_grid = 0;
    if (step) {
      st.it = st.t;
      st.t += 1;
      st.updates += (unsigned long long)(st.n > 0 ? st.n : 0);
    }
    if (st.n <= 0) {
      for (int a = 0; a < 3; ++a) { st.bmin[a] = ~0ull; st.bmax[a] = 0ull; }
      st.dmax = 0ull;
      if (step) st.has_prev = 0;
      continue;
    }
    double mx[3];
    for (int a = 0; a < 3; ++a) {
      st.o[a] = ord_val(st.bmin[a]);
      mx[a] = ord_val(st.bmax[a]);
    }
    double dmax = ord_val(st.dmax);
    double L = sc.box_length > 0.0 ? sc.box_length : dmax;
    st.L = L;
    bool ok = L > 0.0 && isfinite(L);
    int64_t nb = 1;
    for (int a = 0; a < 3; ++a) {
      if (!isfinite(st.o[a]) || !isfinite(mx[a])) ok = false;
      double q = ok ? floor(__ddiv_rn(__dsub_rn(mx[a], st.o[a]), L)) : 0.0;
      if (!(q < (double)(1ll << kCoordBits) - 1.0)) { ok = false; q = 0.0; }
      st.dims[a] = (int64_t)q + 1;
      nb *= st.dims[a];
    }
    if (!ok) set_err(g, ERR_COORD | ERR_NONFINITE);
    st.nboxes = nb;
    if (ok && (nb > sc.table_cap || nb >= (1ll << 32))) {
      set_err(g, ERR_TABLE);
      ok = false;
    }
    st.valid = ok ? 1 : 0;
    st.same_grid = (step && st.has_prev && ok && st.o[0] == st.prev_o[0] && st.o[1] == st.prev_o[1] &&
                    st.o[2] == st.prev_o[2] && L == st.prev_L && st.dims[0] == st.prev_dims[0] &&
                    st.dims[1] == st.prev_dims[1] && st.dims[2] == st.prev_dims[2]) ? 1 : 0;
    // float-float constants
    split_pos(L, st.Lh, st.Ll);
    double il = __ddiv_rn(1.0, L);
    split_pos(il, st.ilh, st.ill);
    // FP32 filter margin: truncated hi parts are off by < 1 ulp of values
    // below 2L; differences and squares add a few more ulps.
    st.marg = (float)(L * 0x1p-19) + 0x1p-30f;
    if (step) {
      for (int a = 0; a < 3; ++a) { st.prev_o[a] = st.o[a]; st.prev_dims[a] = st.dims[a]; }
      st.prev_L = L;
      st.has_prev = ok ? 1 : 0;
    }
    // accumulators for the next bounding box
    for (int a = 0; a < 3; ++a) { st.bmin[a] = ~0ull; st.bmax[a] = 0ull; }
    st.dmax = 0ull;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    g->stamp += 1u;
    int64_t cells = 0;
    for (int k = 0; k < C.n_sims; ++k) {
      const int s = C.order[k];
      if (s < 0) break;
      C.ss[s].cell_base = cells;
      cells += C.ss[s].n;
    }
    g->n_cells = cells;
  }
}

// ---------------------------------------------------------------------------
// S1: box index, per-box count with timestamps, dirty marks for static
// detection (§5.5).
// ---------------------------------------------------------------------------
// Add one agent (count) and/or a dirty mark to a box entry; returns the
// agent's rank inside the box.  Entries whose stamp is not the current one
// are empty, whatever their count says.
__device__ __forceinline__ uint32_t tab_add(unsigned long long *e, uint32_t stamp, bool dirty, uint32_t count,
                                            Globals *g) {
  unsigned long long old = *(volatile unsigned long long *)e;
  for (int tries = 0; tries < (1 << 22); ++tries) {
    const unsigned long long assumed = old;
    const bool live = ent_stamp(assumed) == stamp;
    const uint32_t cnt = live ? ent_count(assumed) : 0u;
    const bool dir = (live && ent_dirty(assumed)) || dirty;
    uint32_t ncnt = cnt + count;
    if (ncnt > kMaxBoxCount) {
      // more agents in one box than the table word holds: the step is
      // invalid (latched error); placement skips the agents beyond it
      set_err(g, ERR_TABLE);
      ncnt = kMaxBoxCount;
    }
    const unsigned long long nv = ((unsigned long long)stamp << 43) | ((unsigned long long)(dir ? 1u : 0u) << 42) |
                                  ((unsigned long long)ncnt << 32) | (live ? (assumed & 0xFFFFFFFFull) : 0ull);
    if (nv == assumed) return cnt;
    old = atomicCAS(e, assumed, nv);
    if (old == assumed) return cnt;
  }
  set_err(g, ERR_TIMEOUT);
  return 0u;
}

// hist: the per-slot box history (the step passes it; queries pass null so
// that the history of the last iteration survives them).
__global__ void __launch_bounds__(kThreads) k_count(DevCtx C, uint64_t *hist) {
  int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= C.total_slots) return;
  int sim = C.a.sim[slot];
  if (sim < 0) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (slot - sc.base >= s.n || !s.valid) return;
  double p[3] = {C.a.x[slot], C.a.y[slot], C.a.z[slot]};
  int64_t c[3];
  for (int a = 0; a < 3; ++a) {
    double av = __dsub_rn(p[a], s.o[a]);
    float ah, al;
    split_ff(av, ah, al);
    int64_t ca = box_coord(av, ah, al, s.ilh, s.ill, s.L);
    c[a] = ca < 0 ? 0 : (ca >= s.dims[a] ? s.dims[a] - 1 : ca);
  }
  uint64_t pk = pack_coords(c[0], c[1], c[2]);
  C.a.pkey[slot] = pk;
  uint64_t pk_prev = pk;
  if (hist) {
    pk_prev = hist[slot];
    hist[slot] = pk;
  }
  bool changed = hist && (C.a.flags[slot] & FLAG_CHANGED) != 0;
  const uint32_t stamp = C.g->stamp & kStampMask;
  int64_t idx = sc.table_base + linear_box(s, c[0], c[1], c[2]);
  // Lanes of a warp that share a box add their count with one atomic
  // (neighbouring slots mostly share boxes once the storage is sorted).
  const unsigned mask = __activemask();
  const unsigned peers = __match_any_sync(mask, (unsigned long long)idx);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const unsigned dirty_any = __reduce_or_sync(peers, changed ? 1u : 0u);
  uint32_t base = 0;
  if (lane == leader) base = tab_add(&C.tab.e[idx], stamp, dirty_any != 0, (uint32_t)__popc(peers), C.g);
  base = __shfl_sync(peers, base, leader);
  C.a.rank[slot] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
  if (changed && s.same_grid && pk_prev != pk) {
    int64_t px, py, pz;
    unpack_coords(pk_prev, px, py, pz);
    if (px < s.dims[0] && py < s.dims[1] && pz < s.dims[2])
      tab_add(&C.tab.e[sc.table_base + linear_box(s, px, py, pz)], stamp, true, 0u, C.g);
  }
}

// ---------------------------------------------------------------------------
// S2: exclusive prefix sum over box leaders (the rank-0 agent of each box
// contributes the box's count), in slot order, giving every box its first
// cell position; then placement of every agent at start + rank.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t leader_value(const DevCtx &C, int64_t slot, int64_t &idx) {
  idx = -1;
  if (slot >= C.total_slots) return 0u;
  int sim = C.a.sim[slot];
  if (sim < 0) return 0u;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (slot - sc.base >= s.n || !s.valid) return 0u;
  if (C.a.rank[slot] != 0u) return 0u;
  int64_t cx, cy, cz;
  unpack_coords(C.a.pkey[slot], cx, cy, cz);
  idx = sc.table_base + linear_box(s, cx, cy, cz);
  return ent_count(C.tab.e[idx]);
}

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *sh) {
  v = __reduce_add_sync(0xffffffffu, v);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  uint32_t t = 0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
    t = __reduce_add_sync(0xffffffffu, t);
  }
  __syncthreads();
  return t;  // valid in warp 0
}

// Exclusive scan inside the block; *total receives the block total.
__device__ __forceinline__ uint32_t block_exscan_u32(uint32_t v, uint32_t *sh, uint32_t *total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? sh[lane] : 0u;
    uint32_t ws = w;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    if (lane < nw) sh[lane] = ws - w;
    if (lane == nw - 1) sh[32] = ws;
  }
  __syncthreads();
  uint32_t r = sh[warp] + x - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_up(DevCtx C, int64_t chunk, uint32_t *partial) {
  __shared__ uint32_t sh[33];
  int64_t begin = (int64_t)blockIdx.x * chunk;
  int64_t end = begin + chunk < C.total_slots ? begin + chunk : C.total_slots;
  uint32_t sum = 0;
  for (int64_t slot = begin + threadIdx.x; slot < end; slot += blockDim.x) {
    int64_t idx;
    sum += leader_value(C, slot, idx);
  }
  uint32_t t = block_sum_u32(sum, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *partial, int n) {
  __shared__ uint32_t sh[33];
  uint32_t v = (int)threadIdx.x < n ? partial[threadIdx.x] : 0u;
  uint32_t total;
  uint32_t ex = block_exscan_u32(v, sh, &total);
  if ((int)threadIdx.x < n) partial[threadIdx.x] = ex;
}

__global__ void __launch_bounds__(1024) k_scan_down(DevCtx C, int64_t chunk, const uint32_t *partial) {
  __shared__ uint32_t sh[33];
  int64_t begin = (int64_t)blockIdx.x * chunk;
  int64_t end = begin + chunk < C.total_slots ? begin + chunk : C.total_slots;
  uint32_t base = partial[blockIdx.x];
  for (int64_t t0 = begin; t0 < end; t0 += blockDim.x) {
    int64_t slot = t0 + threadIdx.x;
    int64_t idx = -1;
    uint32_t v = slot < end ? leader_value(C, slot, idx) : 0u;
    uint32_t total;
    uint32_t ex = block_exscan_u32(v, sh, &total);
    if (idx >= 0) C.tab.e[idx] = (C.tab.e[idx] & 0xFFFFFFFF00000000ull) | (unsigned long long)(base + ex);
    base += total;
  }
}

// Place every agent at start + rank of its box in `cells`.  fp64_records:
// write the FP64 record whatever the simulation's precision (queries).
__global__ void __launch_bounds__(kThreads) k_place(DevCtx C, Cells cells, int fp64_records) {
  int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= C.total_slots) return;
  int sim = C.a.sim[slot];
  if (sim < 0) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (slot - sc.base >= s.n || !s.valid) return;
  uint64_t pk = C.a.pkey[slot];
  int64_t c[3];
  unpack_coords(pk, c[0], c[1], c[2]);
  int64_t idx = sc.table_base + linear_box(s, c[0], c[1], c[2]);
  const unsigned long long e = C.tab.e[idx];
  const uint32_t rank = C.a.rank[slot];
  if (rank >= ent_count(e)) return;  // box overflow (error latched by the count)
  int64_t p = (int64_t)ent_start(e) + rank;
  cells.slot[p] = (int32_t)slot;
  cells.sim[p] = sim;
  cells.pkey[p] = pk;
  if (cells.flag) {
    uint8_t fl = C.a.flags[slot];
    cells.flag[p] = (!(fl & FLAG_CHANGED) && C.a.nnz[slot] <= 1) ? CELL_STATIC_ELIGIBLE : 0;
  }
  double pos[3] = {C.a.x[slot], C.a.y[slot], C.a.z[slot]};
  double r = 0.5 * C.a.d[slot];
  if (fp64_records || sc.precision == BDM_PREC_FP64) {
    cells.r64[p] = make_double4_32a(pos[0], pos[1], pos[2], r);
  } else {
    float h[3], l[3], rh, rl;
    for (int a = 0; a < 3; ++a) {
      // offset inside the own box, exact in FP64: a - c L
      double av = __dsub_rn(pos[a], s.o[a]);
      double w = __fma_rn(-(double)c[a], s.L, av);
      split_ff(w, h[a], l[a]);
    }
    split_ff(r, rh, rl);
    cells.r0[p] = make_float4(h[0], h[1], h[2], rh);
    cells.r1[p] = make_float4(l[0], l[1], l[2], rl);
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

void launch_bbox(const DevCtx &C, cudaStream_t st) {
  int64_t nb = blocks_for(C.total_slots, kThreads);
  int64_t G = nb < 152 * 8 ? nb : 152 * 8;
  if (G < 1) G = 1;
  int64_t chunk = (C.total_slots + G - 1) / G;
  chunk = (chunk + kThreads - 1) / kThreads * kThreads;
  G = (C.total_slots + chunk - 1) / chunk;
  if (G < 1) G = 1;
  k_bbox<<<(unsigned int)G, kThreads, 0, st>>>(C, chunk);
}

void launch_params(const DevCtx &C, cudaStream_t st, int step) { k_params<<<1, 256, 0, st>>>(C, step); }

void launch_count(const DevCtx &C, cudaStream_t st, int step) {
  k_count<<<blocks_for(C.total_slots, kThreads), kThreads, 0, st>>>(C, step ? C.a.pkey_hist : nullptr);
}

void launch_scan(const DevCtx &C, cudaStream_t st, uint32_t *partial) {
  int64_t G = blocks_for(C.total_slots, 4096);
  if (G > 1024) G = 1024;
  if (G < 1) G = 1;
  int64_t chunk = (C.total_slots + G - 1) / G;
  chunk = (chunk + 1023) / 1024 * 1024;
  G = (C.total_slots + chunk - 1) / chunk;
  if (G < 1) G = 1;
  k_scan_up<<<(unsigned int)G, 1024, 0, st>>>(C, chunk, partial);
  k_scan_top<<<1, 1024, 0, st>>>(partial, (int)G);
  k_scan_down<<<(unsigned int)G, 1024, 0, st>>>(C, chunk, partial);
}

void launch_place(const DevCtx &C, cudaStream_t st, int step) {
  k_place<<<blocks_for(C.total_slots, kThreads), kThreads, 0, st>>>(C, step ? C.c : C.q, step ? 0 : 1);
}

}  // namespace bdm
