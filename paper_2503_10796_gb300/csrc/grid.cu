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

// step: the bounding box of a step iteration, which an iteration that
// keeps the last build's grid (grid reuse) does not need.
__global__ void __launch_bounds__(kThreads) k_bbox(DevCtx C, int64_t chunk, int step) {
  __shared__ unsigned long long sh[kThreads / 32][7];
  __shared__ int tile_sim[2];
  if (step && C.g->reuse) return;
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
      const int64_t stop = end < last ? end : last;
      auto add = [&](double x, double y, double z, double d) {
        const unsigned long long kx = ord_key(x), ky = ord_key(y), kz = ord_key(z), kd = ord_key(d);
        acc.mn[0] = kx < acc.mn[0] ? kx : acc.mn[0];
        acc.mn[1] = ky < acc.mn[1] ? ky : acc.mn[1];
        acc.mn[2] = kz < acc.mn[2] ? kz : acc.mn[2];
        acc.mx[0] = kx > acc.mx[0] ? kx : acc.mx[0];
        acc.mx[1] = ky > acc.mx[1] ? ky : acc.mx[1];
        acc.mx[2] = kz > acc.mx[2] ? kz : acc.mx[2];
        acc.dm = kd > acc.dm ? kd : acc.dm;
      };
      // four slots per thread and round: 16 independent loads in flight
      const int64_t step = blockDim.x;
      int64_t slot = begin + threadIdx.x;
      for (; slot + 3 * step < stop; slot += 4 * step) {
        double x[4], y[4], z[4], d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = C.a.x[slot + u * step]; y[u] = C.a.y[slot + u * step];
          z[u] = C.a.z[slot + u * step]; d[u] = C.a.d[slot + u * step];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) add(x[u], y[u], z[u], d[u]);
      }
      for (; slot < stop; slot += step) add(C.a.x[slot], C.a.y[slot], C.a.z[slot], C.a.d[slot]);
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

// One thread per simulation; thread 0 then lays out the cell ranges.  An
// iteration that keeps the last build's grid (grid reuse) only advances the
// counters.
__global__ void k_params(DevCtx C, int32_t step) {
  Globals *g = C.g;
  if (step && g->reuse) {
    for (int k = threadIdx.x; k < C.n_sims; k += blockDim.x) {
      const int s = C.order[k];
      if (s < 0) continue;
      SimState &st = C.ss[s];
      st.it = st.t;
      st.t += 1;
      st.updates += (unsigned long long)(st.n > 0 ? st.n : 0);
      for (int a = 0; a < 3; ++a) { st.bmin[a] = ~0ull; st.bmax[a] = 0ull; }
      st.dmax = 0ull;
    }
    if (threadIdx.x == 0) {
      g->n_ovf = 0u;
      g->reused = 1u;
    }
    return;
  }
  for (int k = threadIdx.x; k < C.n_sims; k += blockDim.x) {
    int s = C.order[k];
    if (s < 0) continue;
    const SimConst &sc = C.sc[s];
    SimState &st = C.ss[s];
    st.ncell = st.n;
    st.valid = 0;
    st.same_grid = 0;
    st.keep_boxes = 0;
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
    // box length: the user's value, else the largest diameter (times the
    // tuned scale, which only simulations without static detection take)
    double L = sc.box_length > 0.0 ? sc.box_length : (sc.box_scale > 1.0 ? __dmul_rn(dmax, sc.box_scale) : dmax);
    st.L = L;
    bool ok = L > 0.0 && isfinite(L);
    int64_t nb = 1;
    if (sc.boundary == BOUND_TORUS) {
      // the grid tiles the space: floor(size / L) >= 3 boxes per axis of
      // length size / n from bmin (§4.4.11, toroidal)
      for (int a = 0; a < 3; ++a)
        if (!isfinite(st.o[a]) || !isfinite(mx[a])) ok = false;
      if (!ok) set_err(g, ERR_COORD | ERR_NONFINITE);
      const double q = ok ? floor(__ddiv_rn(sc.bsize, L)) : 0.0;
      if (ok && !(q >= 3.0 && q < (double)(1ll << kCoordBits) - 1.0)) {
        set_err(g, ERR_COORD | ERR_TORUS);
        ok = false;
      }
      if (ok) {
        L = __ddiv_rn(sc.bsize, q);
        st.L = L;
      }
      for (int a = 0; a < 3; ++a) {
        st.o[a] = sc.bmin;
        st.dims[a] = ok ? (int64_t)q : 1;
        nb *= st.dims[a];
      }
    } else {
      for (int a = 0; a < 3; ++a) {
        if (!isfinite(st.o[a]) || !isfinite(mx[a])) ok = false;
        double q = ok ? floor(__ddiv_rn(__dsub_rn(mx[a], st.o[a]), L)) : 0.0;
        if (!(q < (double)(1ll << kCoordBits) - 1.0)) { ok = false; q = 0.0; }
        st.dims[a] = (int64_t)q + 1;
        nb *= st.dims[a];
      }
      if (!ok) set_err(g, ERR_COORD | ERR_NONFINITE);
    }
    st.nboxes = nb;
    if (ok && (nb > sc.table_cap || nb >= (1ll << 32))) {
      set_err(g, ERR_TABLE);
      ok = false;
    }
    st.valid = ok ? 1 : 0;
    st.same_grid = (step && st.has_prev && ok && st.o[0] == st.prev_o[0] && st.o[1] == st.prev_o[1] &&
                    st.o[2] == st.prev_o[2] && L == st.prev_L && st.dims[0] == st.prev_dims[0] &&
                    st.dims[1] == st.prev_dims[1] && st.dims[2] == st.prev_dims[2]) ? 1 : 0;
    // after iterations that kept their grid (or a restored state), an agent
    // may have moved since the last build without moving in the last
    // iteration: the count then computes every box
    st.keep_boxes = (st.same_grid && !g->reused) ? 1 : 0;
    // float-float constants
    split_pos(L, st.Lh, st.Ll);
    double il = __ddiv_rn(1.0, L);
    split_pos(il, st.ilh, st.ill);
    // FP32 filter margin: truncated hi parts are off by < 1 ulp of values
    // below 2L; differences and squares add a few more ulps.
    st.marg = (float)(L * 0x1p-19) + 0x1p-30f;
    st.rmaxf = __double2float_ru(__dmul_rn(0.5, dmax));
    // grid reuse: an agent that stays within `skin` of its box (per axis)
    // still finds every partner in the 27-box stencil, as long as L - 2 skin
    // >= the largest diameter (with room for rounding)
    st.skin = __dsub_rn(__dmul_rn(0.5, __dsub_rn(L, dmax)), __dmul_rn(L, 0x1p-20));
    // bounds of the FP32 check on the leading part of an offset (its low
    // part is below 2^-23 of it: an inward margin of 2^-21 L covers it)
    st.skin_lo = -__double2float_rd(__dsub_rn(st.skin, __dmul_rn(L, 0x1p-21)));
    st.skin_hi = __double2float_rd(__dsub_rn(__dadd_rn(L, st.skin), __dmul_rn(L, 0x1p-21)));
    st.skin_pad = st.skin > 0.0 ? __double2float_ru(st.skin) : 0.f;
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
    g->tile_ticket = 0u;
    g->n_ovf = 0u;
    if (step) {
      g->n_builds += 1ull;
      g->reused = 0u;
    }
    int64_t cells = 0;
    for (int k = 0; k < C.n_sims; ++k) {
      const int s = C.order[k];
      if (s < 0) break;
      C.ss[s].cell_base = cells;
      C.ss[s].cell_cursor = (unsigned long long)cells;
      cells += C.ss[s].n;
    }
    g->n_cells = cells;
  }
}

// ---------------------------------------------------------------------------
// S1: box index, per-box count with timestamps, dirty marks for static
// detection (§5.5).
// ---------------------------------------------------------------------------
// Table update without a retry loop.  A max with (stamp << 43) turns an
// entry of an older build into an empty current one (count 0, clean) and
// leaves a current entry alone, since every current word is at least that
// value; the add that follows (same thread, same address, so ordered after
// the max) returns the count before it, i.e. the rank of the first agent
// added.  Dirty marks are an OR.  A count that would pass the 10-bit field
// (or a returned word of another stamp, which only such a carry makes) is a
// table error: the scan then empties every box of the build, so no later
// kernel indexes cells through a corrupted word.
__device__ __forceinline__ void tab_revive(unsigned long long *e, uint32_t stamp) {
  atomicMax(e, (unsigned long long)stamp << 43);
}

__device__ __forceinline__ uint32_t tab_add(unsigned long long *e, uint32_t stamp, bool dirty, uint32_t count,
                                            Globals *g) {
  tab_revive(e, stamp);
  const unsigned long long old = atomicAdd(e, (unsigned long long)count << 32);
  if (dirty) atomicOr(e, 1ull << 42);
  const uint32_t cnt = ent_count(old);
  if (ent_stamp(old) != stamp || cnt + count > kMaxBoxCount) set_err(g, ERR_TABLE);
  return cnt;
}

__device__ __forceinline__ void tab_mark_dirty(unsigned long long *e, uint32_t stamp) {
  tab_revive(e, stamp);
  atomicOr(e, 1ull << 42);
}

// step: the step's build, which reads each agent's box of the last step
// (the history of static detection and of the unchanged-agent shortcut)
// before it rewrites it; a query build (step = 0) writes its boxes to the
// query keys and leaves the history alone.  Every load that does not depend
// on another is issued before the first test, so that one thread waits for
// few round trips in a row.
// kOne: the context holds one simulation, which owns every slot below
// total_slots (no per-slot simulation index to wait for).
template <bool kOne>
__global__ void __launch_bounds__(kAgentThreads) k_count(DevCtx C, int step) {
  if (step && C.g->reuse) return;  // the iteration keeps the last build's grid
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = slot < C.total_slots;
  const int64_t sl = in ? slot : C.total_slots - 1;
  const int sim = kOne ? 0 : C.a.sim[sl];
  const double p[3] = {C.a.x[sl], C.a.y[sl], C.a.z[sl]};
  const uint64_t pk_prev_in = step ? C.a.pkey[sl] : 0ull;
  const uint8_t fl = step ? C.a.flags[sl] : (uint8_t)0;
  const uint32_t stamp = C.g->stamp & kStampMask;
  const SimConst &sc = C.sc[sim < 0 ? 0 : sim];
  const SimState &s = C.ss[sim < 0 ? 0 : sim];
  const bool valid = in && sim >= 0 && sl - sc.base < s.n && s.valid;
  const bool changed = valid && step && (fl & FLAG_CHANGED) != 0;
  uint32_t c[3] = {0u, 0u, 0u};
  if (!valid) {
  } else if (step && s.keep_boxes && !changed) {
    // unchanged agent, unchanged grid: the box of the last iteration
    c[0] = (uint32_t)(pk_prev_in & kCoordMask);
    c[1] = (uint32_t)((pk_prev_in >> kCoordBits) & kCoordMask);
    c[2] = (uint32_t)((pk_prev_in >> (2 * kCoordBits)) & kCoordMask);
  } else {
    for (int a = 0; a < 3; ++a) c[a] = grid_coord(s, p[a], a);
  }
  const uint64_t pk = (uint64_t)c[0] | ((uint64_t)c[1] << kCoordBits) | ((uint64_t)c[2] << (2 * kCoordBits));
  const int64_t idx =
      sc.table_base + (int64_t)(c[0] + (uint32_t)s.dims[0] * (c[1] + (uint32_t)s.dims[1] * c[2]));
  // Runs of neighbouring lanes in one box add their count with one atomic
  // (agents of a box are neighbours once the storage is sorted; a box met
  // in two runs takes two atomics).  Lanes without an agent get keys of
  // their own.
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned long long key = valid ? (unsigned long long)idx : (0xFFFFFFFF00000000ull | (unsigned)lane);
  const unsigned long long prev = __shfl_up_sync(FULL, key, 1);
  const unsigned H = __ballot_sync(FULL, lane == 0 || prev != key);
  const int start = 31 - __clz(H & (FULL >> (31 - lane)));
  const unsigned above = H & ~(FULL >> (31 - lane));
  const int end = above ? __ffs(above) - 2 : 31;
  const unsigned run = (end == 31 ? FULL : ((1u << (end + 1)) - 1u)) & ~((1u << start) - 1u);
  const unsigned dirty_any = __ballot_sync(FULL, changed) & run;
  uint32_t base = 0;
  if (valid && lane == start)
    base = tab_add(&C.tab.e[idx], stamp, dirty_any != 0u, (uint32_t)(end - start + 1), C.g);
  base = __shfl_sync(FULL, base, start);
  if (!valid) return;
  if (step)
    C.a.pkey[slot] = pk;
  else
    C.qkey[slot] = pk;
  if (changed && s.same_grid && pk_prev_in != pk) {
    int64_t px, py, pz;
    unpack_coords(pk_prev_in, px, py, pz);
    if (px < s.dims[0] && py < s.dims[1] && pz < s.dims[2])
      tab_mark_dirty(&C.tab.e[sc.table_base + linear_box(s, px, py, pz)], stamp);
  }
  C.a.rank[slot] = base + (uint32_t)(lane - start);
}


// ---------------------------------------------------------------------------
// S2: every box gets a contiguous range of cells, claimed by its leader
// (the rank-0 agent, which contributes the box's count): an exclusive
// prefix sum over the leaders in slot order, or ranges claimed by atomics
// (see k_scan); then placement of every agent at start + rank.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

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

// Box starts: every box's leader (the agent of rank 0) receives the first
// cell of its box.  kOrdered: one pass with decoupled look-back, so that the
// boxes' ranges follow the storage order of their leaders.  A block claims
// the next tile through a ticket (so every earlier tile belongs to a block
// that is already running), sums its leaders' counts, publishes that sum,
// and walks back over the earlier tiles' published values until it meets an
// inclusive prefix; it then publishes its own inclusive prefix.  Otherwise a
// block claims its leaders' cells with one atomic add on its simulation's
// cell cursor (or, in a block that holds leaders of several simulations,
// one per leader): no block waits for another, and the tiles' ranges follow
// the order in which the blocks finish.  The iterations that re-sort the
// storage into cell order take the ordered scan, so that arrival order
// never reaches the storage.  Each thread takes
// kScanItems slots of the tile (strided, so that loads coalesce) and issues
// all their loads before any is used.  Every wait is bounded: a tile that
// never publishes latches ERR_TIMEOUT.  Tile words carry the build's stamp,
// so they need no clearing between builds.
constexpr uint32_t kLookSpin = 1u << 20;
constexpr uint32_t kTestSpin = 64u;  // polls per awaited tile under TEST_SCAN_TIMEOUT

__device__ __forceinline__ void tile_publish(unsigned long long *w, uint32_t stamp, uint32_t state, uint32_t v) {
  *(volatile unsigned long long *)w =
      ((unsigned long long)stamp << 34) | ((unsigned long long)state << 32) | (unsigned long long)v;
}

template <bool kOrdered, bool kOne>
__global__ void __launch_bounds__(kScanThreads) k_scan(DevCtx C, const uint64_t *keys, int step) {
  __shared__ uint32_t sh[33];
  __shared__ uint32_t s_tile, s_base;
  __shared__ int s_lo, s_hi;
  if (step && C.g->reuse) return;  // every block: none waits for another
  if (threadIdx.x == 0) {
    s_tile = kOrdered ? atomicAdd(&C.g->tile_ticket, 1u) : blockIdx.x;
    s_base = 0u;
    s_lo = 0x7fffffff;
    s_hi = -1;
  }
  __syncthreads();
  const uint32_t tile = s_tile;
  // each thread takes kScanItems consecutive slots (vector loads)
  const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t rank[kScanItems];
  uint64_t pk[kScanItems];
  int sim[kScanItems];
  if (base + kScanItems <= C.total_slots) {
    const uint4 r4 = *reinterpret_cast<const uint4 *>(C.a.rank + base);
    const int4 s4 = kOne ? make_int4(0, 0, 0, 0) : *reinterpret_cast<const int4 *>(C.a.sim + base);
    const ulonglong2 k01 = *reinterpret_cast<const ulonglong2 *>(keys + base);
    const ulonglong2 k23 = *reinterpret_cast<const ulonglong2 *>(keys + base + 2);
    rank[0] = r4.x; rank[1] = r4.y; rank[2] = r4.z; rank[3] = r4.w;
    sim[0] = s4.x; sim[1] = s4.y; sim[2] = s4.z; sim[3] = s4.w;
    pk[0] = k01.x; pk[1] = k01.y; pk[2] = k23.x; pk[3] = k23.y;
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const int64_t slot = base + i;
      const int64_t sl = slot < C.total_slots ? slot : C.total_slots - 1;
      rank[i] = C.a.rank[sl];
      pk[i] = keys[sl];
      sim[i] = slot < C.total_slots ? (kOne ? 0 : C.a.sim[sl]) : -1;
    }
  }
  unsigned long long e[kScanItems];
  int64_t idx[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t slot = base + i;
    idx[i] = -1;
    e[i] = 0ull;
    if (sim[i] >= 0) {
      const SimConst &sc = C.sc[sim[i]];
      const SimState &s = C.ss[sim[i]];
      if (slot - sc.base < s.n && s.valid && rank[i] == 0u) {
        int64_t cx, cy, cz;
        unpack_coords(pk[i], cx, cy, cz);
        idx[i] = sc.table_base + linear_box(s, cx, cy, cz);
        e[i] = C.tab.e[idx[i]];
      }
    }
  }
  uint32_t loc[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = sum;
    sum += idx[i] >= 0 ? ent_count(e[i]) : 0u;
  }
  uint32_t agg;
  const uint32_t ex = block_exscan_u32(sum, sh, &agg);
  const uint32_t stamp = C.g->stamp & kStampMask;
  bool one = true;  // unordered: the block's leaders belong to one simulation
  if (!kOrdered) {
    int smin = 0x7fffffff, smax = -1;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
      if (idx[i] >= 0) {
        smin = sim[i] < smin ? sim[i] : smin;
        smax = sim[i] > smax ? sim[i] : smax;
      }
    smin = __reduce_min_sync(0xffffffffu, smin);
    smax = __reduce_max_sync(0xffffffffu, smax);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&s_lo, smin);
      atomicMax(&s_hi, smax);
    }
    __syncthreads();
    one = s_lo == s_hi;
    if (one && threadIdx.x == 0 && agg)
      s_base = (uint32_t)atomicAdd(&C.ss[s_lo].cell_cursor, (unsigned long long)agg);
  } else if (threadIdx.x < 32) {
    // warp 0 looks back 32 tiles at a time: the nearest inclusive prefix
    // ends the walk, the aggregates before it are added
    const int lane = threadIdx.x;
    uint32_t run = 0;
    // under the timeout test hook the walk waits for a stamp that no tile of
    // this build publishes, with a short bound
    const bool test = (C.g->test_flags & TEST_SCAN_TIMEOUT) != 0u;
    const uint32_t want = test ? ((stamp + 1u) & kStampMask) : stamp;
    const uint32_t limit = test ? kTestSpin : kLookSpin;
    if (tile == 0) {
      if (lane == 0) tile_publish(&C.tstat[0], stamp, 2u, agg);
    } else {
      if (lane == 0) tile_publish(&C.tstat[tile], stamp, 1u, agg);
      for (int64_t j = (int64_t)tile - 1 - lane;; j -= 32) {
        uint32_t state = 2u, v = 0u;
        if (j >= 0) {
          unsigned long long w = 0;
          uint32_t spins = 0;
          for (;;) {
            w = *(volatile unsigned long long *)&C.tstat[j];
            if ((uint32_t)(w >> 34) == want && ((w >> 32) & 3ull) != 0ull) break;
            if (++spins >= limit) break;
            __nanosleep(32);
          }
          if (spins >= limit) {
            set_err(C.g, ERR_TIMEOUT);
            w = 2ull << 32;  // give up: treat as a prefix of 0
          }
          state = (uint32_t)(w >> 32) & 3u;
          v = (uint32_t)w;
        }
        const unsigned pm = __ballot_sync(0xffffffffu, state == 2u);
        const int first = pm ? __ffs(pm) - 1 : 31;
        run += __reduce_add_sync(0xffffffffu, lane <= first ? v : 0u);
        if (pm) break;
      }
      if (lane == 0) tile_publish(&C.tstat[tile], stamp, 2u, run + agg);
    }
    if (lane == 0) s_base = run;
  }
  __syncthreads();
  // each leader writes its box's first cell into the low half of the table
  // word (a 32-bit store: the high half, stamp | dirty | count, stays as the
  // count left it).  After a table error every leader writes an empty
  // current word instead, so that placement, forces and queries see no
  // agents in any box of the build.
  const bool bad = (C.g->err & ERR_TABLE) != 0u;
  const uint32_t off = s_base + ex;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (idx[i] >= 0) {
      unsigned long long *w = &C.tab.e[idx[i]];
      if (bad)
        *w = (unsigned long long)stamp << 43;
      else if (one)
        *reinterpret_cast<uint32_t *>(w) = off + loc[i];
      else
        *reinterpret_cast<uint32_t *>(w) =
            (uint32_t)atomicAdd(&C.ss[sim[i]].cell_cursor, (unsigned long long)ent_count(e[i]));
    }
  }
}

// zero_f32: clear the FP32 force of every placed FP32-path agent (the
// symmetric force walk adds into it).
template <bool kOne>
__global__ void __launch_bounds__(kAgentThreads) k_place(DevCtx C, Cells cells, const uint64_t *keys, int fp64_records,
                                                   int zero_f32) {
  // fp64_records is set only for query builds: a step iteration that keeps
  // the last build's grid places nothing
  if (!fp64_records && C.g->reuse) return;
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= C.total_slots) return;
  // every per-slot load first: they do not depend on one another
  const int sim = kOne ? 0 : C.a.sim[slot];
  const uint64_t pk = keys[slot];
  const uint32_t rank = C.a.rank[slot];
  const double pos[3] = {C.a.x[slot], C.a.y[slot], C.a.z[slot]};
  const double dia = C.a.d[slot];
  const uint8_t fl = cells.flag ? C.a.flags[slot] : (uint8_t)0;
  const uint8_t nz = cells.flag ? C.a.nnz[slot] : (uint8_t)0;
  if (sim < 0) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (slot - sc.base >= s.n || !s.valid) return;
  const uint32_t c[3] = {(uint32_t)(pk & kCoordMask), (uint32_t)((pk >> kCoordBits) & kCoordMask),
                         (uint32_t)((pk >> (2 * kCoordBits)) & kCoordMask)};
  const uint32_t off = c[0] + (uint32_t)s.dims[0] * (c[1] + (uint32_t)s.dims[1] * c[2]);
  const unsigned long long e = C.tab.e[sc.table_base + off];
  if (rank >= ent_count(e)) return;  // box overflow (error latched by the count)
  const int64_t p = (int64_t)ent_start(e) + rank;
  cells.slot[p] = (int32_t)slot;
  cells.sim[p] = sim;
  cells.pkey[p] = pk;
  if (cells.flag) cells.flag[p] = (!(fl & (FLAG_CHANGED | FLAG_GHOST)) && nz <= 1) ? CELL_STATIC_ELIGIBLE : 0;
  const double r = half_of(dia);
  const bool fp64 = sc.precision == BDM_PREC_FP64;
  if (fp64_records || fp64) cells.r64[p] = make_double4_32a(pos[0], pos[1], pos[2], r);
  if (!fp64_records) {
    // the step's build: box-relative float-float records, whose leading
    // parts are the candidate filter of both paths (the FP64 path needs no
    // tails)
    float h[3], l[3], rh, rl;
    for (int a = 0; a < 3; ++a) {
      // offset inside the own box, exact in FP64: (x - o) - c L
      const double av = __dsub_rn(pos[a], s.o[a]);
      const double w = __fma_rn(neg_u32_to_double(c[a]), s.L, av);
      split_ff(w, h[a], l[a]);
    }
    split_ff(r, rh, rl);
    cells.r0[p] = make_float4(h[0], h[1], h[2], rh);
    if (!fp64) {
      cells.r1[p] = make_float4(l[0], l[1], l[2], rl);
      if (zero_f32) cells.f32[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}


// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

// Grid reuse, at the start of a step iteration: keep the last build's grid
// unless a rebuild is due (an agent left its skin, the host changed the
// simulation, or this iteration re-sorts); an iteration that permutes the
// storage into the cell order (sort == 2) makes the next one rebuild.
__global__ void k_decide(DevCtx C, int sort) {
  Globals *g = C.g;
  bool ok = sort == 0 && g->regrid == 0u && g->n_builds > 0ull;
  for (int k = 0; k < C.n_sims && ok; ++k) {
    const int s = C.order[k];
    if (s < 0) break;
    const SimState &st = C.ss[s];
    if (st.n > 0 && !(st.valid && st.skin > 0.0)) ok = false;
  }
  g->reuse = ok ? 1u : 0u;
  g->regrid = sort == 2 ? 1u : 0u;
}

// Forces of the symmetric FP32 walks start from zero; the placement clears
// them in iterations that build the grid, this kernel in those that keep it.
__global__ void __launch_bounds__(kAgentThreads) k_zero_f32(DevCtx C) {
  if (!C.g->reuse) return;
  const int64_t n = C.g->n_cells;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    if (C.sc[C.c.sim[p]].precision != BDM_PREC_FP64) C.c.f32[p] = make_float4(0.f, 0.f, 0.f, 0.f);
}

void launch_decide(const DevCtx &C, cudaStream_t st, int sort) { k_decide<<<1, 1, 0, st>>>(C, sort); }

// Blocks of the force clearing, which exits at once in iterations that
// build the grid: at most 16 per SM (full occupancy of 128-thread blocks).
static inline unsigned int capped_blocks(int64_t n) {
  const unsigned int nb = blocks_for(n, kAgentThreads);
  return nb < 152u * 16u ? nb : 152u * 16u;
}

void launch_zero_f32(const DevCtx &C, cudaStream_t st) {
  k_zero_f32<<<capped_blocks(C.total_slots), kAgentThreads, 0, st>>>(C);
}

void launch_bbox(const DevCtx &C, cudaStream_t st, int step) {
  int64_t nb = blocks_for(C.total_slots, kThreads);
  int64_t G = nb < 152 * 8 ? nb : 152 * 8;
  if (G < 1) G = 1;
  int64_t chunk = (C.total_slots + G - 1) / G;
  chunk = (chunk + kThreads - 1) / kThreads * kThreads;
  G = (C.total_slots + chunk - 1) / chunk;
  if (G < 1) G = 1;
  k_bbox<<<(unsigned int)G, kThreads, 0, st>>>(C, chunk, step);
}

void launch_params(const DevCtx &C, cudaStream_t st, int step) { k_params<<<1, 256, 0, st>>>(C, step); }

void launch_count(const DevCtx &C, cudaStream_t st, int step) {
  // a full grid, one slot per thread (a capped grid looping over tiles ran
  // the count 0.14 -> 0.17 ms at 8.4M agents)
  if (C.n_sims == 1)
    k_count<true><<<blocks_for(C.total_slots, kAgentThreads), kAgentThreads, 0, st>>>(C, step);
  else
    k_count<false><<<blocks_for(C.total_slots, kAgentThreads), kAgentThreads, 0, st>>>(C, step);
}

int64_t scan_tiles(int64_t total_slots) { return (total_slots + kScanTile - 1) / kScanTile; }

void launch_scan(const DevCtx &C, cudaStream_t st, int step, int ordered) {
  const int64_t G = scan_tiles(C.total_slots);
  const uint64_t *keys = step ? C.a.pkey : C.qkey;
  const bool one = C.n_sims == 1;
  if (ordered) {
    if (one) k_scan<true, true><<<(unsigned int)G, kScanThreads, 0, st>>>(C, keys, step);
    else k_scan<true, false><<<(unsigned int)G, kScanThreads, 0, st>>>(C, keys, step);
  } else {
    if (one) k_scan<false, true><<<(unsigned int)G, kScanThreads, 0, st>>>(C, keys, step);
    else k_scan<false, false><<<(unsigned int)G, kScanThreads, 0, st>>>(C, keys, step);
  }
}

void launch_place(const DevCtx &C, cudaStream_t st, int step, int zero_f32) {
  const unsigned int nb = blocks_for(C.total_slots, kAgentThreads);  // full grid (capped: 0.18 -> 0.23 ms)
  if (C.n_sims == 1)
    k_place<true><<<nb, kAgentThreads, 0, st>>>(C, step ? C.c : C.q, step ? C.a.pkey : C.qkey, step ? 0 : 1,
                                                 step ? zero_f32 : 0);
  else
    k_place<false><<<nb, kAgentThreads, 0, st>>>(C, step ? C.c : C.q, step ? C.a.pkey : C.qkey, step ? 0 : 1,
                                                  step ? zero_f32 : 0);
}

}  // namespace bdm
