// Queries and transfers: box index per agent (parity hook of S1), neighbor
// pairs (§4.4.3 ForEachNeighbor: radius query or overlap query, decided in
// FP64 exactly as defined), gathers by caller ID, and agent upload.
#include "pair.cuh"

namespace bdm {

static inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

// Box index per caller ID, computed as S1 computes it (no table needed).
__global__ void k_boxids(DevCtx C, int sim, int64_t *out) {
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  int64_t slot = sc.base + i;
  int64_t id = C.a.id[slot];
  if (!s.valid) {
    out[id] = -1;
    return;
  }
  double p[3] = {C.a.x[slot], C.a.y[slot], C.a.z[slot]};
  int64_t c[3];
  for (int a = 0; a < 3; ++a) c[a] = grid_coord(s, p[a], a);  // as the step's count
  out[id] = linear_box(s, c[0], c[1], c[2]);
}

void launch_boxids(const DevCtx &C, cudaStream_t st, int sim, int64_t *out_by_id) {
  int64_t n = C.total_slots;
  k_boxids<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, sim, out_by_id);
}

// ---------------------------------------------------------------------------
// Neighbor pairs over the query cells (FP64 records).  Every agent i counts
// (then writes) the j with ID above its own that satisfy the predicate;
// offsets come from an exclusive scan over IDs, and each agent sorts its own
// short list, so the output is ordered by (i, j).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool pair_hit(const SimConst &sc, double4_32a a, double4_32a b, double R2,
                                         bool radius_mode) {
  const double dx = coord_diff(sc, a.x, b.x), dy = coord_diff(sc, a.y, b.y), dz = coord_diff(sc, a.z, b.z);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  if (radius_mode) return s < R2;
  return __dsub_rn(__dadd_rn(a.w, b.w), __dsqrt_rn(s)) > 0.0;
}

template <bool kWrite>
__global__ void k_pairs(DevCtx C, int sim, int64_t cell_base, int64_t n, double R2, int radius_mode,
                        int64_t *counts, const int64_t *offsets, int64_t *pairs, int64_t cap) {
  int64_t p = cell_base + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cell_base + n) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  const Cells &Q = C.q;
  int64_t id = C.a.id[Q.slot[p]];
  double4_32a o = Q.r64[p];
  int64_t cx, cy, cz;
  unpack_coords(Q.pkey[p], cx, cy, cz);
  uint32_t stamp = C.g->stamp & kStampMask;
  int64_t cnt = 0;
  int64_t off = kWrite ? offsets[id] : 0;
  for (int dz = -1; dz <= 1; ++dz) {
    for (int dy = -1; dy <= 1; ++dy) {
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t idx;
        if (!stencil_index(sc, s, cx, cy, cz, dx, dy, dz, idx)) continue;
        const unsigned long long e = C.tab.e[idx];
        const uint32_t c = ent_live(e, stamp);
        if (!c) continue;
        const int64_t start = ent_start(e);
        for (int64_t j = start; j < start + c; ++j) {
          int64_t jd = C.a.id[Q.slot[j]];
          if (jd <= id) continue;
          if (!pair_hit(sc, o, Q.r64[j], R2, radius_mode != 0)) continue;
          if (kWrite) {
            int64_t k = off + cnt;
            if (k < cap) {
              // insertion into this agent's sorted run
              int64_t m = k;
              while (m > off && pairs[2 * (m - 1) + 1] > jd) {
                pairs[2 * m] = pairs[2 * (m - 1)];
                pairs[2 * m + 1] = pairs[2 * (m - 1) + 1];
                --m;
              }
              pairs[2 * m] = id;
              pairs[2 * m + 1] = jd;
            }
          }
          ++cnt;
        }
      }
    }
  }
  if (!kWrite) counts[id] = cnt;
}

// Exclusive scan of n int64 values in place; returns the total through
// *total_dev (device).
__global__ void __launch_bounds__(1024) k_scan64_up(const int64_t *v, int64_t n, int64_t chunk, int64_t *part) {
  __shared__ long long sh[32];
  int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  long long s = 0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) s += v[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_scan64_top(int64_t *part, int G, int64_t *total) {
  if (threadIdx.x != 0) return;
  int64_t run = 0;
  for (int g = 0; g < G; ++g) {
    int64_t v = part[g];
    part[g] = run;
    run += v;
  }
  *total = run;
}

__global__ void __launch_bounds__(1024) k_scan64_down(int64_t *v, int64_t n, int64_t chunk, const int64_t *part) {
  __shared__ long long sh[33];
  int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  long long base = part[blockIdx.x];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t0 = b; t0 < e; t0 += blockDim.x) {
    int64_t i = t0 + threadIdx.x;
    long long x = i < e ? v[i] : 0, inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long run = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        long long t = sh[w];
        sh[w] = run;
        run += t;
      }
      sh[32] = run;
    }
    __syncthreads();
    if (i < e) v[i] = base + sh[warp] + inc - x;
    base += sh[32];
    __syncthreads();
  }
}

int64_t launch_pairs(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n, double radius,
                     int64_t *counts, int64_t *offsets, int64_t *pairs_dev, int64_t cap, uint32_t *partial,
                     cudaError_t *err) {
  (void)partial;
  bool rmode = radius >= 0.0;
  double R2 = radius * radius;
  unsigned int nb = blocks_for(n > 0 ? n : 1, kThreads);
  if (pairs_dev == nullptr) {
    k_pairs<false><<<nb, kThreads, 0, st>>>(C, sim, cell_base, n, R2, rmode, counts, nullptr, nullptr, 0);
    // exclusive scan counts -> offsets (offsets also holds the part sums
    // after n entries: offsets has n + 1024 + 1 slots)
    cudaMemcpyAsync(offsets, counts, sizeof(int64_t) * (size_t)(n > 0 ? n : 1), cudaMemcpyDeviceToDevice, st);
    int64_t G = (n + 4095) / 4096;
    if (G > 1024) G = 1024;
    if (G < 1) G = 1;
    int64_t chunk = (n + G - 1) / G;
    chunk = (chunk + 1023) / 1024 * 1024;
    if (chunk < 1024) chunk = 1024;
    G = (n + chunk - 1) / chunk;
    if (G < 1) G = 1;
    int64_t *part = offsets + n;
    int64_t *total = part + 1024;
    k_scan64_up<<<(unsigned int)G, 1024, 0, st>>>(offsets, n, chunk, part);
    k_scan64_top<<<1, 32, 0, st>>>(part, (int)G, total);
    k_scan64_down<<<(unsigned int)G, 1024, 0, st>>>(offsets, n, chunk, part);
    int64_t h_total = 0;
    cudaMemcpyAsync(&h_total, total, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    *err = cudaStreamSynchronize(st);
    return h_total;
  }
  k_pairs<true><<<nb, kThreads, 0, st>>>(C, sim, cell_base, n, R2, rmode, counts, offsets, pairs_dev, cap);
  *err = cudaGetLastError();
  return 0;
}

// ---------------------------------------------------------------------------
// Gathers by caller ID and uploads.
// ---------------------------------------------------------------------------
__global__ void k_gather_agents(DevCtx C, int64_t base, int64_t n, double *xyz, double *diam) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t slot = base + i;
  int64_t id = C.a.id[slot];
  if (xyz) {
    xyz[3 * id] = C.a.x[slot];
    xyz[3 * id + 1] = C.a.y[slot];
    xyz[3 * id + 2] = C.a.z[slot];
  }
  if (diam) diam[id] = C.a.d[slot];
}

void launch_gather_agents(const DevCtx &C, cudaStream_t st, int sim, int64_t base, int64_t n, double *xyz,
                          double *diam) {
  (void)sim;
  if (n <= 0) return;
  k_gather_agents<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, xyz, diam);
}

__global__ void k_gather_forces(DevCtx C, int sim, int64_t cell_base, int64_t n, double *force, int32_t *nnz,
                                uint8_t *stat, int32_t *overlaps) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = cell_base + i;
  if (C.c.sim[p] != sim) return;
  int64_t id = C.a.id[C.c.slot[p]];
  bool st = C.c.stat[p] != 0;
  double f[3] = {0.0, 0.0, 0.0};
  int32_t nz = 0, ov = -1;
  if (!st) {
    if (C.sc[sim].precision == BDM_PREC_FP64) {
      double4_32a F = C.c.f64[p];
      f[0] = F.x; f[1] = F.y; f[2] = F.z;
      nz = (int32_t)C.c.nnz[p];
      ov = (int32_t)F.w;
    } else {
      // FP32 path: w carries the pair counts
      float4 F = C.c.f32[p];
      f[0] = F.x; f[1] = F.y; f[2] = F.z;
      uint32_t o, z;
      decode_counts(F.w, o, z);
      nz = (int32_t)(z > 255u ? 255u : z);
      ov = (int32_t)o;
    }
  } else {
    nz = (int32_t)C.a.nnz[C.c.slot[p]];
  }
  if (force) {
    force[3 * id] = f[0];
    force[3 * id + 1] = f[1];
    force[3 * id + 2] = f[2];
  }
  if (nnz) nnz[id] = nz;
  if (stat) stat[id] = st ? 1 : 0;
  if (overlaps) overlaps[id] = ov;
}

void launch_gather_forces(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n, double *force,
                          int32_t *nnz, uint8_t *stat, int32_t *overlaps) {
  if (n <= 0) return;
  k_gather_forces<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, sim, cell_base, n, force, nnz, stat, overlaps);
}

__global__ void k_count_flags(DevCtx C, int sim, int64_t cell_base, int64_t n, unsigned long long *counts2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int st = 0, mv = 0;
  if (i < n) {
    int64_t p = cell_base + i;
    if (C.c.sim[p] == sim) {
      st = C.c.stat[p] ? 1u : 0u;
      mv = (!st && (C.a.flags[C.c.slot[p]] & FLAG_CHANGED)) ? 1u : 0u;
    }
  }
  unsigned int a = __reduce_add_sync(0xffffffffu, st), b = __reduce_add_sync(0xffffffffu, mv);
  if ((threadIdx.x & 31) == 0) {
    if (a) atomicAdd(&counts2[0], (unsigned long long)a);
    if (b) atomicAdd(&counts2[1], (unsigned long long)b);
  }
}

void launch_count_flags(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n,
                        unsigned long long *counts2) {
  if (n <= 0) return;
  k_count_flags<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, sim, cell_base, n, counts2);
}

// Upload: xyz is n x 3 row-major (device memory), diam n values.
__global__ void k_set_agents(DevCtx C, int sim, int64_t base, int64_t n, int64_t cap, const double *xyz,
                             const double *diam) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  int64_t slot = base + i;
  C.a.sim[slot] = sim;
  if (i >= n) return;
  C.a.x[slot] = xyz[3 * i];
  C.a.y[slot] = xyz[3 * i + 1];
  C.a.z[slot] = xyz[3 * i + 2];
  double d = diam[i];
  C.a.d[slot] = d;
  // volume of a sphere of diameter d: (pi * ((d * d) * d)) / 6
  C.a.v[slot] = __ddiv_rn(__dmul_rn(3.141592653589793, __dmul_rn(__dmul_rn(d, d), d)), 6.0);
  C.a.id[slot] = (int32_t)i;
  C.a.flags[slot] = FLAG_CHANGED;
  C.a.nnz[slot] = 0;
  C.a.pkey[slot] = 0;
  C.a.rank[slot] = 0;
}

void launch_set_agents(const DevCtx &C, cudaStream_t st, int sim, int64_t base, int64_t n, int64_t cap,
                       const double *xyz, const double *diam) {
  if (cap <= 0) return;
  k_set_agents<<<blocks_for(cap, kThreads), kThreads, 0, st>>>(C, sim, base, n, cap, xyz, diam);
}

// New positions (and, when diam is given, diameters) of the agents of a
// simulation, by ID, keeping the storage order and the history; an agent
// whose values change is marked changed (static detection, box reuse).
__global__ void k_update_agents(DevCtx C, int64_t base, int64_t n, const double *xyz, const double *diam) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = base + i;
  const int64_t id = C.a.id[slot];
  const double x = xyz[3 * id], y = xyz[3 * id + 1], z = xyz[3 * id + 2];
  bool changed = x != C.a.x[slot] || y != C.a.y[slot] || z != C.a.z[slot];
  if (changed) {
    C.a.x[slot] = x; C.a.y[slot] = y; C.a.z[slot] = z;
  }
  if (diam) {
    const double d = diam[id];
    if (d != C.a.d[slot]) {
      C.a.d[slot] = d;
      // volume of a sphere of diameter d: (pi * ((d * d) * d)) / 6
      C.a.v[slot] = __ddiv_rn(__dmul_rn(3.141592653589793, __dmul_rn(__dmul_rn(d, d), d)), 6.0);
      changed = true;
    }
  }
  if (changed) C.a.flags[slot] |= FLAG_CHANGED;
}

// Ghost flags by ID (mask[id] != 0: read-only neighbour); an agent whose
// flag changes counts as changed (its neighbours' static checks).
__global__ void k_set_ghosts(DevCtx C, int64_t base, int64_t n, const uint8_t *mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = base + i;
  const uint8_t fl = C.a.flags[slot];
  const uint8_t g = mask[C.a.id[slot]] ? FLAG_GHOST : 0;
  if ((fl & FLAG_GHOST) != g) C.a.flags[slot] = (uint8_t)((fl & ~FLAG_GHOST & ~FLAG_STATIC) | g | FLAG_CHANGED);
}

void launch_set_ghosts(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const uint8_t *mask) {
  if (n <= 0) return;
  k_set_ghosts<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, mask);
}

void launch_update_agents(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const double *xyz,
                          const double *diam) {
  if (n <= 0) return;
  k_update_agents<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, xyz, diam);
}

// Smallest row with a non-finite coordinate or (diam given) a diameter that
// is not finite and > 0 (*bad stays all-ones when every row is valid).
__global__ void k_check_input(int64_t n, const double *xyz, const double *diam, unsigned long long *bad, int boundary,
                              double bmin, double bmax) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool ok = (!diam || (diam[i] > 0.0 && isfinite(diam[i])));
  for (int a = 0; a < 3; ++a) {
    const double v = xyz[3 * i + a];
    ok = ok && isfinite(v);
    // positions of a closed space lie in [bmin, bmax], of a torus in [bmin, bmax)
    if (boundary == BOUND_CLOSED) ok = ok && v >= bmin && v <= bmax;
    if (boundary == BOUND_TORUS) ok = ok && v >= bmin && v < bmax;
  }
  if (!ok) atomicMin(bad, (unsigned long long)i);
}

void launch_check_input(cudaStream_t st, int64_t n, const double *xyz, const double *diam, unsigned long long *bad,
                        int boundary, double bmin, double bmax) {
  k_check_input<<<blocks_for(n, kThreads), kThreads, 0, st>>>(n, xyz, diam, bad, boundary, bmin, bmax);
}

// ---------------------------------------------------------------------------
// Checkpoint state (bdm_get_state / bdm_set_state): per-agent arrays by
// caller ID, laid out as x, y, z, d, v (doubles), box key (uint64), flags,
// nnz (bytes), each array n long, in device staging memory.
// ---------------------------------------------------------------------------
struct StateArrays {
  double *x, *y, *z, *d, *v;
  uint64_t *pkey;
  uint8_t *flags, *nnz;
};

__host__ __device__ inline StateArrays state_arrays(void *base, int64_t n) {
  StateArrays a;
  char *b = (char *)base;
  a.x = (double *)b; a.y = a.x + n; a.z = a.y + n; a.d = a.z + n; a.v = a.d + n;
  a.pkey = (uint64_t *)(a.v + n);
  a.flags = (uint8_t *)(a.pkey + n);
  a.nnz = a.flags + n;
  return a;
}

int64_t state_array_bytes(int64_t n) { return n * (5 * 8 + 8 + 1 + 1); }

__global__ void k_state_gather(DevCtx C, int64_t base, int64_t n, StateArrays o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = base + i;
  const int64_t id = C.a.id[slot];
  o.x[id] = C.a.x[slot]; o.y[id] = C.a.y[slot]; o.z[id] = C.a.z[slot];
  o.d[id] = C.a.d[slot]; o.v[id] = C.a.v[slot];
  o.pkey[id] = C.a.pkey[slot];
  o.flags[id] = C.a.flags[slot];
  o.nnz[id] = C.a.nnz[slot];
}

// Rows in ID order into the slots of `sim` (the rest of its region is
// marked as owned and empty).
__global__ void k_state_scatter(DevCtx C, int sim, int64_t base, int64_t n, int64_t cap, StateArrays a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const int64_t slot = base + i;
  C.a.sim[slot] = sim;
  if (i >= n) return;
  C.a.x[slot] = a.x[i]; C.a.y[slot] = a.y[i]; C.a.z[slot] = a.z[i];
  C.a.d[slot] = a.d[i]; C.a.v[slot] = a.v[i];
  C.a.id[slot] = (int32_t)i;
  C.a.pkey[slot] = a.pkey[i];
  C.a.flags[slot] = a.flags[i];
  C.a.nnz[slot] = a.nnz[i];
  C.a.rank[slot] = 0;
}

// The first invalid row of restored arrays (a position not finite, a
// diameter or volume not finite and > 0, a flag outside the defined bits).
__global__ void k_state_check(int64_t n, StateArrays a, unsigned long long *bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool ok = isfinite(a.x[i]) && isfinite(a.y[i]) && isfinite(a.z[i]) && isfinite(a.d[i]) && a.d[i] > 0.0 &&
                  isfinite(a.v[i]) && a.v[i] > 0.0 && (a.flags[i] & ~(FLAG_CHANGED | FLAG_STATIC | FLAG_GHOST)) == 0;
  if (!ok) atomicMin(bad, (unsigned long long)i);
}

void launch_state_gather(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, void *staging) {
  if (n <= 0) return;
  k_state_gather<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, state_arrays(staging, n));
}

void launch_state_check(cudaStream_t st, int64_t n, const void *staging, unsigned long long *bad) {
  if (n <= 0) return;
  k_state_check<<<blocks_for(n, kThreads), kThreads, 0, st>>>(n, state_arrays(const_cast<void *>(staging), n), bad);
}

void launch_state_scatter(const DevCtx &C, cudaStream_t st, int sim, int64_t base, int64_t n, int64_t cap,
                          const void *staging, int64_t layout_n) {
  if (cap <= 0) return;
  k_state_scatter<<<blocks_for(cap, kThreads), kThreads, 0, st>>>(
      C, sim, base, n, cap, state_arrays(const_cast<void *>(staging), layout_n < 0 ? n : layout_n));
}

// Removal (§5.3.2): rows of the by-ID state arrays move from movers[k] into
// holes[k] (holes below the new count, movers at or above it, so no row is
// both); then every surviving row counts as changed and not static.
__global__ void k_state_move(StateArrays a, const int64_t *holes, const int64_t *movers, int64_t np) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int64_t h = holes[k], m = movers[k];
  a.x[h] = a.x[m]; a.y[h] = a.y[m]; a.z[h] = a.z[m]; a.d[h] = a.d[m]; a.v[h] = a.v[m];
  a.pkey[h] = a.pkey[m]; a.nnz[h] = a.nnz[m];
}

__global__ void k_state_mark_changed(StateArrays a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a.flags[i] = FLAG_CHANGED;
}

void launch_state_remove(cudaStream_t st, void *staging, int64_t n_old, int64_t n_new, const int64_t *holes,
                         const int64_t *movers, int64_t np) {
  const StateArrays a = state_arrays(staging, n_old);
  if (np > 0) k_state_move<<<blocks_for(np, kThreads), kThreads, 0, st>>>(a, holes, movers, np);
  if (n_new > 0) k_state_mark_changed<<<blocks_for(n_new, kThreads), kThreads, 0, st>>>(a, n_new);
}

}  // namespace bdm
