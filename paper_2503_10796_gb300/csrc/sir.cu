// Epidemiology use case (§4.6.3): one step of the infection (Algorithm 3),
// recovery (Algorithm 4) and random movement (Algorithm 5) behaviours of a
// simulation's agents, on the query grid (box length at least the infection
// radius, so the 27-box stencil holds every person within the radius).
//
// Copy execution context: every agent reads the states and positions at
// the start of the step (states in one buffer, written to another; new
// positions to scratch, committed by a second kernel); an agent's own
// behaviours see its own updates in the order infection, recovery,
// movement.  Random numbers: Philox4x64-10, key {seed, 1}, counter
// {ID, t, draw, 0}; draw 0 gives the infection and recovery uniforms, draw
// 1 the three movement uniforms.  Every FP64 operation is an IEEE
// intrinsic in the order of the definition, so results equal the plain
// definition's bit for bit.
#include "kernels.cuh"
#include "philox.cuh"

namespace bdm {

namespace {

enum : uint8_t { SIR_S = 0, SIR_I = 1, SIR_R = 2 };

// Any other agent infected at the start of the step within the radius:
// (x_j - x_i)^2 summed as (dx dx + dy dy) + dz dz, strictly below r2.
__device__ bool infected_within(const DevCtx &C, const SimConst &sc, const SimState &s, int64_t p,
                                const double4_32a &o, const uint8_t *st_in, double r2, uint32_t stamp) {
  const Cells &Q = C.q;
  int64_t cx, cy, cz;
  unpack_coords(Q.pkey[p], cx, cy, cz);
  for (int dz = -1; dz <= 1; ++dz) {
    const int64_t z = cz + dz;
    if (z < 0 || z >= s.dims[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int64_t y = cy + dy;
      if (y < 0 || y >= s.dims[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int64_t x = cx + dx;
        if (x < 0 || x >= s.dims[0]) continue;
        const unsigned long long e = C.tab.e[sc.table_base + linear_box(s, x, y, z)];
        const uint32_t cnt = ent_live(e, stamp);
        const int64_t j0 = ent_start(e);
        for (int64_t j = j0; j < j0 + cnt; ++j) {
          if (j == p) continue;
          if (st_in[C.a.id[Q.slot[j]]] != SIR_I) continue;
          const double4_32a q = Q.r64[j];
          const double ex = __dsub_rn(q.x, o.x), ey = __dsub_rn(q.y, o.y), ez = __dsub_rn(q.z, o.z);
          if (__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)) < r2) return true;
        }
      }
    }
  }
  return false;
}

__device__ __forceinline__ double wrap_torus(double v, double L) {
  const double r = fmod(v, L);
  return r < 0.0 ? __dadd_rn(L, r) : r;
}

__global__ void k_sir(DevCtx C, int sim, int64_t cell_base, int64_t n, int64_t base, const uint8_t *st_in,
                      uint8_t *st_out, double *nxyz, bdm_sir_params prm, long long t) {
  const int64_t p = cell_base + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cell_base + n) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid) return;
  const Cells &Q = C.q;
  const int64_t slot = Q.slot[p];
  const int64_t id = C.a.id[slot];
  const double4_32a o = Q.r64[p];
  const unsigned long long key[2] = {(unsigned long long)prm.seed, 1ull};
  unsigned long long w[4];
  const unsigned long long c0[4] = {(unsigned long long)id, (unsigned long long)t, 0ull, 0ull};
  philox4x64_10(c0, key, w);
  uint8_t st = st_in[id];
  if (st == SIR_S && unit53(w[0]) < prm.p_infect &&
      infected_within(C, sc, s, p, o, st_in, __dmul_rn(prm.radius, prm.radius), C.g->stamp & kStampMask))
    st = SIR_I;
  if (st == SIR_I && unit53(w[1]) < prm.p_recover) st = SIR_R;
  st_out[id] = st;
  const unsigned long long c1[4] = {(unsigned long long)id, (unsigned long long)t, 1ull, 0ull};
  unsigned long long m[4];
  philox4x64_10(c1, key, m);
  double v[3];
  for (int a = 0; a < 3; ++a) v[a] = __dsub_rn(__dmul_rn(2.0, unit53(m[a])), 1.0);
  const double norm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])), __dmul_rn(v[2], v[2])));
  const double pos[3] = {o.x, o.y, o.z};
  for (int a = 0; a < 3; ++a) {
    double x = pos[a];
    if (norm > 0.0) x = __dadd_rn(x, __dmul_rn(__ddiv_rn(v[a], norm), prm.speed));
    nxyz[3 * (slot - base) + a] = wrap_torus(x, prm.length);
  }
}

// The new positions become the agents' positions; moved agents are marked
// changed for the grid history and static detection.
__global__ void k_sir_commit(DevCtx C, int64_t base, int64_t n, const double *nxyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t slot = base + i;
  const double x = nxyz[3 * i], y = nxyz[3 * i + 1], z = nxyz[3 * i + 2];
  if (x != C.a.x[slot] || y != C.a.y[slot] || z != C.a.z[slot]) {
    C.a.x[slot] = x;
    C.a.y[slot] = y;
    C.a.z[slot] = z;
    C.a.flags[slot] |= FLAG_CHANGED;
  }
}

inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

}  // namespace

void launch_sir_step(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n, int64_t base,
                     const uint8_t *st_in, uint8_t *st_out, double *nxyz, const bdm_sir_params &prm, long long t) {
  if (n <= 0) return;
  k_sir<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, sim, cell_base, n, base, st_in, st_out, nxyz, prm, t);
  k_sir_commit<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, nxyz);
}

}  // namespace bdm
