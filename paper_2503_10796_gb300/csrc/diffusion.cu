// Soma-clustering slice: extracellular diffusion (§4.5.2, Eq 4.3),
// substance secretion (Algorithm 6) and chemotaxis (Algorithm 7).
//
// The diffusion grid holds n0 x n1 x n2 FP64 concentrations, point
// (i, j, k) at i + n0 (j + n1 k); it stands for the box
// [lo + (i, j, k) h, lo + (i + 1, j + 1, k + 1) h).  Outside the grid the
// concentration is zero: substances diffuse out of the space (§4.5.2).
// Every FP64 operation is an IEEE round-to-nearest intrinsic, in the order
// Eq 4.3 prints its terms, so that the results equal those of the plain
// definition bit for bit.
#include "kernels.cuh"

namespace bdm {

namespace {

constexpr int kDiffThreads = 256;

struct DiffCoef {
  double keep, cx, cy, cz;
};

// keep = 1 - mu dt; c_a = (nu dt) / (h_a h_a), on the device so that no
// host compiler contracts them into fused multiply-adds.
__device__ __forceinline__ DiffCoef diff_coef(double nu, double mu, double dt, double hx, double hy, double hz) {
  DiffCoef k;
  k.keep = __dsub_rn(1.0, __dmul_rn(mu, dt));
  const double nd = __dmul_rn(nu, dt);
  k.cx = __ddiv_rn(nd, __dmul_rn(hx, hx));
  k.cy = __ddiv_rn(nd, __dmul_rn(hy, hy));
  k.cz = __ddiv_rn(nd, __dmul_rn(hz, hz));
  return k;
}

// One explicit step of Eq 4.3, a thread per grid point (x fastest, so the
// x neighbours share cache lines and the y and z rows are re-read from L2).
// The FP64 operations of a point (13, the coefficients come from shared
// memory) bound the kernel on this part, not its 16 bytes of HBM traffic.
__global__ void __launch_bounds__(kDiffThreads) k_diffuse(const double *__restrict__ in, double *__restrict__ out,
                                                         int64_t n0, int64_t n1, int64_t n2, double nu, double mu,
                                                         double dt, double hx, double hy, double hz) {
  __shared__ DiffCoef sk;
  if (threadIdx.x == 0) sk = diff_coef(nu, mu, dt, hx, hy, hz);
  __syncthreads();
  const DiffCoef k = sk;
  const int64_t plane = n0 * n1, total = plane * n2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = p % n0, j = (p / n0) % n1, l = p / plane;
    const double c = in[p];
    const double xp = i + 1 < n0 ? in[p + 1] : 0.0, xm = i > 0 ? in[p - 1] : 0.0;
    const double yp = j + 1 < n1 ? in[p + n0] : 0.0, ym = j > 0 ? in[p - n0] : 0.0;
    const double zp = l + 1 < n2 ? in[p + plane] : 0.0, zm = l > 0 ? in[p - plane] : 0.0;
    const double c2 = __dmul_rn(2.0, c);
    const double lx = __dadd_rn(__dsub_rn(xp, c2), xm);
    const double ly = __dadd_rn(__dsub_rn(yp, c2), ym);
    const double lz = __dadd_rn(__dsub_rn(zp, c2), zm);
    out[p] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(c, k.keep), __dmul_rn(k.cx, lx)), __dmul_rn(k.cy, ly)),
                       __dmul_rn(k.cz, lz));
  }
}

// Box of a position in the diffusion grid: floor((x - lo) / h) per axis in
// IEEE FP64; false outside the grid.
__device__ __forceinline__ bool diff_box(const DiffGrid &g, double x, double y, double z, int64_t &b0, int64_t &b1,
                                         int64_t &b2) {
  const double q0 = floor(__ddiv_rn(__dsub_rn(x, g.lo[0]), g.h[0]));
  const double q1 = floor(__ddiv_rn(__dsub_rn(y, g.lo[1]), g.h[1]));
  const double q2 = floor(__ddiv_rn(__dsub_rn(z, g.lo[2]), g.h[2]));
  if (!(q0 >= 0.0) || !(q0 < (double)g.n[0]) || !(q1 >= 0.0) || !(q1 < (double)g.n[1]) || !(q2 >= 0.0) ||
      !(q2 < (double)g.n[2]))
    return false;
  b0 = (int64_t)q0;
  b1 = (int64_t)q1;
  b2 = (int64_t)q2;
  return true;
}

__device__ __forceinline__ double diff_at(const double *u, const DiffGrid &g, int64_t i, int64_t j, int64_t k) {
  if (i < 0 || j < 0 || k < 0 || i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return 0.0;
  return u[i + g.n[0] * (j + g.n[1] * k)];
}

// Algorithm 6: every agent of the simulation inside the grid adds
// `quantity` to its box.  The additions to one box commute exactly (equal
// addends), so the result does not depend on the order of the atomics.
// sim >= 0: a step of bdm_step, which takes the simulation's agent count
// from the device (n is then the simulation's capacity) and serves the
// agents of one kind (kind < 0: every agent).
__device__ __forceinline__ bool of_kind(const DevCtx &C, int64_t base, int64_t slot, int kind) {
  if (kind < 0) return true;
  const int k = C.kind ? (int)C.kind[base + C.a.id[slot]] : 0;
  return k == kind;
}

__global__ void k_secrete(DevCtx C, int64_t base, int64_t n, int sim, int kind, DiffGrid g, double *u,
                          double quantity) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sim >= 0 && i >= C.ss[sim].n) return;
  if (i >= n) return;
  const int64_t slot = base + i;
  if (!of_kind(C, base, slot, kind)) return;
  int64_t b0, b1, b2;
  if (!diff_box(g, C.a.x[slot], C.a.y[slot], C.a.z[slot], b0, b1, b2)) return;
  atomicAdd(&u[b0 + g.n[0] * (b1 + g.n[1] * b2)], quantity);
}

// Algorithm 7: every agent inside the grid moves by weight times the
// normalized central-difference gradient of its box; the grid is only read.
// Agents that move are marked changed (their box must be recomputed and
// they disturb static neighbours).
__global__ void k_chemotaxis(DevCtx C, int64_t base, int64_t n, int sim, int kind, DiffGrid g, const double *u,
                             double weight) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sim >= 0 && i >= C.ss[sim].n) return;
  if (i >= n) return;
  const int64_t slot = base + i;
  if (!of_kind(C, base, slot, kind)) return;
  const double x = C.a.x[slot], y = C.a.y[slot], z = C.a.z[slot];
  int64_t b0, b1, b2;
  if (!diff_box(g, x, y, z, b0, b1, b2)) return;
  double gx = __ddiv_rn(__dsub_rn(diff_at(u, g, b0 + 1, b1, b2), diff_at(u, g, b0 - 1, b1, b2)), __dmul_rn(2.0, g.h[0]));
  double gy = __ddiv_rn(__dsub_rn(diff_at(u, g, b0, b1 + 1, b2), diff_at(u, g, b0, b1 - 1, b2)), __dmul_rn(2.0, g.h[1]));
  double gz = __ddiv_rn(__dsub_rn(diff_at(u, g, b0, b1, b2 + 1), diff_at(u, g, b0, b1, b2 - 1)), __dmul_rn(2.0, g.h[2]));
  const double norm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz)));
  if (!(norm > 0.0)) return;  // no gradient, no move
  gx = __ddiv_rn(gx, norm);
  gy = __ddiv_rn(gy, norm);
  gz = __ddiv_rn(gz, norm);
  const double nx = __dadd_rn(x, __dmul_rn(gx, weight));
  const double ny = __dadd_rn(y, __dmul_rn(gy, weight));
  const double nz = __dadd_rn(z, __dmul_rn(gz, weight));
  if (nx != x || ny != y || nz != z) {
    C.a.x[slot] = nx;
    C.a.y[slot] = ny;
    C.a.z[slot] = nz;
    C.a.flags[slot] |= FLAG_CHANGED;
    C.g->regrid = 1u;  // moved outside the displacement: a kept grid no longer fits
  }
}

inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

}  // namespace

void launch_diffuse_step(cudaStream_t st, const double *in, double *out, const DiffGrid &g, double nu, double mu,
                         double dt) {
  const int64_t total = g.n[0] * g.n[1] * g.n[2];
  if (total <= 0) return;
  // a grid-stride loop over at most 152 SMs x 8 blocks
  const int64_t want = (total + kDiffThreads - 1) / kDiffThreads;
  const unsigned int nb = (unsigned int)(want < 152 * 8 ? want : 152 * 8);
  k_diffuse<<<nb, kDiffThreads, 0, st>>>(in, out, g.n[0], g.n[1], g.n[2], nu, mu, dt, g.h[0], g.h[1], g.h[2]);
}

void launch_secrete(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const DiffGrid &g, double *u,
                    double quantity) {
  if (n <= 0) return;
  k_secrete<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, -1, -1, g, u, quantity);
}

void launch_secrete_step(const DevCtx &C, cudaStream_t st, int sim, int kind, int64_t base, int64_t cap,
                         const DiffGrid &g, double *u, double quantity) {
  if (cap <= 0) return;
  k_secrete<<<blocks_for(cap, kThreads), kThreads, 0, st>>>(C, base, cap, sim, kind, g, u, quantity);
}

void launch_chemotaxis_step(const DevCtx &C, cudaStream_t st, int sim, int kind, int64_t base, int64_t cap,
                            const DiffGrid &g, const double *u, double weight) {
  if (cap <= 0) return;
  k_chemotaxis<<<blocks_for(cap, kThreads), kThreads, 0, st>>>(C, base, cap, sim, kind, g, u, weight);
}

// Kinds of the agents that removal renumbers: hole[k] takes mover[k]'s.
__global__ void k_kinds_move(uint8_t *kind, int64_t base, const int64_t *hole, const int64_t *mover, int64_t np) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < np) kind[base + hole[k]] = kind[base + mover[k]];
}

void launch_kinds_move(const DevCtx &C, cudaStream_t st, int64_t base, const int64_t *hole, const int64_t *mover,
                       int64_t np) {
  if (!C.kind || np <= 0) return;
  k_kinds_move<<<blocks_for(np, kThreads), kThreads, 0, st>>>(C.kind, base, hole, mover, np);
}

void launch_chemotaxis(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const DiffGrid &g, const double *u,
                       double weight) {
  if (n <= 0) return;
  k_chemotaxis<<<blocks_for(n, kThreads), kThreads, 0, st>>>(C, base, n, -1, -1, g, u, weight);
}

}  // namespace bdm
