// S7 growth and division (Table D.1 GrowthDivision, Cell::Divide), in the
// copy execution context: decisions use the volume at the start of the
// iteration, the daughters appear for the next iteration (§5.2).
//
//   V < V_div : V += g dt, d = cbrt(6 V / pi) (correctly rounded);
//   V >= V_div: divide while the simulation is below its capacity, in
//               ascending parent ID (new IDs n, n+1, ...).  Both daughters
//               get V / 2 and d' = cbrt(6 (V/2) / pi); the mother keeps its
//               ID and moves to x - (d'/4) u, the new agent is placed at
//               x + (d'/4) u, u a uniform direction from Philox4x64-10
//               (Salmon et al., SC 2011) with counter {ID, iteration,
//               attempt, 0} and key {seed, 0}: the counter-based generator
//               that §7.1.4 proposes for reproducible runs.
#include "kernels.cuh"
#include "philox.cuh"

namespace bdm {

// ---------------------------------------------------------------------------
// Correctly rounded cube root: CUDA's cbrt gives a start within an ulp or
// so; the result is moved to the double nearest to the exact cube root by
// comparing the cubes of midpoints between adjacent doubles with x in exact
// 192-bit integer arithmetic.
// ---------------------------------------------------------------------------
struct U192 { unsigned long long w[3]; };

__device__ __forceinline__ U192 u192_mul(U192 a, unsigned long long b) {
  U192 r;
  unsigned long long carry = 0;
  for (int k = 0; k < 3; ++k) {
    unsigned long long lo = a.w[k] * b;
    unsigned long long hi = __umul64hi(a.w[k], b);
    unsigned long long s = lo + carry;
    hi += (s < lo) ? 1ull : 0ull;
    r.w[k] = s;
    carry = hi;
  }
  return r;
}

__device__ __forceinline__ int u192_bits(U192 a) {
  for (int k = 2; k >= 0; --k)
    if (a.w[k]) return 64 * k + 64 - __clzll((long long)a.w[k]);
  return 0;
}

__device__ __forceinline__ U192 u192_shl(U192 a, int s) {
  U192 r = {{0, 0, 0}};
  int q = s / 64, m = s % 64;
  for (int k = 2; k >= 0; --k) {
    int src = k - q;
    if (src < 0) continue;
    unsigned long long v = a.w[src] << m;
    if (m && src - 1 >= 0) v |= a.w[src - 1] >> (64 - m);
    r.w[k] = v;
  }
  return r;
}

__device__ __forceinline__ int u192_cmp(U192 a, U192 b) {
  for (int k = 2; k >= 0; --k)
    if (a.w[k] != b.w[k]) return a.w[k] < b.w[k] ? -1 : 1;
  return 0;
}

// Sign of M^3 2^(3e) - X 2^ex.
__device__ int cube_cmp(unsigned long long M, int e, unsigned long long X, int ex) {
  U192 m = {{M, 0, 0}};
  U192 c = u192_mul(u192_mul(m, M), M);
  U192 x = {{X, 0, 0}};
  int s = 3 * e - ex;
  if (s >= 0) {
    if (u192_bits(c) + s > 190) return 1;
    c = u192_shl(c, s);
  } else {
    if (u192_bits(x) - s > 190) return -1;
    x = u192_shl(x, -s);
  }
  return u192_cmp(c, x);
}

__device__ __forceinline__ void split_dbl(double v, unsigned long long &M, int &e) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  int E = (int)((b >> 52) & 0x7FF);
  unsigned long long f = b & ((1ull << 52) - 1);
  if (E == 0) { M = f; e = -1074; }
  else { M = f | (1ull << 52); e = E - 1075; }
}

__device__ __forceinline__ void mid_of(double a, double b, unsigned long long &M, int &e) {
  unsigned long long Ma, Mb;
  int ea, eb;
  split_dbl(a, Ma, ea);
  split_dbl(b, Mb, eb);
  int m = ea < eb ? ea : eb;
  M = (Ma << (ea - m)) + (Mb << (eb - m));
  e = m - 1;
}

__device__ double cbrt_rn(double x) {
  if (!(x > 0.0) || isinf(x)) return cbrt(x);
  unsigned long long X;
  int ex;
  split_dbl(x, X, ex);
  double y = cbrt(x);
  for (int it = 0; it < 16; ++it) {
    unsigned long long M;
    int e;
    double up = nextafter(y, __longlong_as_double(0x7FF0000000000000ll));
    mid_of(y, up, M, e);
    if (cube_cmp(M, e, X, ex) < 0) { y = up; continue; }
    double dn = nextafter(y, 0.0);
    if (dn > 0.0) {
      mid_of(dn, y, M, e);
      if (cube_cmp(M, e, X, ex) > 0) { y = dn; continue; }
    }
    break;
  }
  return y;
}

__device__ __forceinline__ double diameter_of_volume(double V) {
  return cbrt_rn(__ddiv_rn(__dmul_rn(6.0, V), 3.141592653589793));
}

__device__ void division_axis(unsigned long long seed, long long id, long long t, double u[3]) {
  for (unsigned long long k = 0; k < 1000000ull; ++k) {
    unsigned long long ctr[4] = {(unsigned long long)id, (unsigned long long)t, k, 0ull};
    unsigned long long key[2] = {seed, 0ull}, w[4];
    philox4x64_10(ctr, key, w);
    double p[3];
    for (int a = 0; a < 3; ++a)
      p[a] = __dsub_rn(__dmul_rn(2.0, __dmul_rn((double)(w[a] >> 11), 0x1.0p-53)), 1.0);
    double s = __dadd_rn(__dadd_rn(__dmul_rn(p[0], p[0]), __dmul_rn(p[1], p[1])), __dmul_rn(p[2], p[2]));
    if (s > 1e-6 && s <= 1.0) {
      double r = __dsqrt_rn(s);
      u[0] = __ddiv_rn(p[0], r);
      u[1] = __ddiv_rn(p[1], r);
      u[2] = __ddiv_rn(p[2], r);
      return;
    }
  }
  u[0] = 1.0; u[1] = 0.0; u[2] = 0.0;
}

// ---------------------------------------------------------------------------
// Kernels.  `flag` is indexed by base_s + ID (the region of simulation s in
// ID order); `rank` receives its exclusive prefix sum over all regions.
// ---------------------------------------------------------------------------
struct GrowBufs {
  uint32_t *flag;    // total_slots + 1
  uint32_t *rank;    // total_slots + 1
  uint32_t *part;    // 2048
};

static size_t al256(size_t b) { return (b + 255) / 256 * 256; }

static GrowBufs carve_grow(void *scratch, int64_t M) {
  GrowBufs g;
  char *p = (char *)scratch;
  g.flag = (uint32_t *)p;
  p += al256(4 * (size_t)(M + 1));
  g.rank = (uint32_t *)p;
  p += al256(4 * (size_t)(M + 1));
  g.part = (uint32_t *)p;
  return g;
}

size_t growth_scratch_bytes(int64_t total_slots, int n_sims) {
  (void)n_sims;
  size_t M = (size_t)(total_slots > 0 ? total_slots : 1);
  return 2 * al256(4 * (M + 1)) + al256(4 * 2048);
}

// Decide on the volume at the start of the iteration: dividers are marked
// (in ID space), the others grow.
__global__ void k_grow_mark(DevCtx C, GrowBufs B) {
  int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= C.total_slots) return;
  int sim = C.a.sim[slot];
  if (sim < 0) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!sc.grows || slot - sc.base >= s.n || (C.a.flags[slot] & FLAG_GHOST)) return;
  double V = C.a.v[slot];
  if (V < sc.divide_volume) {
    V = __dadd_rn(V, __dmul_rn(sc.growth_rate, sc.dt));
    C.a.v[slot] = V;
    C.a.d[slot] = diameter_of_volume(V);
    C.a.flags[slot] |= FLAG_CHANGED;
  } else {
    B.flag[sc.base + C.a.id[slot]] = 1u;
  }
}

__global__ void __launch_bounds__(1024) k_gscan_up(const uint32_t *v, int64_t n, int64_t chunk, uint32_t *part) {
  __shared__ uint32_t sh[32];
  int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  uint32_t s = 0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) s += v[i];
  s = __reduce_add_sync(0xffffffffu, s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_gscan_top(uint32_t *part, int G) {
  if (threadIdx.x != 0) return;
  uint32_t run = 0;
  for (int g = 0; g < G; ++g) {
    uint32_t v = part[g];
    part[g] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(1024) k_gscan_down(const uint32_t *v, uint32_t *out, int64_t n, int64_t chunk,
                                                     const uint32_t *part) {
  __shared__ uint32_t sh[33];
  int64_t b = (int64_t)blockIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
  uint32_t base = part[blockIdx.x];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t0 = b; t0 < e; t0 += blockDim.x) {
    int64_t i = t0 + threadIdx.x;
    uint32_t x = i < e ? v[i] : 0u, inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        uint32_t t = sh[w];
        sh[w] = run;
        run += t;
      }
      sh[32] = run;
    }
    __syncthreads();
    if (i < e) out[i] = base + sh[warp] + inc - x;
    base += sh[32];
    __syncthreads();
  }
}

// Divide: the r-th divider (ascending ID) of a simulation with n0 agents
// creates agent ID n0 + r in slot base + n0 + r, while n0 + r < capacity.
__global__ void k_divide(DevCtx C, GrowBufs B) {
  int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= C.total_slots) return;
  int sim = C.a.sim[slot];
  if (sim < 0) return;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  int64_t n0 = s.n;
  if (!sc.grows || slot - sc.base >= n0) return;
  int64_t id = C.a.id[slot];
  if (!B.flag[sc.base + id]) return;
  int64_t r = (int64_t)B.rank[sc.base + id] - (int64_t)B.rank[sc.base];
  if (n0 + r >= sc.cap) return;  // capacity reached: no division
  double vh = __dmul_rn(0.5, C.a.v[slot]);
  double dh = diameter_of_volume(vh);
  double u[3];
  division_axis(sc.seed, id, s.it, u);
  double off = __dmul_rn(0.25, dh);
  double px = C.a.x[slot], py = C.a.y[slot], pz = C.a.z[slot];
  int64_t j = sc.base + n0 + r;
  // daughters under the space boundary condition (§4.4.11)
  C.a.x[j] = bound_apply(sc, __dadd_rn(px, __dmul_rn(off, u[0])));
  C.a.y[j] = bound_apply(sc, __dadd_rn(py, __dmul_rn(off, u[1])));
  C.a.z[j] = bound_apply(sc, __dadd_rn(pz, __dmul_rn(off, u[2])));
  C.a.x[slot] = bound_apply(sc, __dsub_rn(px, __dmul_rn(off, u[0])));
  C.a.y[slot] = bound_apply(sc, __dsub_rn(py, __dmul_rn(off, u[1])));
  C.a.z[slot] = bound_apply(sc, __dsub_rn(pz, __dmul_rn(off, u[2])));
  C.a.v[slot] = vh;
  C.a.v[j] = vh;
  C.a.d[slot] = dh;
  C.a.d[j] = dh;
  C.a.flags[slot] |= FLAG_CHANGED;
  C.a.flags[j] = FLAG_CHANGED;
  C.a.nnz[j] = 0;
  C.a.id[j] = (int32_t)(n0 + r);
  if (C.kind) C.kind[sc.base + n0 + r] = C.kind[sc.base + id];  // a daughter of the mother's kind
  C.a.pkey[j] = C.a.pkey[slot];
  C.a.rank[j] = 0;
}

__global__ void k_division_counts(DevCtx C, GrowBufs B) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= C.n_sims) return;
  int s = C.order[k];
  if (s < 0) return;
  const SimConst &sc = C.sc[s];
  SimState &st = C.ss[s];
  if (!sc.grows) return;
  int64_t n0 = st.n;
  int64_t dividers = (int64_t)B.rank[sc.base + n0] - (int64_t)B.rank[sc.base];
  int64_t room = sc.cap - n0;
  int64_t made = dividers < room ? dividers : room;
  if (dividers > room) set_err(C.g, ERR_CAPACITY);
  st.n = n0 + made;
}

void launch_growth(const DevCtx &C, cudaStream_t st, void *scratch, size_t scratch_bytes) {
  (void)scratch_bytes;
  int64_t M = C.total_slots;
  if (M <= 0) return;
  GrowBufs B = carve_grow(scratch, M);
  unsigned int nb = (unsigned int)((M + 1 + kThreads - 1) / kThreads);
  cudaMemsetAsync(B.flag, 0, sizeof(uint32_t) * (size_t)(M + 1), st);
  k_grow_mark<<<nb, kThreads, 0, st>>>(C, B);
  int64_t n = M + 1;
  int64_t G = (n + 4095) / 4096;
  if (G > 1024) G = 1024;
  if (G < 1) G = 1;
  int64_t chunk = (n + G - 1) / G;
  chunk = (chunk + 1023) / 1024 * 1024;
  G = (n + chunk - 1) / chunk;
  if (G < 1) G = 1;
  k_gscan_up<<<(unsigned int)G, 1024, 0, st>>>(B.flag, n, chunk, B.part);
  k_gscan_top<<<1, 32, 0, st>>>(B.part, (int)G);
  k_gscan_down<<<(unsigned int)G, 1024, 0, st>>>(B.flag, B.rank, n, chunk, B.part);
  k_divide<<<nb, kThreads, 0, st>>>(C, B);
  k_division_counts<<<(C.n_sims + 127) / 128, 128, 0, st>>>(C, B);
}

}  // namespace bdm
