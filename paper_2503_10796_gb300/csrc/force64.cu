// S4 force of the FP64 path (Eq 4.1 / Eq 4.2, §4.5.1), summed in ascending
// partner ID.
//
// Every pair is evaluated by the definition, operation by operation, with
// IEEE FP64 intrinsics (pair64), and an agent's pair forces are added in
// ascending caller ID of the partner, starting from zero: the order of the
// sum over neighbours that the definition of one iteration uses.  Since the
// displacement, growth and division kernels evaluate their definitions the
// same way, an FP64-path trajectory is the same bit for bit whatever the
// storage order, the grid's cell order or the launch configuration.
//
// k_force64r: a thread per stencil row, 9 per agent, 32 agents per block
// (the FP64 square roots and divisions run at a small fraction of the FP32
// rate on this part, and nine times the threads hide their latency).  A row
// walks with the FP32 filter of the FP32 path (box-relative leading parts,
// a margin above their error, so every pair that overlaps in FP64 passes)
// and queues up to kRowCap passing candidates; the warp evaluates the queued
// pairs one per lane and round (a row with more candidates evaluates them in
// place).  Each evaluated pair appends {partner ID, force} to its agent's
// list in shared memory; the agent's first thread then orders the list by
// partner ID and adds it up.  An agent with more than kSortCap candidates
// passing the filter evaluates nothing here and is left to k_force64o.
//
// k_force64o: a warp per such agent: the overlapping pairs of the whole
// stencil (found through the same FP32 filter) in shared memory, sorted by
// partner ID, added in that order (and, beyond kOvfCap partners, a
// selection of the next partner ID at a time).
#include "pair.cuh"

namespace bdm {
namespace {

constexpr int kRowAgents = 32;
constexpr int kRowThreads = kRowAgents * 9;
constexpr int kRowCap = 4;
constexpr int kSortCap = 24;

struct Contrib {
  double gx, gy, gz;
  uint32_t id;      // partner's caller ID
  uint32_t flags;   // bit 0: non-zero force; bit 1: the pair has a direction (distance > 0)
};

__device__ __forceinline__ uint32_t partner_id(const DevCtx &C, int64_t j) { return (uint32_t)C.a.id[C.c.slot[j]]; }

__global__ void __launch_bounds__(kRowThreads, 3) k_force64r(DevCtx C) {
  __shared__ uint32_t rq[kRowCap][kRowThreads];
  __shared__ uint8_t skip[kRowAgents];
  __shared__ uint32_t ncon[kRowAgents];
  __shared__ uint32_t nfil[kRowAgents];  // candidates that pass the FP32 filter, per agent
  __shared__ Contrib con[kRowAgents][kSortCap];
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  const int a = threadIdx.x / 9, r = threadIdx.x % 9;
  const int64_t p = (int64_t)blockIdx.x * kRowAgents + a;
  bool active = p < C.g->n_cells;
  const int sim = active ? C.c.sim[p] : 0;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  active = active && s.valid && sc.precision == BDM_PREC_FP64;
  int64_t cx = 0, cy = 0, cz = 0;
  if (active) unpack_coords(C.c.pkey[p], cx, cy, cz);
  const uint32_t stamp = C.g->stamp & kStampMask;
  if (r == 0) {
    bool st = false;
    if (active) {
      st = is_static_cell(C, sc, s, p, cx, cy, cz, stamp);
      C.c.stat[p] = st ? 1 : 0;
    }
    skip[a] = (!active || st) ? 1 : 0;
    ncon[a] = 0u;
    nfil[a] = 0u;
  }
  __syncthreads();
  auto append = [&](int agent, int64_t j, double gx, double gy, double gz, bool nz, bool dir) {
    const uint32_t k = atomicAdd(&ncon[agent], 1u);
    if (k < (uint32_t)kSortCap) {
      Contrib &c = con[agent][k];
      c.gx = gx; c.gy = gy; c.gz = gz;
      c.id = partner_id(C, j);
      c.flags = (nz ? 1u : 0u) | (dir ? 2u : 0u);
    }
  };
  uint32_t n = 0;
  const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
  const int dz = r / 3 - 1, dy = r % 3 - 1;
  const bool walk = !skip[a] && dz >= t.zlo && dz <= t.zhi && dy >= t.ylo && dy <= t.yhi;
  const float Lh = s.Lh, marg = s.marg;
  // the FP32 filter: box-relative leading parts with a margin above their
  // error, so every pair that overlaps in FP64 passes
  auto passes = [&](const float4 &o0, int64_t j, float sx, float sy, float sz) {
    const float4 q = C.c.r0[j];
    const float ddx = __fsub_rn(sx, q.x), ddy = __fsub_rn(sy, q.y), ddz = __fsub_rn(sz, q.z);
    const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
    const float Rm = __fadd_rn(__fadd_rn(o0.w, q.w), marg);
    return s2 < __fmul_rn(Rm, Rm);
  };
  if (walk) {
    const float4 o0 = C.c.r0[p];
    const float sy = __fsub_rn(o0.y, __fmul_rn((float)dy, Lh)), sz = __fsub_rn(o0.z, __fmul_rn((float)dz, Lh));
    for (int dx = t.xlo; dx <= t.xhi; ++dx) {
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      const uint32_t cnt = ent_live(e, stamp);
      const int64_t j0 = ent_start(e);
      const float sx = __fsub_rn(o0.x, __fmul_rn((float)dx, Lh));
      for (uint32_t m = 0; m < cnt; ++m) {
        const int64_t j = j0 + m;
        if (j == p || !passes(o0, j, sx, sy, sz)) continue;
        if (n < (uint32_t)kRowCap) rq[n][threadIdx.x] = (uint32_t)j;
        ++n;
      }
    }
    if (n) atomicAdd(&nfil[a], n);
  }
  __syncthreads();
  // an agent with more candidates than its list holds goes to k_force64o
  // untouched; the others evaluate their rows
  const bool crowded = nfil[a] > (uint32_t)kSortCap;
  uint32_t mine = crowded ? 0u : n;
  if (!crowded && n > (uint32_t)kRowCap) {
    // crowded row: evaluate it in place (the records are loaded again, so
    // that nothing of the walk stays live across the barrier)
    mine = 0;
    const double4_32a o = C.c.r64[p];
    const float4 o0 = C.c.r0[p];
    const float sy = __fsub_rn(o0.y, __fmul_rn((float)dy, Lh)), sz = __fsub_rn(o0.z, __fmul_rn((float)dz, Lh));
    for (int dx = t.xlo; dx <= t.xhi; ++dx) {
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      const uint32_t cnt = ent_live(e, stamp);
      const int64_t j0 = ent_start(e);
      const float sx = __fsub_rn(o0.x, __fmul_rn((float)dx, Lh));
      for (uint32_t m = 0; m < cnt; ++m) {
        const int64_t j = j0 + m;
        if (j == p || !passes(o0, j, sx, sy, sz)) continue;
        double gx, gy, gz;
        bool nz, dir;
        if (pair64(sc, o, C.c.r64[j], sc.k, sc.gamma, gx, gy, gz, nz, dir)) append(a, j, gx, gy, gz, nz, dir);
      }
    }
  }
  // warp-wide evaluation of the queues laid end to end
  {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    uint32_t incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += y;
    }
    const uint32_t excl = incl - mine;
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t kk = base + (uint32_t)lane;
      int ow = 0;  // owner: the first lane whose inclusive prefix exceeds kk
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const uint32_t v = __shfl_sync(FULL, incl, ow + step - 1);
        if (v <= kk) ow += step;
      }
      const uint32_t ex = __shfl_sync(FULL, excl, ow);
      if (kk < total) {
        const int to = wbase + ow;  // the owner's thread in the block
        const int agent = to / 9;
        const int64_t po = (int64_t)blockIdx.x * kRowAgents + agent;
        const SimConst &so = C.sc[C.c.sim[po]];
        const int64_t j = (int64_t)rq[kk - ex][to];
        double gx, gy, gz;
        bool nz, dir;
        if (pair64(so, C.c.r64[po], C.c.r64[j], so.k, so.gamma, gx, gy, gz, nz, dir)) append(agent, j, gx, gy, gz, nz, dir);
      }
    }
  }
  __syncthreads();
  if (r == 0 && !skip[a]) {
    const uint32_t cnt = ncon[a];
    if (crowded) {
      C.ovf[atomicAdd(&C.g->n_ovf, 1u)] = (int32_t)p;
      return;
    }
    // the list in ascending partner ID (insertion sort of indices)
    uint8_t ord[kSortCap];
    for (uint32_t i = 0; i < cnt; ++i) {
      const uint32_t id = con[a][i].id;
      uint32_t k = i;
      while (k > 0 && con[a][ord[k - 1]].id > id) {
        ord[k] = ord[k - 1];
        --k;
      }
      ord[k] = (uint8_t)i;
    }
    double fx = 0.0, fy = 0.0, fz = 0.0;
    uint32_t nz = 0;
    for (uint32_t i = 0; i < cnt; ++i) {
      const Contrib &c = con[a][ord[i]];
      nz += c.flags & 1u;
      if (c.flags & 2u) {
        fx = __dadd_rn(fx, c.gx);
        fy = __dadd_rn(fy, c.gy);
        fz = __dadd_rn(fz, c.gz);
      }
    }
    C.c.f64[p] = make_double4_32a(fx, fy, fz, (double)cnt);  // w: overlapping pairs
    C.c.nnz[p] = (uint8_t)(nz > 255u ? 255u : nz);
  }
}

// One warp per overflow agent (grid-stride over the list the row kernel
// wrote; the grid is fixed, so the launch can be captured).  The warp tests
// the agent's candidates 32 at a time with the FP32 filter and compacts
// those that pass, evaluates them 32 at a time and keeps the overlapping
// pairs in shared memory, sorts them by partner ID (bitonic sort of packed
// {ID, index} keys) and adds them in that order.  More than kOvfCand
// passing candidates or kOvfCap partners (a pathological crowd) take the
// selection loop below instead.
constexpr int kOvfWarps = 4;
constexpr int kOvfCap = 256;  // pairs sorted in shared memory (a power of two)

constexpr int kOvfCand = 512;  // candidates passing the filter, evaluated 32 at a time

struct OvfShared {
  unsigned long long key[kOvfCap];  // partner ID << 32 | index of the contribution
  double gx[kOvfCap], gy[kOvfCap], gz[kOvfCap];
  uint32_t flags[kOvfCap];
  uint32_t cand[kOvfCand];  // cells that passed the FP32 filter
};

// The agent's view of its stencil for the FP32 filter (box-relative
// leading parts; the margin exceeds their error).
struct OvfAgent {
  const SimConst *sc;
  Stencil t;
  double4_32a o;
  float4 o0;
  float Lh, marg;
  int64_t p;
  __device__ bool passes(const DevCtx &C, int64_t j, int dx, int dy, int dz) const {
    const float4 q = C.c.r0[j];
    const float sx = __fsub_rn(o0.x, __fmul_rn((float)dx, Lh));
    const float sy = __fsub_rn(o0.y, __fmul_rn((float)dy, Lh));
    const float sz = __fsub_rn(o0.z, __fmul_rn((float)dz, Lh));
    const float ddx = __fsub_rn(sx, q.x), ddy = __fsub_rn(sy, q.y), ddz = __fsub_rn(sz, q.z);
    const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
    const float Rm = __fadd_rn(__fadd_rn(o0.w, q.w), marg);
    return s2 < __fmul_rn(Rm, Rm);
  }
};

__device__ void ovf_selection(const DevCtx &C, const OvfAgent &A, uint32_t stamp, int lane, double &fx, double &fy,
                              double &fz, uint32_t &nnz, uint32_t &ovl) {
  const unsigned FULL = 0xffffffffu;
  const Stencil &t = A.t;
  const int nx = t.xhi - t.xlo + 1, ny = t.yhi - t.ylo + 1, nzb = t.zhi - t.zlo + 1;
  const int nbox = nx * ny * nzb;
  int64_t last = -1;  // partner ID added last
  for (;;) {
    // the overlapping partner with the smallest ID above `last`
    uint32_t best = 0xFFFFFFFFu;
    int64_t bj = -1;
    for (int b = 0; b < nbox; ++b) {
      const int dx = t.xlo + b % nx, dy = t.ylo + (b / nx) % ny, dz = t.zlo + b / (nx * ny);
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      const uint32_t cnt = ent_live(e, stamp);
      const int64_t j0 = ent_start(e);
      for (uint32_t m = (uint32_t)lane; m < cnt; m += 32u) {
        const int64_t j = j0 + m;
        if (j == A.p) continue;
        const uint32_t id = partner_id(C, j);
        if ((int64_t)id <= last || id >= best || !A.passes(C, j, dx, dy, dz)) continue;
        double gx, gy, gz;
        bool nz, dir;
        if (pair64(*A.sc, A.o, C.c.r64[j], A.sc->k, A.sc->gamma, gx, gy, gz, nz, dir)) {
          best = id;
          bj = j;
        }
      }
    }
    const uint32_t wbest = __reduce_min_sync(FULL, best);
    if (wbest == 0xFFFFFFFFu) break;
    const unsigned who = __ballot_sync(FULL, best == wbest && bj >= 0);
    const int src = __ffs(who) - 1;
    const int64_t jb = __shfl_sync(FULL, bj, src);
    if (lane == 0) {
      double gx, gy, gz;
      bool nz, dir;
      pair64(*A.sc, A.o, C.c.r64[jb], A.sc->k, A.sc->gamma, gx, gy, gz, nz, dir);
      ++ovl;
      nnz += nz ? 1u : 0u;
      if (dir) {
        fx = __dadd_rn(fx, gx);
        fy = __dadd_rn(fy, gy);
        fz = __dadd_rn(fz, gz);
      }
    }
    last = (int64_t)wbest;
  }
}

__global__ void __launch_bounds__(32 * kOvfWarps) k_force64o(DevCtx C) {
  __shared__ OvfShared shw[kOvfWarps];
  if (C.g->err & ERR_TABLE) return;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  OvfShared &sh = shw[wid];
  const uint32_t nov = C.g->n_ovf;
  const uint32_t stamp = C.g->stamp & kStampMask;
  for (uint32_t w = blockIdx.x * kOvfWarps + wid; w < nov; w += gridDim.x * kOvfWarps) {
    OvfAgent A;
    A.p = C.ovf[w];
    const int sim = C.c.sim[A.p];
    A.sc = &C.sc[sim];
    const SimState &s = C.ss[sim];
    int64_t cx, cy, cz;
    unpack_coords(C.c.pkey[A.p], cx, cy, cz);
    A.t = make_stencil(C, *A.sc, s, cx, cy, cz);
    A.o = C.c.r64[A.p];
    A.o0 = C.c.r0[A.p];
    A.Lh = s.Lh;
    A.marg = s.marg;
    const Stencil &t = A.t;
    const int nx = t.xhi - t.xlo + 1, ny = t.yhi - t.ylo + 1, nzb = t.zhi - t.zlo + 1;
    const int nbox = nx * ny * nzb;
    // the candidates of the stencil that pass the FP32 filter, compacted
    // (FP64 instructions occupy the pipe for all 32 lanes, so the
    // definition is evaluated only on full rounds of passing candidates)
    uint32_t nc = 0;  // passing candidates (warp-uniform)
    for (int b = 0; b < nbox; ++b) {
      const int dx = t.xlo + b % nx, dy = t.ylo + (b / nx) % ny, dz = t.zlo + b / (nx * ny);
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      const uint32_t cnt = ent_live(e, stamp);
      const int64_t j0 = ent_start(e);
      for (uint32_t m0 = 0; m0 < cnt; m0 += 32u) {
        const uint32_t m = m0 + (uint32_t)lane;
        const int64_t j = j0 + m;
        const bool pass = m < cnt && j != A.p && A.passes(C, j, dx, dy, dz);
        const unsigned B = __ballot_sync(FULL, pass);
        const uint32_t k = nc + (uint32_t)__popc(B & ((1u << lane) - 1u));
        if (pass && k < (uint32_t)kOvfCand) sh.cand[k] = (uint32_t)j;
        nc += (uint32_t)__popc(B);
      }
    }
    __syncwarp();
    // every overlapping pair among them, 32 at a time
    uint32_t n = 0;  // overlapping pairs found (warp-uniform)
    if (nc <= (uint32_t)kOvfCand) {
      for (uint32_t k0 = 0; k0 < nc; k0 += 32u) {
        const uint32_t kk = k0 + (uint32_t)lane;
        const int64_t j = kk < nc ? (int64_t)sh.cand[kk] : A.p;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        bool nz = false, dir = false, hit = false;
        if (kk < nc) hit = pair64(*A.sc, A.o, C.c.r64[j], A.sc->k, A.sc->gamma, gx, gy, gz, nz, dir);
        const unsigned B = __ballot_sync(FULL, hit);
        const uint32_t k = n + (uint32_t)__popc(B & ((1u << lane) - 1u));
        if (hit && k < (uint32_t)kOvfCap) {
          sh.key[k] = ((unsigned long long)partner_id(C, j) << 32) | k;
          sh.gx[k] = gx; sh.gy[k] = gy; sh.gz[k] = gz;
          sh.flags[k] = (nz ? 1u : 0u) | (dir ? 2u : 0u);
        }
        n += (uint32_t)__popc(B);
      }
    } else {
      n = (uint32_t)kOvfCap + 1u;  // too many candidates: the selection loop
    }
    double fx = 0.0, fy = 0.0, fz = 0.0;
    uint32_t nnz = 0, ovl = 0;
    if (n <= (uint32_t)kOvfCap) {
      uint32_t n2 = 32;  // the sort's size: a power of two >= n
      while (n2 < n) n2 <<= 1;
      for (uint32_t k = n + (uint32_t)lane; k < n2; k += 32u) sh.key[k] = ~0ull;
      __syncwarp();
      // bitonic sort of the keys, ascending
      for (uint32_t size = 2; size <= n2; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t i = (uint32_t)lane; i < n2; i += 32u) {
            const uint32_t jx = i ^ stride;
            if (jx > i) {
              const unsigned long long ka = sh.key[i], kb = sh.key[jx];
              const bool up = (i & size) == 0;
              if ((ka > kb) == up) {
                sh.key[i] = kb;
                sh.key[jx] = ka;
              }
            }
          }
          __syncwarp();
        }
      if (lane == 0) {
        for (uint32_t q = 0; q < n; ++q) {
          const uint32_t k = (uint32_t)sh.key[q];
          nnz += sh.flags[k] & 1u;
          if (sh.flags[k] & 2u) {
            fx = __dadd_rn(fx, sh.gx[k]);
            fy = __dadd_rn(fy, sh.gy[k]);
            fz = __dadd_rn(fz, sh.gz[k]);
          }
        }
        ovl = n;
      }
    } else {
      ovf_selection(C, A, stamp, lane, fx, fy, fz, nnz, ovl);
    }
    if (lane == 0) {
      C.c.f64[A.p] = make_double4_32a(fx, fy, fz, (double)ovl);
      C.c.nnz[A.p] = (uint8_t)(nnz > 255u ? 255u : nnz);
    }
    __syncwarp();
  }
}

}  // namespace

void launch_force64(const DevCtx &C, cudaStream_t st) {
  k_force64r<<<(unsigned int)((C.total_slots + kRowAgents - 1) / kRowAgents), kRowThreads, 0, st>>>(C);
  k_force64o<<<152 * 4, 32 * kOvfWarps, 0, st>>>(C);
}

}  // namespace bdm
