// S4 + S5 under the in-place execution context (§5.2), FP64 path.
//
// In the in-place context an agent's new position is visible to the agents
// processed after it in the same iteration.  The order is fixed so that a
// GPU can run it: boxes by colour, then boxes of a colour in ascending
// index, then the agents of a box in ascending ID.  The colour of a box is
// the parity of each box coordinate, except that on a toroidal axis with an
// odd number of boxes the last box has a third colour (it touches box 0
// across the seam); colours rank x + k_x (y + k_y z).  Two boxes of one
// colour are never in each other's 27-box stencil, and an agent writes only
// its own position, so all boxes of a colour run at once.
//
// Per iteration: the box leaders (first cell of each occupied box) are
// listed by colour (count, prefix, fill); then one launch per colour runs a
// warp per box over that colour's list.  The warp takes the box's agents in
// ascending ID, one after the other.  For each, its lanes filter the
// stencil's candidates in FP32 on the records of the iteration's start
// (widened by twice the clamp: each agent moves once, by at most the clamp,
// so every pair that overlaps at the current positions passes), compact
// them, evaluate the definition (pair64) on the current positions 32 at a
// time, sort the overlapping pairs by partner ID (bitonic, in shared
// memory) and add them in that order; lane 0 then applies the displacement
// (disp64) and the boundary condition before the next agent.  A crowd beyond
// the shared-memory lists takes a selection of the next partner ID.  Ghost
// agents stay in place.  The result equals the oracle's in-place iteration
// bit for bit.
#include "pair.cuh"

namespace bdm {
namespace {

constexpr int kIpWarps = 4;      // warps (boxes) per block
constexpr int kIpCand = 512;     // candidates passing the filter, per agent
constexpr int kIpCap = 256;      // overlapping pairs sorted in shared memory (a power of two)
constexpr int kIpThreads = 128;  // threads of the list kernels

struct IpShared {
  uint32_t cand[kIpCand];            // cells that passed the filter
  unsigned long long key[kIpCap];    // partner ID << 32 | index of the contribution
  double gx[kIpCap], gy[kIpCap], gz[kIpCap];
  uint32_t flags[kIpCap];            // bit 0 non-zero force, bit 1 a direction (distance > 0)
};

__device__ __forceinline__ uint32_t agent_id(const DevCtx &C, int64_t j) { return (uint32_t)C.a.id[C.c.slot[j]]; }

// The current record (x, y, z, r) of cell j's agent.
__device__ __forceinline__ double4_32a current(const DevCtx &C, int64_t j) {
  const int32_t sl = C.c.slot[j];
  return make_double4_32a(C.a.x[sl], C.a.y[sl], C.a.z[sl], half_of(C.a.d[sl]));
}

// Colours per axis of a simulation's grid and the colour of box (cx, cy, cz).
__device__ __forceinline__ int box_colour(const SimConst &sc, const SimState &s, int64_t cx, int64_t cy, int64_t cz) {
  const bool torus = sc.boundary == BOUND_TORUS;
  const int64_t c[3] = {cx, cy, cz};
  int col[3], k[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    k[a] = (torus && (s.dims[a] & 1)) ? 3 : 2;
    col[a] = (k[a] == 3 && c[a] == s.dims[a] - 1) ? 2 : (int)(c[a] & 1);
  }
  return col[0] + k[0] * (col[1] + k[1] * col[2]);
}

// Colour of cell p's box when p leads it (its first cell) in an in-place
// simulation, else -1.
__device__ __forceinline__ int leader_colour(const DevCtx &C, int64_t p, uint32_t stamp) {
  const int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid || sc.exec_ctx != BDM_EXEC_INPLACE) return -1;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[p], cx, cy, cz);
  const unsigned long long e = C.tab.e[sc.table_base + linear_box(s, cx, cy, cz)];
  if (ent_live(e, stamp) == 0u || (int64_t)ent_start(e) != p) return -1;
  return box_colour(sc, s, cx, cy, cz);
}

__global__ void k_ip_reset(DevCtx C) {
  if (threadIdx.x < 27) C.g->ip_count[threadIdx.x] = 0u;
}

__global__ void __launch_bounds__(kIpThreads) k_ip_count(DevCtx C) {
  if (C.g->err & ERR_TABLE) return;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  const int col = leader_colour(C, p, C.g->stamp & kStampMask);
  if (col >= 0) atomicAdd(&C.g->ip_count[col], 1u);
}

__global__ void k_ip_prefix(DevCtx C) {
  uint32_t o = 0;
  for (int k = 0; k < 27; ++k) {
    C.g->ip_off[k] = o;
    C.g->ip_cursor[k] = o;
    o += C.g->ip_count[k];
  }
  C.g->ip_off[27] = o;
}

__global__ void __launch_bounds__(kIpThreads) k_ip_fill(DevCtx C) {
  if (C.g->err & ERR_TABLE) return;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  const int col = leader_colour(C, p, C.g->stamp & kStampMask);
  if (col >= 0) C.ovf[atomicAdd(&C.g->ip_cursor[col], 1u)] = (int32_t)p;
}

// FP32 filter on the start records: cell j, in the box at offset (dx, dy,
// dz) from the agent's, against the agent's record a; radii plus `grow`.
__device__ __forceinline__ bool may_overlap(const DevCtx &C, const float4 &a, int64_t j, int dx, int dy, int dz,
                                            float Lh, float grow) {
  const float4 b = C.c.r0[j];
  const float ddx = __fsub_rn(__fsub_rn(a.x, __fmul_rn((float)dx, Lh)), b.x);
  const float ddy = __fsub_rn(__fsub_rn(a.y, __fmul_rn((float)dy, Lh)), b.y);
  const float ddz = __fsub_rn(__fsub_rn(a.z, __fmul_rn((float)dz, Lh)), b.z);
  const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
  const float R = __fadd_rn(__fadd_rn(a.w, b.w), grow);
  return s2 < __fmul_rn(R, R);
}

// The agent's force when its partners do not fit the shared-memory lists:
// the overlapping partner with the next ID, one at a time (warp-wide search).
__device__ void ip_selection(const DevCtx &C, const SimConst &sc, const Stencil &t, int64_t q, const double4_32a &o,
                             const float4 &a0, uint32_t stamp, int lane, float Lh, float grow, double &fx,
                             double &fy, double &fz, uint32_t &nnz, uint32_t &novl) {
  const unsigned FULL = 0xffffffffu;
  const int nx = t.xhi - t.xlo + 1, ny = t.yhi - t.ylo + 1, nzb = t.zhi - t.zlo + 1;
  const int nbox = nx * ny * nzb;
  int64_t prev = -1;
  for (;;) {
    uint32_t best = 0xFFFFFFFFu;
    int64_t bj = -1;
    for (int bb = 0; bb < nbox; ++bb) {
      const int dx = t.xlo + bb % nx, dy = t.ylo + (bb / nx) % ny, dz = t.zlo + bb / (nx * ny);
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      const uint32_t cnt = ent_live(e, stamp);
      const int64_t j0 = ent_start(e);
      for (uint32_t m = (uint32_t)lane; m < cnt; m += 32u) {
        const int64_t j = j0 + m;
        if (j == q) continue;
        const uint32_t id = agent_id(C, j);
        if ((int64_t)id <= prev || id >= best || !may_overlap(C, a0, j, dx, dy, dz, Lh, grow)) continue;
        double gx, gy, gz;
        bool nz, dir;
        if (pair64(sc, o, current(C, j), sc.k, sc.gamma, gx, gy, gz, nz, dir)) {
          best = id;
          bj = j;
        }
      }
    }
    const uint32_t wbest = __reduce_min_sync(FULL, best);
    if (wbest == 0xFFFFFFFFu) break;
    const unsigned who = __ballot_sync(FULL, best == wbest && bj >= 0);
    const int64_t jb = __shfl_sync(FULL, bj, __ffs(who) - 1);
    if (lane == 0) {
      double gx, gy, gz;
      bool nz, dir;
      pair64(sc, o, current(C, jb), sc.k, sc.gamma, gx, gy, gz, nz, dir);
      ++novl;
      nnz += nz ? 1u : 0u;
      if (dir) {
        fx = __dadd_rn(fx, gx);
        fy = __dadd_rn(fy, gy);
        fz = __dadd_rn(fz, gz);
      }
    }
    prev = (int64_t)wbest;
  }
}

// One warp per box of colour `colour` (grid-stride over the colour's list).
__global__ void __launch_bounds__(32 * kIpWarps) k_inplace(DevCtx C, int colour) {
  __shared__ IpShared shw[kIpWarps];
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  IpShared &sh = shw[wid];
  const uint32_t nlist = C.g->ip_count[colour], off = C.g->ip_off[colour];
  const uint32_t stamp = C.g->stamp & kStampMask;
  for (uint32_t w = blockIdx.x * kIpWarps + wid; w < nlist; w += gridDim.x * kIpWarps) {
    const int64_t b0 = C.ovf[off + w];  // the box's first cell
    const int sim = C.c.sim[b0];
    const SimConst &sc = C.sc[sim];
    const SimState &s = C.ss[sim];
    int64_t cx, cy, cz;
    unpack_coords(C.c.pkey[b0], cx, cy, cz);
    const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
    const uint32_t nb = ent_live(t.e[t.box(0, 0, 0)], stamp);
    const int nx = t.xhi - t.xlo + 1, ny = t.yhi - t.ylo + 1, nzb = t.zhi - t.zlo + 1;
    const int nbox = nx * ny * nzb;
    const float Lh = s.Lh;
    const float grow = __fadd_rn(__fmul_rn(2.f, __double2float_ru(sc.max_disp)), s.marg);
    // The box's agents share its stencil: lane b < nbox holds stencil box b's
    // first cell and live count, and every lane the inclusive prefix of the
    // counts up to its own (lanes from nbox on hold the total), read once per
    // box instead of box by box for every agent.
    int64_t bj0 = 0;
    uint32_t bcnt = 0u;
    if (lane < nbox) {
      const int dx = t.xlo + lane % nx, dy = t.ylo + (lane / nx) % ny, dz = t.zlo + lane / (nx * ny);
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      bcnt = ent_live(e, stamp);
      bj0 = ent_start(e);
    }
    uint32_t bincl = bcnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, bincl, d);
      bincl += lane >= d ? y : 0u;
    }
    const uint32_t ntot = __shfl_sync(FULL, bincl, 31);
    // IDs of the box's agents, one per lane, when they fit the warp
    const uint32_t bid = (nb <= 32u && (uint32_t)lane < nb) ? agent_id(C, b0 + lane) : 0xFFFFFFFFu;
    int64_t last_id = -1;
    for (uint32_t done = 0; done < nb; ++done) {
      // the box's agent with the next ID
      uint32_t myid = 0xFFFFFFFFu;
      int64_t myq = -1;
      if (nb <= 32u) {
        if ((uint32_t)lane < nb && (int64_t)bid > last_id) {
          myid = bid;
          myq = b0 + lane;
        }
      } else {
        for (uint32_t m = (uint32_t)lane; m < nb; m += 32u) {
          const uint32_t id = agent_id(C, b0 + m);
          if ((int64_t)id > last_id && id < myid) {
            myid = id;
            myq = b0 + m;
          }
        }
      }
      const uint32_t qid = __reduce_min_sync(FULL, myid);
      const unsigned who = __ballot_sync(FULL, myid == qid && myq >= 0);
      if (!who) break;  // IDs are distinct: never taken
      const int64_t q = __shfl_sync(FULL, myq, __ffs(who) - 1);
      last_id = (int64_t)qid;
      const int32_t sq = C.c.slot[q];
      const double4_32a o = current(C, q);
      const float4 a0 = C.c.r0[q];
      // the candidates that pass the filter, compacted in stencil-box order
      // and, within a box, in cell order: 32 candidates of the stencil's
      // ntot per round, each lane finding its box by a binary search over
      // the prefix of the counts
      uint32_t nc = 0;
      for (uint32_t base = 0; base < ntot; base += 32u) {
        const uint32_t c = base + (uint32_t)lane;
        int lo = 0, hi = 31;  // the first lane whose inclusive prefix exceeds c
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int mid = (lo + hi) >> 1;
          const uint32_t v = __shfl_sync(FULL, bincl, mid);
          if (v > c) hi = mid;
          else lo = mid + 1;
        }
        lo = lo < 31 ? lo : 31;  // only lanes past the last candidate get beyond
        const uint32_t ib = __shfl_sync(FULL, bincl, lo), nbx = __shfl_sync(FULL, bcnt, lo);
        const int64_t jb = __shfl_sync(FULL, bj0, lo);
        const int64_t j = jb + (int64_t)(c - (ib - nbx));
        const int dx = t.xlo + lo % nx, dy = t.ylo + (lo / nx) % ny, dz = t.zlo + lo / (nx * ny);
        const bool pass = c < ntot && j != q && may_overlap(C, a0, j, dx, dy, dz, Lh, grow);
        const unsigned B = __ballot_sync(FULL, pass);
        const uint32_t k = nc + (uint32_t)__popc(B & lt);
        if (pass && k < (uint32_t)kIpCand) sh.cand[k] = (uint32_t)j;
        nc += (uint32_t)__popc(B);
      }
      __syncwarp();
      // the overlapping pairs at the current positions, 32 at a time
      uint32_t n = 0;
      bool select = nc > (uint32_t)kIpCand;
      if (!select) {
        for (uint32_t k0 = 0; k0 < nc; k0 += 32u) {
          const uint32_t kk = k0 + (uint32_t)lane;
          const int64_t j = kk < nc ? (int64_t)sh.cand[kk] : q;
          double gx = 0.0, gy = 0.0, gz = 0.0;
          bool nz = false, dir = false, hit = false;
          if (kk < nc) hit = pair64(sc, o, current(C, j), sc.k, sc.gamma, gx, gy, gz, nz, dir);
          const unsigned B = __ballot_sync(FULL, hit);
          const uint32_t k = n + (uint32_t)__popc(B & lt);
          if (hit && k < (uint32_t)kIpCap) {
            sh.key[k] = ((unsigned long long)agent_id(C, j) << 32) | k;
            sh.gx[k] = gx; sh.gy[k] = gy; sh.gz[k] = gz;
            sh.flags[k] = (nz ? 1u : 0u) | (dir ? 2u : 0u);
          }
          n += (uint32_t)__popc(B);
        }
        select = n > (uint32_t)kIpCap;
      }
      double fx = 0.0, fy = 0.0, fz = 0.0;
      uint32_t nnz = 0, novl = 0;
      if (!select) {
        if (n > 1u) {  // one pair or none needs no sort
          uint32_t n2 = 32;  // the sort's size: a power of two >= n
          while (n2 < n) n2 <<= 1;
          for (uint32_t k = n + (uint32_t)lane; k < n2; k += 32u) sh.key[k] = ~0ull;
          __syncwarp();
          for (uint32_t size = 2; size <= n2; size <<= 1)
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
              for (uint32_t i = (uint32_t)lane; i < n2; i += 32u) {
                const uint32_t jx = i ^ stride;
                if (jx > i) {
                  const unsigned long long ka = sh.key[i], kb = sh.key[jx];
                  if ((ka > kb) == ((i & size) == 0)) {
                    sh.key[i] = kb;
                    sh.key[jx] = ka;
                  }
                }
              }
              __syncwarp();
            }
        } else {
          __syncwarp();  // the one pair's entries, written by any lane
        }
        if (lane == 0) {
          for (uint32_t r = 0; r < n; ++r) {
            const uint32_t k = (uint32_t)sh.key[r];
            nnz += sh.flags[k] & 1u;
            if (sh.flags[k] & 2u) {
              fx = __dadd_rn(fx, sh.gx[k]);
              fy = __dadd_rn(fy, sh.gy[k]);
              fz = __dadd_rn(fz, sh.gz[k]);
            }
          }
          novl = n;
        }
      } else {
        ip_selection(C, sc, t, q, o, a0, stamp, lane, Lh, grow, fx, fy, fz, nnz, novl);
      }
      // the displacement, committed before the next agent
      if (lane == 0) {
        const uint8_t ghost = C.a.flags[sq] & FLAG_GHOST;
        double Dx, Dy, Dz;
        bool bad;
        const bool moved = disp64(sc, fx, fy, fz, Dx, Dy, Dz, bad) && !ghost;
        if (bad) set_err(C.g, ERR_NONFINITE);
        if (moved) {
          C.a.x[sq] = bound_apply(sc, __dadd_rn(o.x, Dx));
          C.a.y[sq] = bound_apply(sc, __dadd_rn(o.y, Dy));
          C.a.z[sq] = bound_apply(sc, __dadd_rn(o.z, Dz));
        }
        const uint8_t nz8 = (uint8_t)(nnz > 255u ? 255u : nnz);
        C.c.f64[q] = make_double4_32a(fx, fy, fz, (double)novl);
        C.c.nnz[q] = nz8;
        C.c.stat[q] = 0;
        C.a.nnz[sq] = nz8;
        C.a.flags[sq] = (uint8_t)(ghost | (moved ? FLAG_CHANGED : 0));
      }
      __syncwarp();  // the new position is seen by the next agents of the box
    }
  }
}

}  // namespace

void launch_inplace(const DevCtx &C, cudaStream_t st, int colours) {
  const unsigned int nb = (unsigned int)((C.total_slots + kIpThreads - 1) / kIpThreads);
  k_ip_reset<<<1, 32, 0, st>>>(C);
  k_ip_count<<<nb, kIpThreads, 0, st>>>(C);
  k_ip_prefix<<<1, 1, 0, st>>>(C);
  k_ip_fill<<<nb, kIpThreads, 0, st>>>(C);
  for (int col = 0; col < colours; ++col) k_inplace<<<152 * 4, 32 * kIpWarps, 0, st>>>(C, col);
}

}  // namespace bdm
