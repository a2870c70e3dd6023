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
// listed by colour (count, prefix, fill); then one launch per colour runs
// a group of lanes per box: eight lanes, four boxes to a warp, so that one
// FP64 instruction serves the agents of several boxes, once the context
// holds 131,072 slots or more; a whole warp per box below that, where the
// colours have too few boxes to occupy the groups.  A group first loads
// its box's stencil (first cell and live count of each of the 27 boxes,
// with their prefix) into shared memory.  It then takes the box's agents in
// ascending ID, one after the other; each group takes one agent per pass of
// the loop, so the groups of a warp run side by side.  For each agent, its
// lanes filter the stencil's candidates in FP32 on the records of the
// iteration's start (widened by twice the clamp: each agent moves once, by
// at most the clamp, so every pair that overlaps at the current positions
// passes), compact them, evaluate the definition (pair64) on the current
// positions, sort the overlapping pairs by partner ID (bitonic, in shared
// memory) and add them in that order; the group's first lane then applies
// the displacement (disp64) and the boundary condition before the next
// agent.  A crowd beyond the shared-memory lists takes a selection of the
// next partner ID.  Ghost agents stay in place.  The result equals the
// oracle's in-place iteration bit for bit.
#include "pair.cuh"

namespace bdm {
namespace {

constexpr int kIpWarps = 2;        // warps per block
constexpr int kIpBlocksPerSM = 8;  // 16 warps per SM
constexpr int kIpThreads = 128;    // threads of the list kernels

// G lanes per box: 8 (four boxes of a colour per warp) for large
// populations, 32 (a box per warp) for small ones, where the colours have
// too few boxes to occupy the groups and a whole warp serves an agent faster.
template <int G>
struct IpShared {                   // one per lane group
  static constexpr int kCand = G == 32 ? 512 : 128;  // candidates passing the filter, per agent
  static constexpr int kCap = G == 32 ? 256 : 64;    // overlapping pairs sorted here (a power of two)
  unsigned long long key[kCap];     // partner ID << 32 | index of the contribution
  double gx[kCap], gy[kCap], gz[kCap];
  uint32_t cand[kCand];             // cells that passed the filter
  uint32_t flags[kCap];             // bit 0 non-zero force, bit 1 a direction (distance > 0)
  uint32_t bj[27], bn[27], bp[27];  // stencil boxes: first cell, live count, exclusive prefix of the counts
};

// The box a lane group works on.
struct IpBox {
  int64_t b0;                 // its first cell
  uint32_t nb;                // its agents
  uint32_t ntot;              // candidates of its stencil
  uint32_t bid;               // this lane's agent ID when the agents fit the group
  int nbox, nx, ny, xlo, ylo, zlo;
  int sim;
  float Lh, grow;
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

// Loads box b0 for a lane group (gl: lane in the group): its stencil's
// boxes into shared memory, in the order dx fastest, then dy, then dz, with
// the exclusive prefix of their live counts, and the IDs of its agents when
// they fit the group.
template <int G>
__device__ void ip_load_box(const DevCtx &C, IpShared<G> &sh, IpBox &B, int64_t b0, uint32_t stamp, int gl,
                            unsigned gmask) {
  B.b0 = b0;
  B.sim = C.c.sim[b0];
  const SimConst &sc = C.sc[B.sim];
  const SimState &s = C.ss[B.sim];
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[b0], cx, cy, cz);
  const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
  B.nx = t.xhi - t.xlo + 1;
  B.ny = t.yhi - t.ylo + 1;
  B.nbox = B.nx * B.ny * (t.zhi - t.zlo + 1);
  B.xlo = t.xlo;
  B.ylo = t.ylo;
  B.zlo = t.zlo;
  B.Lh = s.Lh;
  B.grow = __fadd_rn(__fmul_rn(2.f, __double2float_ru(sc.max_disp)), s.marg);
  B.nb = ent_live(t.e[t.box(0, 0, 0)], stamp);
  // lane gl takes stencil boxes kPer gl .. kPer gl + kPer - 1
  constexpr int kPer = (27 + G - 1) / G;
  uint32_t cnt[kPer], sum = 0u;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int bb = kPer * gl + u;
    cnt[u] = 0u;
    if (bb < B.nbox) {
      const int dx = t.xlo + bb % B.nx, dy = t.ylo + (bb / B.nx) % B.ny, dz = t.zlo + bb / (B.nx * B.ny);
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      cnt[u] = ent_live(e, stamp);
      sh.bj[bb] = ent_start(e);
      sh.bn[bb] = cnt[u];
    }
    sum += cnt[u];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int d = 1; d < G; d <<= 1) {
    const uint32_t y = __shfl_up_sync(gmask, incl, d, G);
    incl += gl >= d ? y : 0u;
  }
  uint32_t run = incl - sum;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int bb = kPer * gl + u;
    if (bb < B.nbox) sh.bp[bb] = run;
    run += cnt[u];
  }
  B.ntot = __shfl_sync(gmask, incl, G - 1, G);
  B.bid = (B.nb <= (uint32_t)G && (uint32_t)gl < B.nb) ? agent_id(C, b0 + gl) : 0xFFFFFFFFu;
  __syncwarp(gmask);
}

// The agent's force when its partners do not fit the shared-memory lists:
// the overlapping partner with the next ID, one at a time (group-wide search).
template <int G>
__device__ void ip_selection(const DevCtx &C, const SimConst &sc, const IpShared<G> &sh, const IpBox &B, int64_t q,
                             const double4_32a &o, const float4 &a0, int gl, unsigned gmask, double &fx, double &fy,
                             double &fz, uint32_t &nnz, uint32_t &novl) {
  int64_t prev = -1;
  for (;;) {
    uint32_t best = 0xFFFFFFFFu;
    int64_t bj = -1;
    for (int bb = 0; bb < B.nbox; ++bb) {
      const int dx = B.xlo + bb % B.nx, dy = B.ylo + (bb / B.nx) % B.ny, dz = B.zlo + bb / (B.nx * B.ny);
      const uint32_t cnt = sh.bn[bb];
      const int64_t j0 = sh.bj[bb];
      for (uint32_t m = (uint32_t)gl; m < cnt; m += (uint32_t)G) {
        const int64_t j = j0 + m;
        if (j == q) continue;
        const uint32_t id = agent_id(C, j);
        if ((int64_t)id <= prev || id >= best || !may_overlap(C, a0, j, dx, dy, dz, B.Lh, B.grow)) continue;
        double gx, gy, gz;
        bool nz, dir;
        if (pair64(sc, o, current(C, j), sc.k, sc.gamma, gx, gy, gz, nz, dir)) {
          best = id;
          bj = j;
        }
      }
    }
    const uint32_t gbest = __reduce_min_sync(gmask, best);
    if (gbest == 0xFFFFFFFFu) break;
    const unsigned who = __ballot_sync(gmask, best == gbest && bj >= 0) & gmask;
    const int64_t jb = __shfl_sync(gmask, bj, __ffs(who) - 1);
    if (gl == 0) {
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
    prev = (int64_t)gbest;
  }
}

// One agent of the group's box: the one with the next ID after last_id.
// Returns false when the box has none left (never for a listed box).
template <int G>
__device__ bool ip_agent(const DevCtx &C, IpShared<G> &sh, const IpBox &B, int64_t &last_id, int gl, unsigned gmask,
                         unsigned lt) {
  constexpr uint32_t kCand = IpShared<G>::kCand, kCap = IpShared<G>::kCap;
  const SimConst &sc = C.sc[B.sim];
  uint32_t myid = 0xFFFFFFFFu;
  int64_t myq = -1;
  if (B.nb <= (uint32_t)G) {
    if ((uint32_t)gl < B.nb && (int64_t)B.bid > last_id) {
      myid = B.bid;
      myq = B.b0 + gl;
    }
  } else {
    for (uint32_t m = (uint32_t)gl; m < B.nb; m += (uint32_t)G) {
      const uint32_t id = agent_id(C, B.b0 + m);
      if ((int64_t)id > last_id && id < myid) {
        myid = id;
        myq = B.b0 + m;
      }
    }
  }
  const uint32_t qid = __reduce_min_sync(gmask, myid);
  const unsigned who = __ballot_sync(gmask, myid == qid && myq >= 0) & gmask;
  if (!who) return false;
  const int64_t q = __shfl_sync(gmask, myq, __ffs(who) - 1);
  last_id = (int64_t)qid;
  const int32_t sq = C.c.slot[q];
  const double4_32a o = current(C, q);
  const float4 a0 = C.c.r0[q];
  // the candidates that pass the filter, compacted in stencil-box order and,
  // within a box, in cell order; a lane finds its candidate's box by a
  // binary search over the prefix of the counts
  uint32_t nc = 0;
  for (uint32_t base = 0; base < B.ntot; base += (uint32_t)G) {
    const uint32_t c = base + (uint32_t)gl;
    bool pass = false;
    int64_t j = q;
    if (c < B.ntot) {
      int lo = 0, hi = B.nbox - 1;  // the last stencil box whose prefix is at most c
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sh.bp[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      j = (int64_t)sh.bj[lo] + (int64_t)(c - sh.bp[lo]);
      const int dx = B.xlo + lo % B.nx, dy = B.ylo + (lo / B.nx) % B.ny, dz = B.zlo + lo / (B.nx * B.ny);
      pass = j != q && may_overlap(C, a0, j, dx, dy, dz, B.Lh, B.grow);
    }
    const unsigned bal = __ballot_sync(gmask, pass) & gmask;
    const uint32_t k = nc + (uint32_t)__popc(bal & lt);
    if (pass && k < kCand) sh.cand[k] = (uint32_t)j;
    nc += (uint32_t)__popc(bal);
  }
  __syncwarp(gmask);
  // the overlapping pairs at the current positions, G at a time
  uint32_t n = 0;
  bool select = nc > kCand;
  if (!select) {
    for (uint32_t k0 = 0; k0 < nc; k0 += (uint32_t)G) {
      const uint32_t kk = k0 + (uint32_t)gl;
      double gx = 0.0, gy = 0.0, gz = 0.0;
      bool nz = false, dir = false, hit = false;
      int64_t j = q;
      if (kk < nc) {
        j = (int64_t)sh.cand[kk];
        hit = pair64(sc, o, current(C, j), sc.k, sc.gamma, gx, gy, gz, nz, dir);
      }
      const unsigned bal = __ballot_sync(gmask, hit) & gmask;
      const uint32_t k = n + (uint32_t)__popc(bal & lt);
      if (hit && k < kCap) {
        sh.key[k] = ((unsigned long long)agent_id(C, j) << 32) | k;
        sh.gx[k] = gx;
        sh.gy[k] = gy;
        sh.gz[k] = gz;
        sh.flags[k] = (nz ? 1u : 0u) | (dir ? 2u : 0u);
      }
      n += (uint32_t)__popc(bal);
    }
    select = n > kCap;
  }
  double fx = 0.0, fy = 0.0, fz = 0.0;
  uint32_t nnz = 0, novl = 0;
  if (!select) {
    __syncwarp(gmask);  // the pairs' entries, written by any lane of the group
    if (n > 1u) {       // one pair or none needs no sort
      uint32_t n2 = 2;  // the sort's size: a power of two >= n
      while (n2 < n) n2 <<= 1;
      for (uint32_t k = n + (uint32_t)gl; k < n2; k += (uint32_t)G) sh.key[k] = ~0ull;
      __syncwarp(gmask);
      for (uint32_t size = 2; size <= n2; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t i = (uint32_t)gl; i < n2; i += (uint32_t)G) {
            const uint32_t jx = i ^ stride;
            if (jx > i) {
              const unsigned long long ka = sh.key[i], kb = sh.key[jx];
              if ((ka > kb) == ((i & size) == 0)) {
                sh.key[i] = kb;
                sh.key[jx] = ka;
              }
            }
          }
          __syncwarp(gmask);
        }
    }
    if (gl == 0) {
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
    ip_selection(C, sc, sh, B, q, o, a0, gl, gmask, fx, fy, fz, nnz, novl);
  }
  // the displacement, committed before the next agent
  if (gl == 0) {
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
  __syncwarp(gmask);  // the new position is seen by the box's next agents
  return true;
}

// Groups of G lanes, one box of colour `colour` each (grid-stride over the
// colour's list).  Every group takes one agent per pass of the loop, so the
// groups of a warp run their agents side by side.
template <int G>
__global__ void __launch_bounds__(32 * kIpWarps, kIpBlocksPerSM) k_inplace(DevCtx C, int colour) {
  constexpr int kGroups = 32 / G;
  __shared__ IpShared<G> shg[kIpWarps * kGroups];
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  const unsigned gmask = G == 32 ? FULL : ((1u << (G & 31)) - 1u) << (grp * G);
  const unsigned lt = gmask & ((1u << lane) - 1u);  // lanes of the group below this one
  IpShared<G> &sh = shg[wid * kGroups + grp];
  const uint32_t nlist = C.g->ip_count[colour], off = C.g->ip_off[colour];
  const uint32_t stamp = C.g->stamp & kStampMask;
  const uint32_t stride = gridDim.x * (uint32_t)(kIpWarps * kGroups);
  uint32_t w = (blockIdx.x * (uint32_t)kIpWarps + (uint32_t)wid) * (uint32_t)kGroups + (uint32_t)grp;
  IpBox B{};
  bool have = w < nlist;
  if (have) ip_load_box(C, sh, B, C.ovf[off + w], stamp, gl, gmask);
  uint32_t done = 0;
  int64_t last_id = -1;
  while (__any_sync(FULL, have)) {
    if (!have) continue;
    const bool more = ip_agent(C, sh, B, last_id, gl, gmask, lt);
    if (!more || ++done >= B.nb) {
      w += stride;
      have = w < nlist;
      done = 0;
      last_id = -1;
      if (have) ip_load_box(C, sh, B, C.ovf[off + w], stamp, gl, gmask);
    }
  }
}
}  // namespace

void launch_inplace(const DevCtx &C, cudaStream_t st, int colours, bool narrow) {
  const unsigned int nb = (unsigned int)((C.total_slots + kIpThreads - 1) / kIpThreads);
  k_ip_reset<<<1, 32, 0, st>>>(C);
  k_ip_count<<<nb, kIpThreads, 0, st>>>(C);
  k_ip_prefix<<<1, 1, 0, st>>>(C);
  k_ip_fill<<<nb, kIpThreads, 0, st>>>(C);
  for (int col = 0; col < colours; ++col) {
    if (narrow) k_inplace<8><<<152 * kIpBlocksPerSM, 32 * kIpWarps, 0, st>>>(C, col);
    else k_inplace<32><<<152 * kIpBlocksPerSM, 32 * kIpWarps, 0, st>>>(C, col);
  }
}

}  // namespace bdm
