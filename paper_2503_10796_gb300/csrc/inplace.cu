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
// its own position, so all boxes of a colour run at once: one launch per
// colour, one thread per box (its first cell), the box's agents in
// ascending ID one after the other.
//
// An agent's neighbours are the agents of its stencil in the grid built at
// the iteration's start, at their current positions (storage arrays, which
// earlier colours and earlier agents of the box have updated).  Candidates
// pass an FP32 filter on the start records first, widened by twice the
// clamp (each agent moves once, by at most the clamp).  Pair forces are
// evaluated by the definition (pair64) and added in ascending partner ID; the displacement (disp64) and the boundary condition are
// applied at once.  Ghost agents stay in place.  The result equals the
// oracle's in-place iteration bit for bit.
#include "pair.cuh"

namespace bdm {
namespace {

constexpr int kInThreads = 128;
constexpr int kInCap = 48;  // partners sorted in registers/local memory; more take the selection loop

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

struct Contrib {
  double gx, gy, gz;
  uint32_t id, flags;  // flags: bit 0 non-zero force, bit 1 a direction (distance > 0)
};

__global__ void __launch_bounds__(kInThreads) k_inplace(DevCtx C, int colour) {
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  const int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid || sc.exec_ctx != BDM_EXEC_INPLACE) return;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[p], cx, cy, cz);
  const uint32_t stamp = C.g->stamp & kStampMask;
  const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
  const unsigned long long eb = t.e[t.box(0, 0, 0)];
  const int64_t b0 = ent_start(eb);
  const uint32_t nb = ent_live(eb, stamp);
  if (p != b0 || box_colour(sc, s, cx, cy, cz) != colour) return;  // one thread per box of this colour
  const int nx = t.xhi - t.xlo + 1, ny = t.yhi - t.ylo + 1, nzb = t.zhi - t.zlo + 1;
  const int nbox = nx * ny * nzb;
  // FP32 filter on the records of the iteration's start (box-relative
  // leading parts): an agent moves once per iteration, by at most the
  // clamp, so a pair that overlaps at the current positions lies within
  // r_i + r_j + 2 max_displacement at the start (plus the records' margin)
  const float Lh = s.Lh;
  const float grow = __fadd_rn(__fmul_rn(2.f, __double2float_ru(sc.max_disp)), s.marg);
  auto may_overlap = [&](const float4 &a, int64_t j, int dx, int dy, int dz) {
    const float4 b = C.c.r0[j];
    const float ddx = __fsub_rn(__fsub_rn(a.x, __fmul_rn((float)dx, Lh)), b.x);
    const float ddy = __fsub_rn(__fsub_rn(a.y, __fmul_rn((float)dy, Lh)), b.y);
    const float ddz = __fsub_rn(__fsub_rn(a.z, __fmul_rn((float)dz, Lh)), b.z);
    const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
    const float R = __fadd_rn(__fadd_rn(a.w, b.w), grow);
    return s2 < __fmul_rn(R, R);
  };
  int64_t last_id = -1;
  for (uint32_t done = 0; done < nb; ++done) {
    // the box's agent with the next ID
    int64_t q = -1;
    uint32_t qid = 0xFFFFFFFFu;
    for (uint32_t m = 0; m < nb; ++m) {
      const uint32_t id = agent_id(C, b0 + m);
      if ((int64_t)id > last_id && id < qid) {
        qid = id;
        q = b0 + m;
      }
    }
    if (q < 0) break;  // IDs are distinct: never taken
    last_id = (int64_t)qid;
    const int32_t sq = C.c.slot[q];
    const double4_32a o = current(C, q);
    const float4 a0 = C.c.r0[q];
    // its overlapping partners, kept sorted by ID while they fit
    Contrib con[kInCap];
    uint32_t n = 0;
    for (int bb = 0; bb < nbox; ++bb) {
      const int dx = t.xlo + bb % nx, dy = t.ylo + (bb / nx) % ny, dz = t.zlo + bb / (nx * ny);
      const unsigned long long e = t.e[t.box(dx, dy, dz)];
      const uint32_t cnt = ent_live(e, stamp);
      const int64_t j0 = ent_start(e);
      for (uint32_t m = 0; m < cnt; ++m) {
        const int64_t j = j0 + m;
        if (j == q || !may_overlap(a0, j, dx, dy, dz)) continue;
        double gx, gy, gz;
        bool nz, dir;
        if (!pair64(sc, o, current(C, j), sc.k, sc.gamma, gx, gy, gz, nz, dir)) continue;
        if (n < (uint32_t)kInCap) {
          const uint32_t id = agent_id(C, j);
          uint32_t k = n;
          while (k > 0 && con[k - 1].id > id) {
            con[k] = con[k - 1];
            --k;
          }
          con[k].gx = gx; con[k].gy = gy; con[k].gz = gz;
          con[k].id = id;
          con[k].flags = (nz ? 1u : 0u) | (dir ? 2u : 0u);
        }
        ++n;
      }
    }
    double fx = 0.0, fy = 0.0, fz = 0.0;
    uint32_t nnz = 0;
    if (n <= (uint32_t)kInCap) {
      for (uint32_t k = 0; k < n; ++k) {
        nnz += con[k].flags & 1u;
        if (con[k].flags & 2u) {
          fx = __dadd_rn(fx, con[k].gx);
          fy = __dadd_rn(fy, con[k].gy);
          fz = __dadd_rn(fz, con[k].gz);
        }
      }
    } else {
      // a crowd: the partner with the next ID, one at a time
      int64_t prev = -1;
      for (uint32_t k = 0; k < n; ++k) {
        uint32_t best = 0xFFFFFFFFu;
        int64_t bj = -1;
        for (int bb = 0; bb < nbox; ++bb) {
          const int dx = t.xlo + bb % nx, dy = t.ylo + (bb / nx) % ny, dz = t.zlo + bb / (nx * ny);
          const unsigned long long e = t.e[t.box(dx, dy, dz)];
          const uint32_t cnt = ent_live(e, stamp);
          const int64_t j0 = ent_start(e);
          for (uint32_t m = 0; m < cnt; ++m) {
            const int64_t j = j0 + m;
            if (j == q) continue;
            const uint32_t id = agent_id(C, j);
            if ((int64_t)id <= prev || id >= best || !may_overlap(a0, j, dx, dy, dz)) continue;
            double gx, gy, gz;
            bool nz, dir;
            if (pair64(sc, o, current(C, j), sc.k, sc.gamma, gx, gy, gz, nz, dir)) {
              best = id;
              bj = j;
            }
          }
        }
        if (bj < 0) break;
        double gx, gy, gz;
        bool nz, dir;
        pair64(sc, o, current(C, bj), sc.k, sc.gamma, gx, gy, gz, nz, dir);
        nnz += nz ? 1u : 0u;
        if (dir) {
          fx = __dadd_rn(fx, gx);
          fy = __dadd_rn(fy, gy);
          fz = __dadd_rn(fz, gz);
        }
        prev = (int64_t)best;
      }
    }
    // the displacement, committed at once
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
    C.c.f64[q] = make_double4_32a(fx, fy, fz, (double)n);
    C.c.nnz[q] = nz8;
    C.c.stat[q] = 0;
    C.a.nnz[sq] = nz8;
    C.a.flags[sq] = (uint8_t)(ghost | (moved ? FLAG_CHANGED : 0));
  }
}

}  // namespace

void launch_inplace(const DevCtx &C, cudaStream_t st, int colours) {
  const unsigned int nb = (unsigned int)((C.total_slots + kInThreads - 1) / kInThreads);
  for (int col = 0; col < colours; ++col) k_inplace<<<nb, kInThreads, 0, st>>>(C, col);
}

}  // namespace bdm
