// S4 pairwise force over the 27-box stencil (Eq 4.1 / Eq 4.2, §4.5.1),
// S5 displacement (adherence threshold, norm clamp) and the static-agent
// skip of §5.5.
//
// FP32 path.  No FP64 arithmetic per pair: every agent carries its offset
// inside its own box, w = (x - o) - c L (exact in FP64 when placed), as a
// float-float pair.  A candidate in the neighbor box at offset dc has the
// center difference x_i - x_j = (w_i - w_j) - dc L, so the FP32 filter and
// the float-float refinement only ever see magnitudes below 2L.  Pairs
// deeper than kFastDelta use the plain FP32 overlap; shallower pairs
// recompute the overlap as (R^2 - s) / (R + dist) in float-float, which
// keeps its relative accuracy as delta shrinks.  The float-float numerator
// carries an absolute error near 1e-12, so when it is within 2^-19 of zero
// (delta below about 1e-7, a rare pair) the FP64 expression of the
// definition gives the sign and size of delta instead.
//
// FP64 path.  The definition, operation by operation, with IEEE FP64
// intrinsics (no contraction): the pair set and the per-pair forces equal
// the definition's; only the order of the sum over neighbors differs.
#include "kernels.cuh"

namespace bdm {

constexpr float kFastDelta = 2.0f;
constexpr float kTinyNum = 0x1p-19f;

__device__ __forceinline__ void ff_diff(float hi_i, float lo_i, float hi_j, float lo_j, float off_h,
                                        float off_l, float &dh, float &dl) {
  float s1, e1, s2, e2;
  two_sum(hi_i, -hi_j, s1, e1);
  two_sum(s1, -off_h, s2, e2);
  float l = __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(__fsub_rn(lo_i, lo_j), off_l));
  fast_two_sum(s2, l, dh, dl);
}

// Overlap of two spheres from the definition in FP64 (used only to decide
// pairs whose float-float overlap is within rounding of zero).
__device__ __noinline__ double exact_delta(const DevCtx &C, int32_t si, int32_t sj) {
  double dx = __dsub_rn(C.a.x[si], C.a.x[sj]);
  double dy = __dsub_rn(C.a.y[si], C.a.y[sj]);
  double dz = __dsub_rn(C.a.z[si], C.a.z[sj]);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double R = __dadd_rn(__dmul_rn(0.5, C.a.d[si]), __dmul_rn(0.5, C.a.d[sj]));
  return __dsub_rn(R, __dsqrt_rn(s));
}

__device__ __forceinline__ void force32(const DevCtx &C, const SimConst &sc, const SimState &s, int64_t p,
                                        int64_t cx, int64_t cy, int64_t cz, uint32_t stamp) {
  const float4 o0 = C.c.r0[p];
  const float4 o1 = C.c.r1[p];
  const float Lh = s.Lh, Ll = s.Ll, marg = s.marg;
  const float kf = sc.kf, gf = sc.gammaf;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  uint32_t nnz = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int64_t z = cz + dz;
    if (z < 0 || z >= s.dims[2]) continue;
    const float ozh = dz ? (dz > 0 ? Lh : -Lh) : 0.f, ozl = dz ? (dz > 0 ? Ll : -Ll) : 0.f;
    for (int dy = -1; dy <= 1; ++dy) {
      int64_t y = cy + dy;
      if (y < 0 || y >= s.dims[1]) continue;
      const float oyh = dy ? (dy > 0 ? Lh : -Lh) : 0.f, oyl = dy ? (dy > 0 ? Ll : -Ll) : 0.f;
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t x = cx + dx;
        if (x < 0 || x >= s.dims[0]) continue;
        const float oxh = dx ? (dx > 0 ? Lh : -Lh) : 0.f, oxl = dx ? (dx > 0 ? Ll : -Ll) : 0.f;
        int64_t idx = sc.table_base + linear_box(s, x, y, z);
        unsigned long long e = C.tab.cnt[idx];
        if ((uint32_t)(e >> 32) != stamp) continue;
        uint32_t cnt = (uint32_t)(e & 0x7FFFFFFFull);
        int64_t start = C.tab.start[idx];
        for (int64_t j = start; j < start + cnt; ++j) {
          if (j == p) continue;
          const float4 q = C.c.r0[j];
          float ddx = __fsub_rn(__fsub_rn(o0.x, q.x), oxh);
          float ddy = __fsub_rn(__fsub_rn(o0.y, q.y), oyh);
          float ddz = __fsub_rn(__fsub_rn(o0.z, q.z), ozh);
          float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
          float R = __fadd_rn(o0.w, q.w);
          float Rm = __fadd_rn(R, marg);
          if (!(s2 < __fmul_rn(Rm, Rm))) continue;
          float dist = sqrtf(s2);
          float del = __fsub_rn(R, dist);
          float ux = ddx, uy = ddy, uz = ddz;
          if (!(del > kFastDelta)) {
            // float-float overlap
            const float4 q1 = C.c.r1[j];
            float xh, xl, yh, yl, zh, zl;
            ff_diff(o0.x, o1.x, q.x, q1.x, oxh, oxl, xh, xl);
            ff_diff(o0.y, o1.y, q.y, q1.y, oyh, oyl, yh, yl);
            ff_diff(o0.z, o1.z, q.z, q1.z, ozh, ozl, zh, zl);
            float p0, e0, p1, e1, p2, e2;
            two_prod(xh, xh, p0, e0);
            e0 = __fmaf_rn(__fmul_rn(2.f, xh), xl, e0);
            two_prod(yh, yh, p1, e1);
            e1 = __fmaf_rn(__fmul_rn(2.f, yh), yl, e1);
            two_prod(zh, zh, p2, e2);
            e2 = __fmaf_rn(__fmul_rn(2.f, zh), zl, e2);
            float S, Se, S2, Se2;
            two_sum(p0, p1, S, Se);
            two_sum(S, p2, S2, Se2);
            float sl = __fadd_rn(__fadd_rn(Se, Se2), __fadd_rn(__fadd_rn(e0, e1), e2));
            float sh, sll;
            fast_two_sum(S2, sl, sh, sll);
            float Rh, Rl;
            two_sum(o0.w, q.w, Rh, Rl);
            Rl = __fadd_rn(Rl, __fadd_rn(o1.w, q1.w));
            float Qh, Ql;
            two_prod(Rh, Rh, Qh, Ql);
            Ql = __fmaf_rn(__fmul_rn(2.f, Rh), Rl, Ql);
            float num = __fadd_rn(__fsub_rn(Qh, sh), __fsub_rn(Ql, sll));
            dist = sqrtf(sh);
            if (fabsf(num) < kTinyNum) {
              double d64 = exact_delta(C, C.c.slot[p], C.c.slot[j]);
              del = d64 > 0.0 ? (float)d64 : 0.f;
              if (!(d64 > 0.0)) continue;
            } else {
              if (!(num > 0.f)) continue;
              del = __fdividef(num, __fadd_rn(Rh, dist));
            }
            ux = xh; uy = yh; uz = zh;
          }
          float rr = __fdividef(__fmul_rn(o0.w, q.w), R);
          float fn = __fsub_rn(__fmul_rn(kf, del), __fmul_rn(gf, sqrtf(__fmul_rn(rr, del))));
          nnz += (fn != 0.f);
          if (dist > 0.f) {
            float sc_ = __fdividef(fn, dist);
            fx = __fmaf_rn(sc_, ux, fx);
            fy = __fmaf_rn(sc_, uy, fy);
            fz = __fmaf_rn(sc_, uz, fz);
          }
        }
      }
    }
  }
  C.c.f32[p] = make_float4(fx, fy, fz, 0.f);
  C.c.nnz[p] = (uint8_t)(nnz > 255u ? 255u : nnz);
}

__device__ __forceinline__ void force64(const DevCtx &C, const SimConst &sc, const SimState &s, int64_t p,
                                        int64_t cx, int64_t cy, int64_t cz, uint32_t stamp) {
  const double4_32a o = C.c.r64[p];
  const double k = sc.k, gam = sc.gamma;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  uint32_t nnz = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int64_t z = cz + dz;
    if (z < 0 || z >= s.dims[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int64_t y = cy + dy;
      if (y < 0 || y >= s.dims[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t x = cx + dx;
        if (x < 0 || x >= s.dims[0]) continue;
        int64_t idx = sc.table_base + linear_box(s, x, y, z);
        unsigned long long e = C.tab.cnt[idx];
        if ((uint32_t)(e >> 32) != stamp) continue;
        uint32_t cnt = (uint32_t)(e & 0x7FFFFFFFull);
        int64_t start = C.tab.start[idx];
        for (int64_t j = start; j < start + cnt; ++j) {
          if (j == p) continue;
          const double4_32a q = C.c.r64[j];
          double ddx = __dsub_rn(o.x, q.x), ddy = __dsub_rn(o.y, q.y), ddz = __dsub_rn(o.z, q.z);
          double s2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
          double R = __dadd_rn(o.w, q.w);
          if (!(s2 < __dmul_rn(R, R) * 1.0000001)) continue;  // cheap reject far beyond contact
          double dist = __dsqrt_rn(s2);
          double del = __dsub_rn(R, dist);
          if (!(del > 0.0)) continue;
          double rr = __ddiv_rn(__dmul_rn(o.w, q.w), R);
          double rep = __dmul_rn(k, del);
          double adh = __dmul_rn(gam, __dsqrt_rn(__dmul_rn(rr, del)));
          double fn = __dsub_rn(rep, adh);
          nnz += (fn != 0.0);
          if (dist > 0.0) {
            fx = __dadd_rn(fx, __dmul_rn(fn, __ddiv_rn(ddx, dist)));
            fy = __dadd_rn(fy, __dmul_rn(fn, __ddiv_rn(ddy, dist)));
            fz = __dadd_rn(fz, __dmul_rn(fn, __ddiv_rn(ddz, dist)));
          }
        }
      }
    }
  }
  C.c.f64[p] = make_double4_32a(fx, fy, fz, 0.0);
  C.c.nnz[p] = (uint8_t)(nnz > 255u ? 255u : nnz);
}

// fp64_only: leave FP32-path simulations to the queue kernel (force32.cu).
__global__ void __launch_bounds__(kThreads) k_force(DevCtx C, int fp64_only) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid) return;
  if (fp64_only && sc.precision != BDM_PREC_FP64) return;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[p], cx, cy, cz);
  uint32_t stamp = C.g->stamp;
  bool st = is_static_cell(C, sc, s, p, cx, cy, cz, stamp);
  C.c.stat[p] = st ? 1 : 0;
  if (st) return;
  if (sc.precision == BDM_PREC_FP64)
    force64(C, sc, s, p, cx, cy, cz, stamp);
  else
    force32(C, sc, s, p, cx, cy, cz, stamp);
}

// S5: displacement.  Static agents keep their position and nnz.
__global__ void __launch_bounds__(kThreads) k_displace(DevCtx C) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  if (!C.ss[sim].valid) return;
  int32_t slot = C.c.slot[p];
  if (C.c.stat[p]) {
    C.a.flags[slot] = FLAG_STATIC;
    return;
  }
  C.a.nnz[slot] = C.c.nnz[p];
  bool moved = false, bad = false;
  if (sc.precision == BDM_PREC_FP64) {
    double4_32a F = C.c.f64[p];
    double fn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(F.x, F.x), __dmul_rn(F.y, F.y)), __dmul_rn(F.z, F.z)));
    bad = !isfinite(fn);
    if (fn > sc.adherence) {
      double Dx = __dmul_rn(sc.dt, F.x), Dy = __dmul_rn(sc.dt, F.y), Dz = __dmul_rn(sc.dt, F.z);
      double dn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy)), __dmul_rn(Dz, Dz)));
      if (dn > sc.max_disp) {
        double f = __ddiv_rn(sc.max_disp, dn);
        Dx = __dmul_rn(Dx, f); Dy = __dmul_rn(Dy, f); Dz = __dmul_rn(Dz, f);
      }
      moved = (Dx != 0.0 || Dy != 0.0 || Dz != 0.0);
      if (moved) {
        C.a.x[slot] = __dadd_rn(C.a.x[slot], Dx);
        C.a.y[slot] = __dadd_rn(C.a.y[slot], Dy);
        C.a.z[slot] = __dadd_rn(C.a.z[slot], Dz);
      }
    }
  } else {
    float4 F = C.c.f32[p];
    float f2 = __fmaf_rn(F.z, F.z, __fmaf_rn(F.y, F.y, __fmul_rn(F.x, F.x)));
    bad = !isfinite(f2);
    if (f2 > sc.adherence2f) {
      float Dx = __fmul_rn(sc.dtf, F.x), Dy = __fmul_rn(sc.dtf, F.y), Dz = __fmul_rn(sc.dtf, F.z);
      float d2 = __fmaf_rn(Dz, Dz, __fmaf_rn(Dy, Dy, __fmul_rn(Dx, Dx)));
      if (d2 > sc.max_disp2f) {
        float f = __fmul_rn(sc.max_dispf, rsqrtf(d2));
        Dx = __fmul_rn(Dx, f); Dy = __fmul_rn(Dy, f); Dz = __fmul_rn(Dz, f);
      }
      moved = (Dx != 0.f || Dy != 0.f || Dz != 0.f);
      if (moved) {
        C.a.x[slot] = __dadd_rn(C.a.x[slot], f2d(Dx));
        C.a.y[slot] = __dadd_rn(C.a.y[slot], f2d(Dy));
        C.a.z[slot] = __dadd_rn(C.a.z[slot], f2d(Dz));
      }
    }
  }
  if (bad) set_err(C.g, ERR_NONFINITE);
  C.a.flags[slot] = moved ? FLAG_CHANGED : 0;
}

static inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

void launch_force(const DevCtx &C, cudaStream_t st, int variant, bool has_fp32, bool has_fp64) {
  if (variant == 0 || variant == 2) {
    if (has_fp32) {
      if (variant == 0) launch_force32s(C, st);
      else launch_force32q(C, st);
    }
    if (has_fp64) k_force<<<blocks_for(C.total_slots, kThreads), kThreads, 0, st>>>(C, 1);
  } else {
    k_force<<<blocks_for(C.total_slots, kThreads), kThreads, 0, st>>>(C, 0);
  }
}

void launch_displace(const DevCtx &C, cudaStream_t st) {
  k_displace<<<blocks_for(C.total_slots, kThreads), kThreads, 0, st>>>(C);
}

}  // namespace bdm
