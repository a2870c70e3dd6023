// Pair arithmetic shared by the force kernels (Eq 4.1 / Eq 4.2, §4.5.1).
//
// FP32 path.  No FP64 arithmetic per pair: every agent carries its offset
// inside its own box, w = (x - o) - c L (exact in FP64 when placed), as a
// float-float pair.  A candidate in the neighbor box at offset dc has the
// center difference x_i - x_j = (w_i - w_j) - dc L, so the FP32 filter and
// the float-float refinement only ever see magnitudes below 2L.  The overlap
// is (R^2 - s) / (R + dist) in float-float, which keeps its relative accuracy
// as delta shrinks; when the float-float numerator is within 2^-19 of zero
// (delta below about 1e-7, a rare pair) the FP64 expression of the
// definition gives the sign and size of delta instead.
//
// Pair counts of the FP32 path travel in the w component of the force:
// every overlapping pair adds 1, and a pair whose force is exactly zero adds
// 65536 more, so that w = overlaps + 65536 x zero-force pairs (exact in FP32
// below 2^24) and the non-zero count is overlaps - zero-force pairs.
#pragma once

#include "kernels.cuh"

namespace bdm {

constexpr float kFastDelta = 0.5f;
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
static __device__ __noinline__ double exact_delta(const DevCtx &C, int32_t si, int32_t sj) {
  const SimConst &sc = C.sc[C.a.sim[si]];  // minimum images on a torus
  double dx = coord_diff(sc, C.a.x[si], C.a.x[sj]);
  double dy = coord_diff(sc, C.a.y[si], C.a.y[sj]);
  double dz = coord_diff(sc, C.a.z[si], C.a.z[sj]);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double R = __dadd_rn(__dmul_rn(0.5, C.a.d[si]), __dmul_rn(0.5, C.a.d[sj]));
  return __dsub_rn(R, __dsqrt_rn(s));
}

// Stencil bounds of a box: neighbor offsets that stay inside the grid (on a
// torus all of them, the boxes wrapping around).
struct Stencil {
  int xlo, xhi, ylo, yhi, zlo, zhi;
  int cx, cy, cz, d0, d1, d2;
  bool torus;
  const unsigned long long *e;    // this simulation's table words
  // table index (in the simulation's region) of stencil box (dx, dy, dz)
  __device__ __forceinline__ uint32_t box(int dx, int dy, int dz) const {
    int x = cx + dx, y = cy + dy, z = cz + dz;
    if (torus) {
      x = x < 0 ? x + d0 : (x >= d0 ? x - d0 : x);
      y = y < 0 ? y + d1 : (y >= d1 ? y - d1 : y);
      z = z < 0 ? z + d2 : (z >= d2 ? z - d2 : z);
    }
    return ((uint32_t)z * (uint32_t)d1 + (uint32_t)y) * (uint32_t)d0 + (uint32_t)x;
  }
};

// kTorus = false: the launch holds no toroidal simulation (no wrap code).
template <bool kTorus = true>
__device__ __forceinline__ Stencil make_stencil(const DevCtx &C, const SimConst &sc, const SimState &s, int64_t cx,
                                                int64_t cy, int64_t cz) {
  Stencil t;
  t.cx = (int)cx; t.cy = (int)cy; t.cz = (int)cz;
  t.d0 = (int)s.dims[0]; t.d1 = (int)s.dims[1]; t.d2 = (int)s.dims[2];
  t.torus = kTorus && sc.boundary == BOUND_TORUS;
  t.xlo = (t.torus || t.cx > 0) ? -1 : 0; t.xhi = (t.torus || t.cx < t.d0 - 1) ? 1 : 0;
  t.ylo = (t.torus || t.cy > 0) ? -1 : 0; t.yhi = (t.torus || t.cy < t.d1 - 1) ? 1 : 0;
  t.zlo = (t.torus || t.cz > 0) ? -1 : 0; t.zhi = (t.torus || t.cz < t.d2 - 1) ? 1 : 0;
  t.e = C.tab.e + sc.table_base;
  return t;
}

// Contribution of candidate j (record q, neighbour-box offset (fdx, fdy,
// fdz)) to the force on p, from the float-float records: the overlap
// delta = (R^2 - s) / (R + dist) keeps its relative accuracy at any depth,
// and the FP64 definition decides when the numerator is within rounding of
// zero.  (One path for every pair: in a warp that evaluates many pairs at
// once, a plain FP32 path for deep pairs beside it cost more than it saved.)
// Returns false when the pair does not interact.
__device__ __forceinline__ bool pair32(const DevCtx &C, int64_t p, const float4 &o0, const float4 &o1, int64_t j,
                                       const float4 &q, float fdx, float fdy, float fdz, float Lh, float Ll,
                                       float kf, float gf, float &fx, float &fy, float &fz, uint32_t &nnz) {
  const float R = __fadd_rn(o0.w, q.w);
  const float4 q1 = C.c.r1[j];
  float xh, xl, yh, yl, zh, zl;
  ff_diff(o0.x, o1.x, q.x, q1.x, __fmul_rn(fdx, Lh), __fmul_rn(fdx, Ll), xh, xl);
  ff_diff(o0.y, o1.y, q.y, q1.y, __fmul_rn(fdy, Lh), __fmul_rn(fdy, Ll), yh, yl);
  ff_diff(o0.z, o1.z, q.z, q1.z, __fmul_rn(fdz, Lh), __fmul_rn(fdz, Ll), zh, zl);
  float p0, e0, p1, e1, p2, e2;
  two_prod(xh, xh, p0, e0);
  e0 = __fmaf_rn(__fmul_rn(2.f, xh), xl, e0);
  two_prod(yh, yh, p1, e1);
  e1 = __fmaf_rn(__fmul_rn(2.f, yh), yl, e1);
  two_prod(zh, zh, p2, e2);
  e2 = __fmaf_rn(__fmul_rn(2.f, zh), zl, e2);
  float Sa, Sea, Sb, Seb;
  two_sum(p0, p1, Sa, Sea);
  two_sum(Sa, p2, Sb, Seb);
  const float sl = __fadd_rn(__fadd_rn(Sea, Seb), __fadd_rn(__fadd_rn(e0, e1), e2));
  float sh, sll;
  fast_two_sum(Sb, sl, sh, sll);
  float Rh, Rl;
  two_sum(o0.w, q.w, Rh, Rl);
  Rl = __fadd_rn(Rl, __fadd_rn(o1.w, q1.w));
  float Qh, Ql;
  two_prod(Rh, Rh, Qh, Ql);
  Ql = __fmaf_rn(__fmul_rn(2.f, Rh), Rl, Ql);
  const float num = __fadd_rn(__fsub_rn(Qh, sh), __fsub_rn(Ql, sll));
  const float dist = sqrtf(sh);
  float del;
  if (fabsf(num) < kTinyNum) {
    const double d64 = exact_delta(C, C.c.slot[p], C.c.slot[j]);
    if (!(d64 > 0.0)) return false;
    del = (float)d64;
  } else {
    if (!(num > 0.f)) return false;
    del = __fdividef(num, __fadd_rn(Rh, dist));
  }
  const float rr = __fdividef(__fmul_rn(o0.w, q.w), R);
  const float fn = __fsub_rn(__fmul_rn(kf, del), __fmul_rn(gf, sqrtf(__fmul_rn(rr, del))));
  nnz += (fn != 0.f);
  if (dist > 0.f) {
    const float f = __fdividef(fn, dist);
    fx = __fmaf_rn(f, xh, fx);
    fy = __fmaf_rn(f, yh, fy);
    fz = __fmaf_rn(f, zh, fz);
  }
  return true;
}

// Pair force of candidate j on p as a vector (the operations of pair32);
// false when the pair does not interact.  nz: the scalar force is not zero.
__device__ __forceinline__ bool pair32_vec(const DevCtx &C, int64_t p, const float4 &o0, const float4 &o1,
                                           int64_t j, const float4 &q, float fdx, float fdy, float fdz, float Lh,
                                           float Ll, float kf, float gf, float &gx, float &gy, float &gz,
                                           bool &nz) {
  float fx = 0.f, fy = 0.f, fz = 0.f;
  uint32_t n = 0;
  const bool hit = pair32(C, p, o0, o1, j, q, fdx, fdy, fdz, Lh, Ll, kf, gf, fx, fy, fz, n);
  gx = fx; gy = fy; gz = fz;
  nz = n != 0u;
  return hit;
}

// Pair force of the FP64 path, the definition operation by operation (Eq.
// 4.1/4.2 and the unit vector from j to i): false when the pair does not
// overlap.  nz: the scalar force is not zero.
__device__ __forceinline__ bool pair64(const SimConst &sc, const double4_32a &o, const double4_32a &q, double k,
                                       double gam, double &gx, double &gy, double &gz, bool &nz, bool &dir) {
  const double ddx = coord_diff(sc, o.x, q.x), ddy = coord_diff(sc, o.y, q.y), ddz = coord_diff(sc, o.z, q.z);
  const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
  const double R = __dadd_rn(o.w, q.w);
  const double dist = __dsqrt_rn(s2);
  const double del = __dsub_rn(R, dist);
  gx = gy = gz = 0.0;
  nz = false;
  dir = dist > 0.0;  // coincident centres: no direction, no force (counted in nnz)
  if (!(del > 0.0)) return false;
  const double rr = __ddiv_rn(__dmul_rn(o.w, q.w), R);
  const double rep = __dmul_rn(k, del);
  const double adh = __dmul_rn(gam, __dsqrt_rn(__dmul_rn(rr, del)));
  const double fn = __dsub_rn(rep, adh);
  nz = fn != 0.0;
  if (dist > 0.0) {
    gx = __dmul_rn(fn, __ddiv_rn(ddx, dist));
    gy = __dmul_rn(fn, __ddiv_rn(ddy, dist));
    gz = __dmul_rn(fn, __ddiv_rn(ddz, dist));
  }
  return true;
}

// Displacement of the FP64 path from the net force F (§4.5.1): zero while
// |F| <= adherence, else dt F with its norm clamped to the maximum
// displacement; operation by operation as the definition.  bad: |F| is not
// finite.  Returns whether the displacement is non-zero.
__device__ __forceinline__ bool disp64(const SimConst &sc, double fx, double fy, double fz, double &Dx, double &Dy,
                                       double &Dz, bool &bad) {
  const double fn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz)));
  bad = !isfinite(fn);
  Dx = Dy = Dz = 0.0;
  if (!(fn > sc.adherence)) return false;
  Dx = __dmul_rn(sc.dt, fx);
  Dy = __dmul_rn(sc.dt, fy);
  Dz = __dmul_rn(sc.dt, fz);
  const double dn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy)), __dmul_rn(Dz, Dz)));
  if (dn > sc.max_disp) {
    const double f = __ddiv_rn(sc.max_disp, dn);
    Dx = __dmul_rn(Dx, f);
    Dy = __dmul_rn(Dy, f);
    Dz = __dmul_rn(Dz, f);
  }
  return Dx != 0.0 || Dy != 0.0 || Dz != 0.0;
}

// Pair force of candidate j on an owner with records (o0, o1) and the
// owner simulation's L (Lh, Ll), k and gamma, as a vector, for the stream
// kernel: the arithmetic of pair32 with square roots as x rsqrt(x) (relative
// error near 2^-22, far below the FP32 path's tolerance; the overlap's sign
// comes from the float-float numerator, not from a root).  nz: the scalar
// force is not zero.  Returns false when the pair does not interact.
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.f ? __fmul_rn(x, rsqrtf(x)) : 0.f; }

__device__ __forceinline__ bool pair32_lite(const DevCtx &C, int64_t p, const float4 &o0, const float4 &o1, int64_t j,
                                            float fdx, float fdy, float fdz, float Lh, float Ll, float kf, float gf,
                                            float &gx, float &gy, float &gz, bool &nz) {
  const float4 q = C.c.r0[j], q1 = C.c.r1[j];
  float xh, xl, yh, yl, zh, zl;
  ff_diff(o0.x, o1.x, q.x, q1.x, __fmul_rn(fdx, Lh), __fmul_rn(fdx, Ll), xh, xl);
  ff_diff(o0.y, o1.y, q.y, q1.y, __fmul_rn(fdy, Lh), __fmul_rn(fdy, Ll), yh, yl);
  ff_diff(o0.z, o1.z, q.z, q1.z, __fmul_rn(fdz, Lh), __fmul_rn(fdz, Ll), zh, zl);
  float p0, e0, p1, e1, p2, e2;
  two_prod(xh, xh, p0, e0);
  e0 = __fmaf_rn(__fmul_rn(2.f, xh), xl, e0);
  two_prod(yh, yh, p1, e1);
  e1 = __fmaf_rn(__fmul_rn(2.f, yh), yl, e1);
  two_prod(zh, zh, p2, e2);
  e2 = __fmaf_rn(__fmul_rn(2.f, zh), zl, e2);
  float Sa, Sea, Sb, Seb;
  two_sum(p0, p1, Sa, Sea);
  two_sum(Sa, p2, Sb, Seb);
  const float sl = __fadd_rn(__fadd_rn(Sea, Seb), __fadd_rn(__fadd_rn(e0, e1), e2));
  float sh, sll;
  fast_two_sum(Sb, sl, sh, sll);
  float Rh, Rl;
  two_sum(o0.w, q.w, Rh, Rl);
  Rl = __fadd_rn(Rl, __fadd_rn(o1.w, q1.w));
  float Qh, Ql;
  two_prod(Rh, Rh, Qh, Ql);
  Ql = __fmaf_rn(__fmul_rn(2.f, Rh), Rl, Ql);
  const float num = __fadd_rn(__fsub_rn(Qh, sh), __fsub_rn(Ql, sll));
  const float dist = sqrt_fast(sh);
  float del = __fdividef(num, __fadd_rn(Rh, dist));
  bool hit = num > 0.f;
  if (fabsf(num) < kTinyNum) {
    const double d64 = exact_delta(C, C.c.slot[p], C.c.slot[j]);
    hit = d64 > 0.0;
    del = (float)d64;
  }
  const float R = __fadd_rn(o0.w, q.w);
  const float rr = __fdividef(__fmul_rn(o0.w, q.w), R);
  const float fn = __fsub_rn(__fmul_rn(kf, del), __fmul_rn(gf, sqrt_fast(__fmul_rn(rr, del))));
  nz = fn != 0.f;
  const float f = dist > 0.f ? __fdividef(fn, dist) : 0.f;
  gx = __fmul_rn(f, xh);
  gy = __fmul_rn(f, yh);
  gz = __fmul_rn(f, zh);
  return hit;
}

// Count word of one overlapping pair (see above).
__device__ __forceinline__ float pair_count_word(bool nz) { return nz ? 1.f : 65537.f; }

// Decoded counts of a force's w component.
__device__ __forceinline__ void decode_counts(float w, uint32_t &overlaps, uint32_t &nonzero) {
  const uint32_t v = (uint32_t)w;
  overlaps = v & 0xFFFFu;
  const uint32_t zeros = v >> 16;
  nonzero = overlaps > zeros ? overlaps - zeros : 0u;
}

}  // namespace bdm
