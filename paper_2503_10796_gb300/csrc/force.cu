// S4 pairwise force over the 27-box stencil (Eq 4.1 / Eq 4.2, §4.5.1),
// S5 displacement (adherence threshold, norm clamp) and the static-agent
// skip of §5.5.  The pair arithmetic of both paths is in pair.cuh; the
// warp candidate-stream kernel of the FP32 path is in force_stream.cu.
//
// FP64 path.  The definition, operation by operation, with IEEE FP64
// intrinsics (no contraction): the pair set and the per-pair forces equal
// the definition's.
#include "pair.cuh"

namespace bdm {

// Direct FP32 loop: per stencil box the own offset is shifted into the
// neighbour box's frame once; per candidate the FP32 filter, and for pairs
// that pass either the plain FP32 overlap (deep pairs) or the float-float
// overlap (shallow pairs).  Box indices are 32-bit offsets inside the
// simulation's table region (the grid holds fewer than 2^32 boxes).
__device__ __forceinline__ void force32(const DevCtx &C, const SimConst &sc, const SimState &s, int64_t p,
                                        int64_t cx, int64_t cy, int64_t cz, uint32_t stamp) {
  const float4 o0 = C.c.r0[p];
  const float4 o1 = C.c.r1[p];
  const float Lh = s.Lh, Ll = s.Ll, marg = s.marg;
  const float kf = sc.kf, gf = sc.gammaf;
  const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
  float fx = 0.f, fy = 0.f, fz = 0.f;
  uint32_t nnz = 0, ovl = 0, zeros = 0;
  for (int dz = t.zlo; dz <= t.zhi; ++dz) {
    const float fdz = (float)dz;
    const float sz = __fsub_rn(o0.z, __fmul_rn(fdz, Lh));
    for (int dy = t.ylo; dy <= t.yhi; ++dy) {
      const float fdy = (float)dy;
      const float sy = __fsub_rn(o0.y, __fmul_rn(fdy, Lh));
      const uint32_t row = ((uint32_t)(t.cz + dz) * (uint32_t)t.d1 + (uint32_t)(t.cy + dy)) * (uint32_t)t.d0 +
                           (uint32_t)t.cx;
      // the row's (up to) three table words and starts, loaded together
      unsigned long long ew[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int dx = q - 1;
        const bool in = dx >= t.xlo && dx <= t.xhi;
        ew[q] = in ? __ldg(t.e + row + dx) : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int dx = q - 1;
        const unsigned long long e = ew[q];
        const uint32_t cnt = ent_live(e, stamp);
        if (!cnt) continue;
        const int64_t j0 = ent_start(e);
        const float fdx = (float)dx;
        const float sx = __fsub_rn(o0.x, __fmul_rn(fdx, Lh));
        for (uint32_t m = 0; m < cnt; ++m) {
          const int64_t j = j0 + m;
          if (j == p) continue;
          const float4 q = C.c.r0[j];
          const float ddx = __fsub_rn(sx, q.x), ddy = __fsub_rn(sy, q.y), ddz = __fsub_rn(sz, q.z);
          const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
          const float R = __fadd_rn(o0.w, q.w);
          const float Rm = __fadd_rn(R, marg);
          if (!(s2 < __fmul_rn(Rm, Rm))) continue;
          float dist = sqrtf(s2);
          float del = __fsub_rn(R, dist);
          float ux = ddx, uy = ddy, uz = ddz;
          if (!(del > kFastDelta)) {
            // float-float overlap
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
            dist = sqrtf(sh);
            if (fabsf(num) < kTinyNum) {
              const double d64 = exact_delta(C, C.c.slot[p], C.c.slot[j]);
              if (!(d64 > 0.0)) continue;
              del = (float)d64;
            } else {
              if (!(num > 0.f)) continue;
              del = __fdividef(num, __fadd_rn(Rh, dist));
            }
            ux = xh; uy = yh; uz = zh;
          }
          const float rr = __fdividef(__fmul_rn(o0.w, q.w), R);
          const float fn = __fsub_rn(__fmul_rn(kf, del), __fmul_rn(gf, sqrtf(__fmul_rn(rr, del))));
          nnz += (fn != 0.f);
          ++ovl;
          zeros += (fn == 0.f);
          if (dist > 0.f) {
            const float f = __fdividef(fn, dist);
            fx = __fmaf_rn(f, ux, fx);
            fy = __fmaf_rn(f, uy, fy);
            fz = __fmaf_rn(f, uz, fz);
          }
        }
      }
    }
  }
  C.c.f32[p] = make_float4(fx, fy, fz, (float)(ovl + 65536u * zeros));
  C.c.nnz[p] = (uint8_t)(nnz > 255u ? 255u : nnz);
}

// Direct loop with deferred pair evaluation.  The stencil walk only filters:
// a candidate that passes the FP32 filter is queued (cell index and
// neighbour-box code) in the thread's column of a shared-memory queue, and
// the queue is evaluated with pair32 after the walk.  The pair arithmetic,
// which the lanes of a warp would otherwise run one after another whenever
// any lane finds a partner, then runs with the lanes together, and the walk
// itself needs fewer registers.  An agent with more than kHitCap queued
// candidates is evaluated again by the plain direct loop.  Both evaluate the
// pairs in the walk's order.
constexpr int kHitCap = 16;  // deferred walk (full stencil)
constexpr int kSymCap = 8;   // symmetric walk (half stencil: about half the pairs)
template <int N>
struct HitQueueN {
  static constexpr int kCap = N;
  uint32_t j[N][kThreads];
  uint8_t b[N][kThreads];
};
using HitQueue = HitQueueN<kHitCap>;
using SymQueue = HitQueueN<kSymCap>;

// Evaluates the queued candidates in order; the agent's own cell, which the
// walk queues rather than test every candidate against it, is skipped here.
__device__ __forceinline__ void flush_hits(const DevCtx &C, uint32_t p, const float4 &o0, int n, const HitQueue &hq,
                                           float Lh, float Ll, float kf, float gf, float &fx, float &fy, float &fz,
                                           uint32_t &nnz, uint32_t &ovl) {
  const float4 o1 = C.c.r1[p];
  for (int k = 0; k < n; ++k) {
    const uint32_t j = hq.j[k][threadIdx.x];
    if (j == p) continue;
    const int b = hq.b[k][threadIdx.x];
    const float fdx = (float)(b % 3 - 1), fdy = (float)((b / 3) % 3 - 1), fdz = (float)(b / 9 - 1);
    if (pair32(C, (int64_t)p, o0, o1, (int64_t)j, C.c.r0[j], fdx, fdy, fdz, Lh, Ll, kf, gf, fx, fy, fz, nnz)) ++ovl;
  }
}

// kRowFlat: the three boxes of a stencil row are walked as one sequence
// (a warp then iterates max over lanes of the row's candidates rather than
// the sum over boxes of the per-box maxima).
template <bool kRowFlat>
__device__ __forceinline__ void force32_deferred(const DevCtx &C, const SimConst &sc, const SimState &s, uint32_t p,
                                                 int64_t cx, int64_t cy, int64_t cz, uint32_t stamp,
                                                 HitQueue &hq) {
  const float4 o0 = C.c.r0[p];
  const float Lh = s.Lh;
  const float rw = __fadd_rn(o0.w, s.marg);
  const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
  const float4 *__restrict__ r0 = C.c.r0;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  uint32_t nnz = 0;
  int n = 0;
  const float sxm = __fadd_rn(o0.x, Lh), sxp = __fsub_rn(o0.x, Lh);
  const bool x0 = t.xlo < 0, x2 = t.xhi > 0;
  for (int dz = t.zlo; dz <= t.zhi; ++dz) {
    const float sz = __fsub_rn(o0.z, __fmul_rn((float)dz, Lh));
    for (int dy = t.ylo; dy <= t.yhi; ++dy) {
      const float sy = __fsub_rn(o0.y, __fmul_rn((float)dy, Lh));
      const uint32_t row = ((uint32_t)(t.cz + dz) * (uint32_t)t.d1 + (uint32_t)(t.cy + dy)) * (uint32_t)t.d0 +
                           (uint32_t)t.cx;
      const unsigned long long ew[3] = {x0 ? __ldg(t.e + row - 1) : 0ull, __ldg(t.e + row),
                                        x2 ? __ldg(t.e + row + 1) : 0ull};
      const int code_row = (dz + 1) * 9 + (dy + 1) * 3;
      if constexpr (kRowFlat) {
        const uint32_t c0 = ent_live(ew[0], stamp), c1 = ent_live(ew[1], stamp), c2 = ent_live(ew[2], stamp);
        const uint32_t e01 = c0 + c1, tot = e01 + c2;
        const uint32_t jb0 = ent_start(ew[0]), jb1 = ent_start(ew[1]) - c0, jb2 = ent_start(ew[2]) - e01;
        for (uint32_t k = 0; k < tot; ++k) {
          const bool b0 = k < c0, b1 = k < e01;
          const uint32_t j = k + (b0 ? jb0 : (b1 ? jb1 : jb2));
          const float sx = b0 ? sxm : (b1 ? o0.x : sxp);
          const float4 qv = r0[j];
          const float ddx = __fsub_rn(sx, qv.x), ddy = __fsub_rn(sy, qv.y), ddz = __fsub_rn(sz, qv.z);
          const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
          const float Rm = __fadd_rn(rw, qv.w);
          if (!(s2 < __fmul_rn(Rm, Rm))) continue;
          if (n < kHitCap) {
            hq.j[n][threadIdx.x] = j;
            hq.b[n][threadIdx.x] = (uint8_t)(code_row + (b0 ? 0 : (b1 ? 1 : 2)));
          }
          ++n;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const uint32_t cnt = ent_live(ew[q], stamp);
          const uint32_t j0 = ent_start(ew[q]);
          const float sx = q == 0 ? sxm : (q == 1 ? o0.x : sxp);
          for (uint32_t j = j0; j < j0 + cnt; ++j) {
            const float4 qv = r0[j];
            const float ddx = __fsub_rn(sx, qv.x), ddy = __fsub_rn(sy, qv.y), ddz = __fsub_rn(sz, qv.z);
            const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
            const float Rm = __fadd_rn(rw, qv.w);
            if (!(s2 < __fmul_rn(Rm, Rm))) continue;
            if (n < kHitCap) {
              hq.j[n][threadIdx.x] = j;
              hq.b[n][threadIdx.x] = (uint8_t)(code_row + q);
            }
            ++n;
          }
        }
      }
    }
  }
  if (n > kHitCap) {
    force32(C, sc, s, (int64_t)p, cx, cy, cz, stamp);
    return;
  }
  uint32_t ovl = 0;
  flush_hits(C, p, o0, n, hq, Lh, s.Ll, sc.kf, sc.gammaf, fx, fy, fz, nnz, ovl);
  C.c.f32[p] = make_float4(fx, fy, fz, (float)(ovl + 65536u * (ovl - nnz)));
  C.c.nnz[p] = (uint8_t)(nnz > 255u ? 255u : nnz);
}

// Symmetric half-stencil walk (FP32 path, simulations without static
// detection).  Every interacting pair is found once: by the agent whose own
// box comes first in the order (z, y, x), or, inside one box, by the agent
// with the lower cell index.  The walk covers the agent's own box after its
// cell and the 13 neighbour boxes ahead of it (5 stencil rows instead of 9);
// the pair force goes to both agents, to the partner (and to the agent
// itself) by vector atomic adds onto forces the placement zeroed.  The w
// component counts the non-zero pair forces.  Candidates that pass the
// filter are queued as in the deferred walk; an agent with more than
// kSymCap of them evaluates its pairs during a second walk instead.
template <bool kQueue>
__device__ __forceinline__ uint32_t sym_walk(const DevCtx &C, const SimConst &sc, const SimState &s, uint32_t p,
                                             const float4 &o0, const Stencil &t, uint32_t stamp, SymQueue &hq,
                                             float &fx, float &fy, float &fz, float &cw) {
  const float Lh = s.Lh;
  const float rw = __fadd_rn(o0.w, s.marg);
  const float4 *__restrict__ r0 = C.c.r0;
  const float sxm = __fadd_rn(o0.x, Lh), sxp = __fsub_rn(o0.x, Lh);
  const bool x0 = t.xlo < 0, x2 = t.xhi > 0;
  float4 o1 = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (!kQueue) o1 = C.c.r1[p];
  uint32_t n = 0;
  for (int r = 0; r < 5; ++r) {
    const int dz = r < 2 ? 0 : 1;
    const int dy = r == 0 ? 0 : (r == 1 ? 1 : r - 3);
    if (dy < t.ylo || dy > t.yhi || dz > t.zhi) continue;
    const float sz = __fsub_rn(o0.z, __fmul_rn((float)dz, Lh));
    const float sy = __fsub_rn(o0.y, __fmul_rn((float)dy, Lh));
    const uint32_t row = ((uint32_t)(t.cz + dz) * (uint32_t)t.d1 + (uint32_t)(t.cy + dy)) * (uint32_t)t.d0 +
                         (uint32_t)t.cx;
    const int code_row = (dz + 1) * 9 + (dy + 1) * 3;
    // three segments A, B, C of candidates, walked as one sequence
    uint32_t cA, cB, cC, jA, jB, jC;
    float sA, sB, sC;
    int kA, kB, kC;
    if (r == 0) {
      const unsigned long long eo = __ldg(t.e + row);
      const unsigned long long ep = x2 ? __ldg(t.e + row + 1) : 0ull;
      // own box: the cells after p (none unless p lies in the box)
      const uint32_t os = ent_start(eo), oc = ent_live(eo, stamp);
      cA = (p >= os && p - os < oc) ? os + oc - (p + 1u) : 0u;
      jA = p + 1u; sA = o0.x; kA = code_row + 1;
      cB = ent_live(ep, stamp); jB = ent_start(ep); sB = sxp; kB = code_row + 2;
      cC = 0u; jC = 0u; sC = 0.f; kC = 0;
    } else {
      const unsigned long long em = x0 ? __ldg(t.e + row - 1) : 0ull;
      const unsigned long long eo = __ldg(t.e + row);
      const unsigned long long ep = x2 ? __ldg(t.e + row + 1) : 0ull;
      cA = ent_live(em, stamp); jA = ent_start(em); sA = sxm; kA = code_row;
      cB = ent_live(eo, stamp); jB = ent_start(eo); sB = o0.x; kB = code_row + 1;
      cC = ent_live(ep, stamp); jC = ent_start(ep); sC = sxp; kC = code_row + 2;
    }
    const uint32_t eAB = cA + cB, tot = eAB + cC;
    const uint32_t bA = jA, bB = jB - cA, bC = jC - eAB;
    for (uint32_t k = 0; k < tot; ++k) {
      const bool inA = k < cA, inB = k < eAB;
      const uint32_t j = k + (inA ? bA : (inB ? bB : bC));
      const float sx = inA ? sA : (inB ? sB : sC);
      const float4 qv = r0[j];
      const float ddx = __fsub_rn(sx, qv.x), ddy = __fsub_rn(sy, qv.y), ddz = __fsub_rn(sz, qv.z);
      const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
      const float Rm = __fadd_rn(rw, qv.w);
      if (!(s2 < __fmul_rn(Rm, Rm))) continue;
      const int code = inA ? kA : (inB ? kB : kC);
      if constexpr (kQueue) {
        if (n < (uint32_t)kSymCap) {
          hq.j[n][threadIdx.x] = j;
          hq.b[n][threadIdx.x] = (uint8_t)code;
        }
        ++n;
      } else {
        float gx, gy, gz;
        bool nz;
        const float fdx = (float)(code % 3 - 1), fdy = (float)((code / 3) % 3 - 1), fdz = (float)(code / 9 - 1);
        if (pair32_vec(C, (int64_t)p, o0, o1, (int64_t)j, qv, fdx, fdy, fdz, Lh, s.Ll, sc.kf, sc.gammaf, gx, gy,
                       gz, nz)) {
          fx = __fadd_rn(fx, gx); fy = __fadd_rn(fy, gy); fz = __fadd_rn(fz, gz);
          const float w = pair_count_word(nz);
          cw = __fadd_rn(cw, w);
          atomicAdd(&C.c.f32[j], make_float4(-gx, -gy, -gz, w));
        }
      }
    }
  }
  return n;
}

// Direct loop of the FP32 path (FP64-path simulations are left to the
// kernels of force64.cu).
__global__ void __launch_bounds__(kThreads, 4) k_force(DevCtx C) {
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid || sc.precision == BDM_PREC_FP64) return;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[p], cx, cy, cz);
  uint32_t stamp = C.g->stamp & kStampMask;
  bool st = is_static_cell(C, sc, s, p, cx, cy, cz, stamp);
  C.c.stat[p] = st ? 1 : 0;
  if (st) return;
  force32(C, sc, s, p, cx, cy, cz, stamp);
}

// FP32-path simulations only, deferred pair evaluation.
template <bool kRowFlat>
__global__ void __launch_bounds__(kThreads, 4) k_force32d(DevCtx C) {
  __shared__ HitQueue hq;
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid || sc.precision == BDM_PREC_FP64) return;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[p], cx, cy, cz);
  uint32_t stamp = C.g->stamp & kStampMask;
  bool st = is_static_cell(C, sc, s, p, cx, cy, cz, stamp);
  C.c.stat[p] = st ? 1 : 0;
  if (st) return;
  force32_deferred<kRowFlat>(C, sc, s, (uint32_t)p, cx, cy, cz, stamp, hq);
}

// FP32-path simulations only (none with static detection), symmetric
// half-stencil walk; the forces were zeroed by the placement.
// Warp-wide evaluation of the queued pairs: the lanes' queues are laid end
// to end and every lane takes one pair per round, so the warp runs
// ceil(total / 32) rounds instead of its longest queue.  A pair is added to
// its owner and, negated, to its partner by vector atomics.  mine: this
// lane's queue length (0 for a lane without queued pairs).
__device__ __forceinline__ void warp_flush(const DevCtx &C, const SymQueue &hq, uint32_t mine, int64_t p) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  uint32_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t excl = incl - mine;
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  const int64_t p0 = p - lane;  // cell of lane 0 (the warp's cells are consecutive)
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t k = base + (uint32_t)lane;
    // owner: the first lane whose inclusive prefix exceeds k
    int o = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const uint32_t v = __shfl_sync(FULL, incl, o + step - 1);
      if (v <= k) o += step;
    }
    const uint32_t ex = __shfl_sync(FULL, excl, o);
    if (k < total) {
      const uint32_t slot = k - ex;
      const uint32_t j = hq.j[slot][wbase + o];
      const int b = hq.b[slot][wbase + o];
      const int64_t po = p0 + o;
      const int so = C.c.sim[po];
      const SimConst &sco = C.sc[so];
      const SimState &sso = C.ss[so];
      const float4 a0 = C.c.r0[po], a1 = C.c.r1[po];
      const float fdx = (float)(b % 3 - 1), fdy = (float)((b / 3) % 3 - 1), fdz = (float)(b / 9 - 1);
      float gx, gy, gz;
      bool nz;
      if (pair32_vec(C, po, a0, a1, (int64_t)j, C.c.r0[j], fdx, fdy, fdz, sso.Lh, sso.Ll, sco.kf, sco.gammaf, gx,
                     gy, gz, nz)) {
        const float w = pair_count_word(nz);
        atomicAdd(&C.c.f32[po], make_float4(gx, gy, gz, w));
        atomicAdd(&C.c.f32[j], make_float4(-gx, -gy, -gz, w));
      }
    }
  }
}

// FP32-path simulations only (none with static detection), symmetric
// half-stencil walk; the forces were zeroed by the placement.  Queued pairs
// are evaluated warp-wide; an agent whose queue overflowed evaluates its
// pairs in a second walk.  kDirect: no queue, every pair evaluated in the
// walk (for crowded agents, whose queues would overflow).
template <bool kDirect>
__global__ void __launch_bounds__(kThreads, 4) k_force32s(DevCtx C) {
  __shared__ SymQueue hq;
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = p < C.g->n_cells;
  const int sim = active ? C.c.sim[p] : 0;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  active = active && s.valid && sc.precision != BDM_PREC_FP64;
  uint32_t mine = 0;
  if (active) {
    int64_t cx, cy, cz;
    unpack_coords(C.c.pkey[p], cx, cy, cz);
    C.c.stat[p] = 0;
    const uint32_t stamp = C.g->stamp & kStampMask;
    const float4 o0 = C.c.r0[p];
    const Stencil t = make_stencil(C, sc, s, cx, cy, cz);
    float fx = 0.f, fy = 0.f, fz = 0.f, cw = 0.f;
    const uint32_t n = kDirect ? (uint32_t)kSymCap + 1u
                               : sym_walk<true>(C, sc, s, (uint32_t)p, o0, t, stamp, hq, fx, fy, fz, cw);
    if (n > (uint32_t)kSymCap) {
      sym_walk<false>(C, sc, s, (uint32_t)p, o0, t, stamp, hq, fx, fy, fz, cw);
      atomicAdd(&C.c.f32[p], make_float4(fx, fy, fz, cw));
    } else {
      mine = n;
    }
  }
  if constexpr (!kDirect) warp_flush(C, hq, mine, p);
}

// S5: displacement, then the space boundary condition (§4.4.11) on the new
// position.  Static agents keep their position and nnz.  kOne: a context
// of one simulation (no per-cell simulation index to wait for).  kTrack:
// grid reuse: a moved agent's cell records follow it, relative to the box
// it is registered in (FP32 path: the float-float offset plus the FP32
// displacement; FP64 path and wall-clamped moves: recomputed as the
// placement computes them), and an agent that left its box by more than the
// build's skin on some axis makes the next iteration rebuild the grid.
template <bool kOne, bool kTrack>
__global__ void __launch_bounds__(kAgentThreads) k_displace(DevCtx C) {
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  int sim = kOne ? 0 : C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid) return;
  int32_t slot = C.c.slot[p];
  if (C.c.stat[p]) {
    C.a.flags[slot] = FLAG_STATIC;
    return;
  }
  const uint8_t ghost = C.a.flags[slot] & FLAG_GHOST;  // read-only: keeps its position
  const bool fp64 = sc.precision == BDM_PREC_FP64;
  bool moved = false, bad = false;
  double np[3] = {0.0, 0.0, 0.0};  // the new position of a moved agent
  float df[3] = {0.f, 0.f, 0.f};   // FP32 path: its displacement
  bool clamped = false;            // a wall cut the displacement short
  if (fp64) {
    C.a.nnz[slot] = C.c.nnz[p];
    const double4_32a F = C.c.f64[p];
    double Dx, Dy, Dz;
    moved = disp64(sc, F.x, F.y, F.z, Dx, Dy, Dz, bad) && !ghost;
    if (moved) {
      np[0] = bound_apply(sc, __dadd_rn(C.a.x[slot], Dx));
      np[1] = bound_apply(sc, __dadd_rn(C.a.y[slot], Dy));
      np[2] = bound_apply(sc, __dadd_rn(C.a.z[slot], Dz));
    }
  } else {
    float4 F = C.c.f32[p];
    // FP32 path: w carries the pair counts
    uint32_t ovl, nz;
    decode_counts(F.w, ovl, nz);
    C.a.nnz[slot] = (uint8_t)(nz > 255u ? 255u : nz);
    float f2 = __fmaf_rn(F.z, F.z, __fmaf_rn(F.y, F.y, __fmul_rn(F.x, F.x)));
    bad = !isfinite(f2);
    if (f2 > sc.adherence2f && !ghost) {
      float Dx = __fmul_rn(sc.dtf, F.x), Dy = __fmul_rn(sc.dtf, F.y), Dz = __fmul_rn(sc.dtf, F.z);
      float d2 = __fmaf_rn(Dz, Dz, __fmaf_rn(Dy, Dy, __fmul_rn(Dx, Dx)));
      if (d2 > sc.max_disp2f) {
        float f = __fmul_rn(sc.max_dispf, rsqrtf(d2));
        Dx = __fmul_rn(Dx, f); Dy = __fmul_rn(Dy, f); Dz = __fmul_rn(Dz, f);
      }
      moved = (Dx != 0.f || Dy != 0.f || Dz != 0.f);
      if (moved) {
        const double u[3] = {__dadd_rn(C.a.x[slot], f2d(Dx)), __dadd_rn(C.a.y[slot], f2d(Dy)),
                             __dadd_rn(C.a.z[slot], f2d(Dz))};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          np[a] = bound_apply(sc, u[a]);
          clamped = clamped || np[a] != u[a];
        }
        df[0] = Dx;
        df[1] = Dy;
        df[2] = Dz;
      }
    }
  }
  if (moved) {
    C.a.x[slot] = np[0];
    C.a.y[slot] = np[1];
    C.a.z[slot] = np[2];
    if (kTrack && !fp64 && !clamped) {
      // FP32 path: the float-float offset plus the FP32 displacement (no
      // FP64 operation: the FP64 pipe is the placement's limit); the
      // radius parts stay
      const float4 a0 = C.c.r0[p], a1 = C.c.r1[p];
      float h[3], l[3];
      ff_add_float(a0.x, a1.x, df[0], h[0], l[0]);
      ff_add_float(a0.y, a1.y, df[1], h[1], l[1]);
      ff_add_float(a0.z, a1.z, df[2], h[2], l[2]);
      bool out = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) out = out || !(h[a] >= s.skin_lo && h[a] < s.skin_hi);
      if (out) C.g->regrid = 1u;
      C.c.r0[p] = make_float4(h[0], h[1], h[2], a0.w);
      C.c.r1[p] = make_float4(l[0], l[1], l[2], a1.w);
    } else if (kTrack) {
      // FP64 path, or a displacement a wall cut short: the offset inside the
      // registered box as the placement computes it
      const uint64_t pk = C.c.pkey[p];
      const uint32_t c[3] = {(uint32_t)(pk & kCoordMask), (uint32_t)((pk >> kCoordBits) & kCoordMask),
                             (uint32_t)((pk >> (2 * kCoordBits)) & kCoordMask)};
      float h[3], l[3];
      bool out = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double w = __fma_rn(neg_u32_to_double(c[a]), s.L, __dsub_rn(np[a], s.o[a]));
        out = out || !(w >= -s.skin && w < __dadd_rn(s.L, s.skin));
        split_ff(w, h[a], l[a]);
      }
      if (out) C.g->regrid = 1u;
      const double r = half_of(C.a.d[slot]);
      float rh, rl;
      split_ff(r, rh, rl);
      C.c.r0[p] = make_float4(h[0], h[1], h[2], rh);
      if (fp64) C.c.r64[p] = make_double4_32a(np[0], np[1], np[2], r);
      else C.c.r1[p] = make_float4(l[0], l[1], l[2], rl);
    }
  }
  if (bad) set_err(C.g, ERR_NONFINITE);
  C.a.flags[slot] = (uint8_t)(ghost | (moved ? FLAG_CHANGED : 0));
}

static inline unsigned int blocks_for(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

// Variants of the FP32 path: 0 symmetric half stencil, 1 deferred walk with
// rows flattened, 2 direct loop, 3 deferred walk box by box.  FP64
// simulations always take the direct loop.
// Threads per block of the force kernels: kThreads, or fewer (down to one
// warp) for small populations, so that the blocks still cover the 152 SMs
// twice (the FP64 pipe of each SM is the limit of the FP64 path).
static inline int force_threads(int64_t n) {
  const int64_t want = (n + 2 * 152 - 1) / (2 * 152);
  int t = (int)((want + 31) / 32 * 32);
  return t < 32 ? 32 : (t > kThreads ? kThreads : t);
}

ForcePlan plan_force(int variant, bool any_static) {
  ForcePlan pl{variant, false};
  // the symmetric walks add pair forces to both agents: a static agent's
  // partner would miss them, so simulations with static detection take the
  // deferred walk instead of 0 and 4
  if ((variant == 0 || variant == 4) && any_static) pl.variant = 1;
  pl.zero_f32 = pl.variant == 0 || pl.variant == 4 || pl.variant == 6 || (pl.variant == 5 && !any_static);
  return pl;
}

void launch_force(const DevCtx &C, cudaStream_t st, int variant, bool has_fp32, bool has_fp64, bool any_static,
                  bool any_torus) {
  const int th = force_threads(C.total_slots);
  const unsigned int nb = blocks_for(C.total_slots, th);
  if (has_fp32) {
    if (variant == 2) k_force<<<nb, th, 0, st>>>(C);
    else if (variant == 0) k_force32s<false><<<nb, th, 0, st>>>(C);
    else if (variant == 4) k_force32s<true><<<nb, th, 0, st>>>(C);
    else if (variant == 3) k_force32d<false><<<nb, th, 0, st>>>(C);
    else if (variant == 5) launch_force_stream(C, st, any_static ? 1 : 0, th, any_torus);
    else if (variant == 6) launch_force_stream(C, st, any_static ? 2 : 0, th, any_torus);
    else k_force32d<true><<<nb, th, 0, st>>>(C);
  }
  if (has_fp64) launch_force64(C, st);
}

void launch_displace(const DevCtx &C, cudaStream_t st, bool track) {
  const unsigned int nb = blocks_for(C.total_slots, kAgentThreads);
  if (C.n_sims == 1) {
    if (track) k_displace<true, true><<<nb, kAgentThreads, 0, st>>>(C);
    else k_displace<true, false><<<nb, kAgentThreads, 0, st>>>(C);
  } else {
    if (track) k_displace<false, true><<<nb, kAgentThreads, 0, st>>>(C);
    else k_displace<false, false><<<nb, kAgentThreads, 0, st>>>(C);
  }
}

}  // namespace bdm
