// S4 force, FP32 path, staged variant (Eq 4.1 / Eq 4.2, §4.5.1): the
// default force kernel of the FP32 path.
//
// A warp owns 32 consecutive cells.  Because cells follow the Morton order
// of their boxes, those 32 agents occupy a compact block of boxes; the warp
// stages the table words and the FP32 records of that block plus its
// one-box halo in shared memory (two rounds of independent loads: table
// words, then records), and every lane then walks the candidates of its
// own 27-box stencil out of shared memory.  Warps whose region holds more
// than kRB boxes or kRK records -- a Morton segment that straddles a large
// power-of-two boundary, or very dense boxes -- read boxes and records from
// global memory instead.  Pairs that pass the FP32 filter are queued per
// warp (ballot + popc) and evaluated 32 at a time by the full warp with the
// float-float overlap, as in force32.cu; results are added to the owning
// lane's accumulator with shared-memory atomics.
#include "kernels.cuh"

namespace bdm {

constexpr int kST = 256;        // threads per block
constexpr int kSW = kST / 32;   // warps per block
constexpr int kRB = 216;        // staged region boxes per warp (6 x 6 x 6)
constexpr int kRK = 256;        // staged records per warp
constexpr int kSQ = 64;         // queue entries per warp
constexpr float kTinyNumS = 0x1p-19f;

struct WarpStage {
  uint16_t rcnt[kRB];
  uint16_t roff[kRB];
  uint32_t rstart[kRB];
  float4 rec[kRK];
  uint32_t ridx[kRK];
  uint2 q[kSQ];
  float4 own0[32], own1[32];
  float acc[4][32];
};

__device__ __forceinline__ void ffs_sub(float hi_i, float lo_i, float hi_j, float lo_j, float off_h, float off_l,
                                        float &dh, float &dl) {
  float s1, e1, s2, e2;
  two_sum(hi_i, -hi_j, s1, e1);
  two_sum(s1, -off_h, s2, e2);
  float l = __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(__fsub_rn(lo_i, lo_j), off_l));
  fast_two_sum(s2, l, dh, dl);
}

__device__ __noinline__ double exact_delta_s(const DevCtx &C, int32_t si, int32_t sj) {
  double dx = __dsub_rn(C.a.x[si], C.a.x[sj]);
  double dy = __dsub_rn(C.a.y[si], C.a.y[sj]);
  double dz = __dsub_rn(C.a.z[si], C.a.z[sj]);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double R = __dadd_rn(__dmul_rn(0.5, C.a.d[si]), __dmul_rn(0.5, C.a.d[sj]));
  return __dsub_rn(R, __dsqrt_rn(s));
}

// Queued pair (lane-parallel): float-float overlap and the force of Eq 4.1.
__device__ __forceinline__ void eval_queued(const DevCtx &C, WarpStage &W, uint2 qe, int64_t warp_p0) {
  const int owner = (int)(qe.y & 31u);
  const int code = (int)(qe.y >> 8);
  const uint32_t j = qe.x;
  const int sim = C.c.sim[warp_p0 + owner];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  const float Lh = s.Lh, Ll = s.Ll;
  float4 o0 = W.own0[owner], o1 = W.own1[owner];
  float4 q0 = C.c.r0[j], q1 = C.c.r1[j];
  float fdx = (float)(code % 3 - 1), fdy = (float)((code / 3) % 3 - 1), fdz = (float)(code / 9 - 1);
  float xh, xl, yh, yl, zh, zl;
  ffs_sub(o0.x, o1.x, q0.x, q1.x, __fmul_rn(fdx, Lh), __fmul_rn(fdx, Ll), xh, xl);
  ffs_sub(o0.y, o1.y, q0.y, q1.y, __fmul_rn(fdy, Lh), __fmul_rn(fdy, Ll), yh, yl);
  ffs_sub(o0.z, o1.z, q0.z, q1.z, __fmul_rn(fdz, Lh), __fmul_rn(fdz, Ll), zh, zl);
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
  float sl = __fadd_rn(__fadd_rn(Sea, Seb), __fadd_rn(__fadd_rn(e0, e1), e2));
  float sh, sll;
  fast_two_sum(Sb, sl, sh, sll);
  float Rh, Rl;
  two_sum(o0.w, q0.w, Rh, Rl);
  Rl = __fadd_rn(Rl, __fadd_rn(o1.w, q1.w));
  float Qh, Ql;
  two_prod(Rh, Rh, Qh, Ql);
  Ql = __fmaf_rn(__fmul_rn(2.f, Rh), Rl, Ql);
  float num = __fadd_rn(__fsub_rn(Qh, sh), __fsub_rn(Ql, sll));
  float dist = sqrtf(sh);
  float del;
  if (fabsf(num) < kTinyNumS) {
    double d64 = exact_delta_s(C, C.c.slot[warp_p0 + owner], C.c.slot[j]);
    if (!(d64 > 0.0)) return;
    del = (float)d64;
  } else {
    if (!(num > 0.f)) return;
    del = __fdividef(num, __fadd_rn(Rh, dist));
  }
  float rr = __fdividef(__fmul_rn(o0.w, q0.w), Rh);
  float fn = __fsub_rn(__fmul_rn(sc.kf, del), __fmul_rn(sc.gammaf, sqrtf(__fmul_rn(rr, del))));
  if (fn != 0.f) atomicAdd(&W.acc[3][owner], 1.0f);
  if (dist > 0.f) {
    float f = __fdividef(fn, dist);
    atomicAdd(&W.acc[0][owner], __fmul_rn(f, xh));
    atomicAdd(&W.acc[1][owner], __fmul_rn(f, yh));
    atomicAdd(&W.acc[2][owner], __fmul_rn(f, zh));
  }
}

__global__ void __launch_bounds__(kST, 3) k_force32s(DevCtx C) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpStage &W = reinterpret_cast<WarpStage *>(smem_raw)[warp];
  const int64_t warp_p0 = (int64_t)blockIdx.x * kST + warp * 32;
  const int64_t p = warp_p0 + lane;
  const int64_t ncell = C.g->n_cells;
  const uint32_t stamp = C.g->stamp;
  bool active = p < ncell;
  const int sim = active ? C.c.sim[p] : 0;
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (active && (!s.valid || sc.precision != BDM_PREC_FP32_FORCE)) active = false;
  int64_t cx = 0, cy = 0, cz = 0;
  if (active) {
    unpack_coords(C.c.pkey[p], cx, cy, cz);
    bool st = is_static_cell(C, sc, s, p, cx, cy, cz, stamp);
    C.c.stat[p] = st ? 1 : 0;
    if (st) active = false;
  }
  float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
  if (active) {
    o0 = C.c.r0[p];
    o1 = C.c.r1[p];
  }
  W.own0[lane] = o0;
  W.own1[lane] = o1;
  W.acc[0][lane] = 0.f; W.acc[1][lane] = 0.f; W.acc[2][lane] = 0.f; W.acc[3][lane] = 0.f;
  const unsigned FULL = 0xffffffffu;
  if (!__any_sync(FULL, active)) return;

  // Region of the warp: box bounding box of its active lanes plus one box.
  const unsigned smin = __reduce_min_sync(FULL, active ? (unsigned)sim : 0xFFFFFFFFu);
  const unsigned smax = __reduce_max_sync(FULL, active ? (unsigned)sim : 0u);
  const bool uniform = smin == smax;
  const SimState &su = C.ss[smin];
  const SimConst &scu = C.sc[smin];
  const unsigned lx = __reduce_min_sync(FULL, active ? (unsigned)cx : 0xFFFFFFFFu);
  const unsigned ly = __reduce_min_sync(FULL, active ? (unsigned)cy : 0xFFFFFFFFu);
  const unsigned lz = __reduce_min_sync(FULL, active ? (unsigned)cz : 0xFFFFFFFFu);
  const unsigned hx = __reduce_max_sync(FULL, active ? (unsigned)cx : 0u);
  const unsigned hy = __reduce_max_sync(FULL, active ? (unsigned)cy : 0u);
  const unsigned hz = __reduce_max_sync(FULL, active ? (unsigned)cz : 0u);
  const int64_t lox = lx > 0 ? lx - 1 : 0, loy = ly > 0 ? ly - 1 : 0, loz = lz > 0 ? lz - 1 : 0;
  const int64_t hix = (int64_t)hx + 1 < su.dims[0] ? hx + 1 : su.dims[0] - 1;
  const int64_t hiy = (int64_t)hy + 1 < su.dims[1] ? hy + 1 : su.dims[1] - 1;
  const int64_t hiz = (int64_t)hz + 1 < su.dims[2] ? hz + 1 : su.dims[2] - 1;
  const int rx = (int)(hix - lox + 1), ry = (int)(hiy - loy + 1), rz = (int)(hiz - loz + 1);
  const int64_t V = (int64_t)rx * ry * rz;
  bool staged = uniform && V <= kRB;
  if (staged) {
    // round 1: table words of every box of the region
    bool over = false;
    for (int b = lane; b < (int)V; b += 32) {
      const int64_t bx = lox + b % rx, by = loy + (b / rx) % ry, bz = loz + b / (rx * ry);
      const int64_t idx = scu.table_base + bx + su.dims[0] * (by + su.dims[1] * bz);
      unsigned long long e = C.tab.cnt[idx];
      uint32_t c = ((uint32_t)(e >> 32) == stamp) ? (uint32_t)(e & 0x7FFFFFFFull) : 0u;
      if (c > 0xFFFFu) { over = true; c = 0; }
      W.rcnt[b] = (uint16_t)c;
      W.rstart[b] = c ? C.tab.start[idx] : 0u;
    }
    __syncwarp();
    // prefix of the counts
    uint32_t run = 0;
    for (int base = 0; base < (int)V; base += 32) {
      const int b = base + lane;
      const uint32_t c = b < (int)V ? W.rcnt[b] : 0u;
      uint32_t inc = c;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
      }
      if (b < (int)V) W.roff[b] = (uint16_t)((run + inc - c) & 0xFFFFu);
      run += __shfl_sync(FULL, inc, 31);
    }
    staged = !__any_sync(FULL, over) && run <= (uint32_t)kRK;
    if (staged) {
      __syncwarp();
      // round 2: records of the region
      for (int b = lane; b < (int)V; b += 32) {
        const uint32_t c = W.rcnt[b], o = W.roff[b], st0 = W.rstart[b];
        for (uint32_t k = 0; k < c; ++k) {
          W.rec[o + k] = C.c.r0[st0 + k];
          W.ridx[o + k] = st0 + k;
        }
      }
    }
    __syncwarp();
  }

  // Candidate loop: one candidate per lane and step, box after box.
  const float Lh = active ? s.Lh : 0.f, marg = active ? s.marg : 0.f;
  const int64_t d0 = s.dims[0], d1 = s.dims[1], d2 = s.dims[2];
  int box = 0;                 // next stencil box (0..27)
  uint32_t k = 0, kend = 0;    // staged: record range; global: cell range
  int code = 13;
  float sx = o0.x, sy = o0.y, sz = o0.z;
  int qn = 0;
  const unsigned lt = (1u << lane) - 1u;
  while (true) {
    bool have = false;
    if (active) {
      while (k == kend && box < 27) {
        const int dx = box % 3 - 1, dy = (box / 3) % 3 - 1, dz = box / 9 - 1;
        const int64_t x = cx + dx, y = cy + dy, z = cz + dz;
        const int bcode = box;
        ++box;
        if (x < 0 || y < 0 || z < 0 || x >= d0 || y >= d1 || z >= d2) continue;
        if (staged) {
          const int lb = (int)((x - lox) + rx * ((y - loy) + (int64_t)ry * (z - loz)));
          k = W.roff[lb];
          kend = k + W.rcnt[lb];
        } else {
          const int64_t idx = sc.table_base + x + d0 * (y + d1 * z);
          unsigned long long e = C.tab.cnt[idx];
          uint32_t c = ((uint32_t)(e >> 32) == stamp) ? (uint32_t)(e & 0x7FFFFFFFull) : 0u;
          k = c ? C.tab.start[idx] : 0u;
          kend = k + c;
        }
        code = bcode;
        sx = __fsub_rn(o0.x, __fmul_rn((float)dx, Lh));
        sy = __fsub_rn(o0.y, __fmul_rn((float)dy, Lh));
        sz = __fsub_rn(o0.z, __fmul_rn((float)dz, Lh));
      }
      have = k < kend;
    }
    if (!__any_sync(FULL, have)) break;
    bool hit = false;
    uint32_t cell = 0;
    if (have) {
      float4 q;
      if (staged) {
        q = W.rec[k];
        cell = W.ridx[k];
      } else {
        cell = k;
        q = C.c.r0[k];
      }
      ++k;
      if ((int64_t)cell != p) {
        float ddx = __fsub_rn(sx, q.x), ddy = __fsub_rn(sy, q.y), ddz = __fsub_rn(sz, q.z);
        float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
        float Rm = __fadd_rn(__fadd_rn(o0.w, q.w), marg);
        hit = s2 < __fmul_rn(Rm, Rm);
      }
    }
    const unsigned bal = __ballot_sync(FULL, hit);
    if (bal) {
      if (hit) W.q[qn + __popc(bal & lt)] = make_uint2(cell, (uint32_t)lane | ((uint32_t)code << 8));
      qn += __popc(bal);
      if (qn >= 32) {
        __syncwarp();
        eval_queued(C, W, W.q[lane], warp_p0);
        __syncwarp();
        if (lane < qn - 32) W.q[lane] = W.q[32 + lane];
        __syncwarp();
        qn -= 32;
      }
    }
  }
  __syncwarp();
  if (lane < qn) eval_queued(C, W, W.q[lane], warp_p0);
  __syncwarp();
  if (active) {
    C.c.f32[p] = make_float4(W.acc[0][lane], W.acc[1][lane], W.acc[2][lane], 0.f);
    const float nz = W.acc[3][lane];
    C.c.nnz[p] = (uint8_t)(nz > 255.f ? 255u : (unsigned)nz);
  }
}

void launch_force32s(const DevCtx &C, cudaStream_t st) {
  const size_t smem = sizeof(WarpStage) * kSW;
  cudaFuncSetAttribute(k_force32s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  unsigned int nb = (unsigned int)((C.total_slots + kST - 1) / kST);
  k_force32s<<<nb, kST, smem, st>>>(C);
}

}  // namespace bdm
