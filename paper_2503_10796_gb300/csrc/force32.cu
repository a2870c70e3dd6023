// S4 force, FP32 path, queue variant (Eq 4.1 / Eq 4.2, §4.5.1).
//
// One thread per agent (cell order, so a warp holds 32 neighbours along
// the Morton curve):
//   1. the 27 stencil boxes' table words are loaded together (one latency)
//      and the non-empty boxes are kept in shared memory;
//   2. one flattened loop walks the agent's candidates box after box, so the
//      lanes of a warp stay busy whatever the per-box counts are; each step
//      is the cheap FP32 filter on box-relative coordinates;
//   3. pairs that pass the filter are appended to a per-warp queue
//      (ballot + popc); whenever 32 are queued, the whole warp evaluates them
//      -- float-float overlap, force of Eq 4.1 -- and adds the result to the
//      owning lane's accumulator with shared-memory atomics.
// The arithmetic per pair is that of the reference kernel in force.cu.
#include "kernels.cuh"

namespace bdm {

constexpr int kFT = 256;          // threads per block
constexpr int kFW = kFT / 32;     // warps per block
constexpr int kQCap = 64;         // queue entries per warp
constexpr float kTinyNum32 = 0x1p-19f;

struct Force32Smem {
  uint2 ent[27 * kFT];            // per thread: (first cell, count | code << 24)
  float4 own0[kFT], own1[kFT];    // the thread's own record
  float acc[4][kFT];              // force x, y, z and nnz count per thread
  uint2 q[kFW][kQCap];            // queued pairs: (candidate cell, owner lane | code << 8)
};

__device__ __forceinline__ void ff_sub(float hi_i, float lo_i, float hi_j, float lo_j, float off_h, float off_l,
                                       float &dh, float &dl) {
  float s1, e1, s2, e2;
  two_sum(hi_i, -hi_j, s1, e1);
  two_sum(s1, -off_h, s2, e2);
  float l = __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(__fsub_rn(lo_i, lo_j), off_l));
  fast_two_sum(s2, l, dh, dl);
}

__device__ __noinline__ double exact_delta32(const DevCtx &C, int32_t si, int32_t sj) {
  double dx = __dsub_rn(C.a.x[si], C.a.x[sj]);
  double dy = __dsub_rn(C.a.y[si], C.a.y[sj]);
  double dz = __dsub_rn(C.a.z[si], C.a.z[sj]);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double R = __dadd_rn(__dmul_rn(0.5, C.a.d[si]), __dmul_rn(0.5, C.a.d[sj]));
  return __dsub_rn(R, __dsqrt_rn(s));
}

// Evaluate one queued pair (lane-parallel): owner lane's record from shared
// memory, candidate record from global memory.
__device__ __forceinline__ void eval_pair(const DevCtx &C, Force32Smem &S, int warp, uint2 qe, float Lh, float Ll,
                                          float kf, float gf, int64_t block_p0) {
  int owner = (int)(qe.y & 31u);
  int code = (int)(qe.y >> 8);
  uint32_t j = qe.x;
  int t = warp * 32 + owner;
  float4 o0 = S.own0[t], o1 = S.own1[t];
  float4 q0 = C.c.r0[j], q1 = C.c.r1[j];
  float fdx = (float)(code % 3 - 1), fdy = (float)((code / 3) % 3 - 1), fdz = (float)(code / 9 - 1);
  float xh, xl, yh, yl, zh, zl;
  ff_sub(o0.x, o1.x, q0.x, q1.x, __fmul_rn(fdx, Lh), __fmul_rn(fdx, Ll), xh, xl);
  ff_sub(o0.y, o1.y, q0.y, q1.y, __fmul_rn(fdy, Lh), __fmul_rn(fdy, Ll), yh, yl);
  ff_sub(o0.z, o1.z, q0.z, q1.z, __fmul_rn(fdz, Lh), __fmul_rn(fdz, Ll), zh, zl);
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
  if (fabsf(num) < kTinyNum32) {
    double d64 = exact_delta32(C, C.c.slot[block_p0 + t], C.c.slot[j]);
    if (!(d64 > 0.0)) return;
    del = (float)d64;
  } else {
    if (!(num > 0.f)) return;
    del = __fdividef(num, __fadd_rn(Rh, dist));
  }
  float rr = __fdividef(__fmul_rn(o0.w, q0.w), Rh);
  float fn = __fsub_rn(__fmul_rn(kf, del), __fmul_rn(gf, sqrtf(__fmul_rn(rr, del))));
  if (fn != 0.f) atomicAdd(&S.acc[3][t], 1.0f);
  if (dist > 0.f) {
    float sc_ = __fdividef(fn, dist);
    atomicAdd(&S.acc[0][t], __fmul_rn(sc_, xh));
    atomicAdd(&S.acc[1][t], __fmul_rn(sc_, yh));
    atomicAdd(&S.acc[2][t], __fmul_rn(sc_, zh));
  }
}

__global__ void __launch_bounds__(kFT, 3) k_force32q(DevCtx C) {
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Force32Smem &S = *reinterpret_cast<Force32Smem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p0 = (int64_t)blockIdx.x * kFT;
  const int64_t p = p0 + tid;
  const int64_t ncell = C.g->n_cells;
  const uint32_t stamp = C.g->stamp & kStampMask;
  bool active = p < ncell;
  int sim = active ? C.c.sim[p] : 0;
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
  S.own0[tid] = o0;
  S.own1[tid] = o1;
  S.acc[0][tid] = 0.f; S.acc[1][tid] = 0.f; S.acc[2][tid] = 0.f; S.acc[3][tid] = 0.f;
  const float Lh = active ? s.Lh : 0.f, Ll = active ? s.Ll : 0.f, marg = active ? s.marg : 0.f;
  // phase 1: stencil boxes
  int m = 0;
  if (active) {
    const int64_t d0 = s.dims[0], d1 = s.dims[1], d2 = s.dims[2];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int64_t y = cy + dy, z = cz + dz;
        const bool rowok = y >= 0 && y < d1 && z >= 0 && z < d2;
        const int64_t row = sc.table_base + cx + d0 * (y + d1 * z);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int64_t x = cx + dx;
          if (rowok && x >= 0 && x < d0) {
            const unsigned long long e = C.tab.e[row + dx];
            uint32_t cnt = ent_live(e, stamp);
            if (cnt) {
              uint32_t st0 = ent_start(e);
              const int code = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
              S.ent[m * kFT + tid] = make_uint2(st0, (cnt & 0xFFFFFFu) | ((uint32_t)code << 24));
              ++m;
            }
          }
        }
      }
    }
  }
  // phase 2: flattened candidate loop with the survivor queue
  const float kf = active ? sc.kf : 0.f, gf = active ? sc.gammaf : 0.f;
  // the queue's pair evaluation needs each sim's own constants; lanes of one
  // warp may belong to different simulations, so the evaluator reads them
  // from the owner's simulation
  int e = 0;
  uint32_t j = 0, jend = 0;
  int code = 13;
  float sx = o0.x, sy = o0.y, sz = o0.z;
  int qn = 0;
  const unsigned lt = (1u << lane) - 1u;
  __syncwarp();
  while (true) {
    bool have = false;
    if (j < jend) {
      have = true;
    } else if (e < m) {
      uint2 en = S.ent[e * kFT + tid];
      ++e;
      j = en.x;
      jend = en.x + (en.y & 0xFFFFFFu);
      code = (int)(en.y >> 24);
      const float fdx = (float)(code % 3 - 1), fdy = (float)((code / 3) % 3 - 1), fdz = (float)(code / 9 - 1);
      sx = __fsub_rn(o0.x, __fmul_rn(fdx, Lh));
      sy = __fsub_rn(o0.y, __fmul_rn(fdy, Lh));
      sz = __fsub_rn(o0.z, __fmul_rn(fdz, Lh));
      have = true;
    }
    if (!__any_sync(0xffffffffu, have)) break;
    bool hit = false;
    uint32_t jc = j;
    if (have) {
      ++j;
      if ((int64_t)jc != p) {
        const float4 q = C.c.r0[jc];
        float ddx = __fsub_rn(sx, q.x), ddy = __fsub_rn(sy, q.y), ddz = __fsub_rn(sz, q.z);
        float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
        float Rm = __fadd_rn(__fadd_rn(o0.w, q.w), marg);
        hit = s2 < __fmul_rn(Rm, Rm);
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, hit);
    if (b) {
      if (hit) S.q[warp][qn + __popc(b & lt)] = make_uint2(jc, (uint32_t)lane | ((uint32_t)code << 8));
      qn += __popc(b);
      if (qn >= 32) {
        __syncwarp();
        uint2 qe = S.q[warp][lane];
        int ow = (int)(qe.y & 31u);
        const SimConst &so = C.sc[C.c.sim[p0 + warp * 32 + ow]];
        const SimState &ss = C.ss[C.c.sim[p0 + warp * 32 + ow]];
        eval_pair(C, S, warp, qe, ss.Lh, ss.Ll, so.kf, so.gammaf, p0);
        __syncwarp();
        if (lane < qn - 32) S.q[warp][lane] = S.q[warp][32 + lane];
        __syncwarp();
        qn -= 32;
      }
    }
  }
  __syncwarp();
  if (lane < qn) {
    uint2 qe = S.q[warp][lane];
    int ow = (int)(qe.y & 31u);
    const SimConst &so = C.sc[C.c.sim[p0 + warp * 32 + ow]];
    const SimState &ss = C.ss[C.c.sim[p0 + warp * 32 + ow]];
    eval_pair(C, S, warp, qe, ss.Lh, ss.Ll, so.kf, so.gammaf, p0);
  }
  __syncwarp();
  if (active) {
    float nz = S.acc[3][tid];
    C.c.f32[p] = make_float4(S.acc[0][tid], S.acc[1][tid], S.acc[2][tid], nz);
    C.c.nnz[p] = (uint8_t)(nz > 255.f ? 255u : (unsigned)nz);
  }
  (void)kf;
  (void)gf;
}

size_t force32q_smem() { return sizeof(Force32Smem); }

void launch_force32q(const DevCtx &C, cudaStream_t st) {
  cudaFuncSetAttribute(k_force32q, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Force32Smem));
  unsigned int nb = (unsigned int)((C.total_slots + kFT - 1) / kFT);
  k_force32q<<<nb, kFT, sizeof(Force32Smem), st>>>(C);
}

}  // namespace bdm
