// S4 force of the FP32 path as a warp candidate stream (Eq 4.1 / Eq 4.2).
//
// A warp takes 32 consecutive cells (cells are grouped by box, boxes in the
// storage's Morton order, so the 32 agents are close in space).  Each lane
// lists, as segments of consecutive cells, the non-empty boxes of its
// stencil that its sphere can reach: a box whose distance from the centre
// is at least r_own + r_max (the largest radius of the iteration) holds no
// partner, because a pair interacts only below the distance r_i + r_j.  The
// warp lays the lanes' segments end to end and tests the candidates 32 at a
// time, one per lane, so that no lane idles while another walks a crowded
// box.  Candidates that pass the FP32 filter (the one of the other force
// kernels) go to a warp queue of pairs, evaluated 32 at a time with the
// float-float pair arithmetic, which decides every pair exactly.  The
// stencil and candidate loops are written without branches (every lane
// loads from an address that is valid for it, and masks the result): on
// this part a branch around a load costs more issue slots than the load.
//
// Modes:
//   kSym   half stencil: the own box after the own cell and the 13 boxes
//          ahead in (z, y, x) order, so every pair is found once; its force
//          goes to the owner (a shared-memory sum) and, negated, to the
//          partner (a vector atomic onto forces the placement zeroed);
//   kFull  the full stencil and only the owner's force, for simulations
//          that detect static agents (static agents walk nothing).
// The static-mask mode of the engine runs kSym after k_static, which wrote
// the static flags: static agents' forces are then computed but unused
// (k_displace keeps them in place), which is exact because the oracle's
// static rules never let a static agent move.
//
// Segment lookup.  Segment s covers candidates [off_s, off_s + n_s) of the
// warp's sequence.  For the round of candidates [base, base + 32), the warp
// holds cur, the segment of candidate `base`; lane k reads the first
// candidate of segment cur + 1 + k, and the OR over lanes of 1 << (that -
// base), for those inside the round, marks where segments start.  A lane's
// segment is then cur plus the number of starts at or below its position.
// Segments are never empty, so at most 32 of them start in one round and
// all are among the 32 read.
#include "pair.cuh"

namespace bdm {

constexpr int kStreamWarps = 8;              // warps per block
constexpr int kStreamThreads = 32 * kStreamWarps;
constexpr int kPhaseBoxes = 9;               // stencil boxes per lane and phase (three rows)
constexpr int kSegCap = 32 * kPhaseBoxes;    // segments per warp and phase
constexpr int kPairCap = 64;                 // queued pairs per warp (flushed at 32)
constexpr uint32_t kOffMask = (1u << 21) - 1u;

struct StreamShared {
  uint2 seg[kStreamWarps][kSegCap];    // {first cell, candidate offset | owner << 21 | code << 26}
  uint2 pq[kStreamWarps][kPairCap];    // queued pairs {cell j, owner | code << 5}
  float4 acc[kStreamWarps][32];        // owner force and pair-count word
  float4 r0[kStreamWarps][32];         // owner records: leading parts (box-relative centre, radius)
  float4 r1[kStreamWarps][32];         //                trailing parts
  float4 kc[kStreamWarps][32];         // owner simulation: L (leading, trailing), k, gamma
  float rw[kStreamWarps][32];          // owner radius plus the filter margin
};

enum : int { kModeSym = 0, kModeFull = 1, kModeSymMasked = 2 };

// Stencil row r of a mode as offsets (dy, dz) and the first x offset x0 of
// the row (the row covers x0 .. +1): kSym rows 0 (own box and x + 1), 1
// (y + 1), 2-4 (z + 1, y - 1 .. y + 1); full rows 0-8 (dz, dy) in (z, y)
// order, each x - 1 .. x + 1 (the own box among them).
template <bool kSym>
__device__ __forceinline__ void stream_row(int r, int &dy, int &dz, int &x0) {
  if (kSym) {
    if (r == 0) { dy = 0; dz = 0; x0 = 0; }
    else if (r == 1) { dy = 1; dz = 0; x0 = -1; }
    else { dy = r - 3; dz = 1; x0 = -1; }
  } else {
    dy = r % 3 - 1; dz = r / 3 - 1; x0 = -1;
  }
}

// Evaluates the first k queued pairs (one per lane) after moving the
// entries beyond the first k (qn in all) down to the front.
template <bool kSym>
__device__ __forceinline__ void stream_flush(const DevCtx &C, StreamShared &sh, int wid, int lane, int64_t p0,
                                             uint32_t qn, uint32_t k) {
  __syncwarp();
  const uint32_t rest = qn - k;
  const uint2 e = sh.pq[wid][lane];
  const uint2 mv = sh.pq[wid][(k + (uint32_t)lane) & (kPairCap - 1)];
  __syncwarp();
  if ((uint32_t)lane < rest) sh.pq[wid][lane] = mv;
  if ((uint32_t)lane < k) {
    const uint32_t j = e.x;
    const int o = (int)(e.y & 31u), code = (int)(e.y >> 5);
    const int64_t po = p0 + o;
    const float4 a0 = sh.r0[wid][o], a1 = sh.r1[wid][o], kc = sh.kc[wid][o];
    const float fdx = (float)(code & 3) - 1.f, fdy = (float)((code >> 2) & 3) - 1.f, fdz = (float)(code >> 4) - 1.f;
    float gx, gy, gz;
    bool nz;
    if (pair32_lite(C, po, a0, a1, (int64_t)j, fdx, fdy, fdz, kc.x, kc.y, kc.z, kc.w, gx, gy, gz, nz)) {
      const float w = pair_count_word(nz);
      float4 &a = sh.acc[wid][o];
      atomicAdd(&a.x, gx);
      atomicAdd(&a.y, gy);
      atomicAdd(&a.z, gz);
      atomicAdd(&a.w, w);
      if (kSym) atomicAdd(&C.c.f32[j], make_float4(-gx, -gy, -gz, w));
    }
  }
  __syncwarp();
}

// kTorus: some simulation of the launch is toroidal (stencil boxes wrap).
// kOne: the context holds one simulation (its constants need no per-cell
// simulation index, which would be the first load every later one waits on).
template <int kMode, bool kTorus, bool kOne>
__global__ void __launch_bounds__(kStreamThreads, 4) k_force32w(DevCtx C) {
  constexpr bool kSym = kMode != kModeFull;
  constexpr int kRows = kSym ? 5 : 9;
  constexpr int kPhases = (kRows + 2) / 3;   // three rows per phase
  __shared__ StreamShared sh;
  if (C.g->err & ERR_TABLE) return;  // boxes of this build emptied: cells not placed
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t p0 = (int64_t)blockIdx.x * blockDim.x + (wid << 5);  // first cell of the warp
  const int64_t ncell = C.g->n_cells;
  if (p0 >= ncell) return;  // the whole warp
  const int64_t p = p0 + lane;
  bool active = p < ncell;
  const int64_t pc = active ? p : p0;  // a valid cell for every lane
  const int sim = kOne ? 0 : C.c.sim[pc];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  active = active && s.valid && sc.precision != BDM_PREC_FP64;
  const uint32_t stamp = C.g->stamp & kStampMask;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[pc], cx, cy, cz);
  const float4 o0 = C.c.r0[pc];
  const float4 o1 = C.c.r1[pc];
  bool walk = active;
  if (kMode == kModeFull) {
    const bool st = active && is_static_cell(C, sc, s, p, cx, cy, cz, stamp);
    if (active) C.c.stat[p] = st ? 1 : 0;
    walk = active && !st;
  } else if (kMode == kModeSym) {
    if (active) C.c.stat[p] = 0;
  }
  const float Lh = s.Lh;
  const float rw = __fadd_rn(o0.w, s.marg);  // own radius plus the filter margin
  sh.acc[wid][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  sh.r0[wid][lane] = o0;
  sh.r1[wid][lane] = o1;
  sh.kc[wid][lane] = make_float4(Lh, s.Ll, sc.kf, sc.gammaf);
  sh.rw[wid][lane] = rw;
  const uint32_t lm_le = FULL >> (31 - lane), lm_lt = lm_le >> 1;  // lanes at or below / below this one
  const Stencil t = make_stencil<kTorus>(C, sc, s, cx, cy, cz);
  const uint32_t row0 = ((uint32_t)t.cz * (uint32_t)t.d1 + (uint32_t)t.cy) * (uint32_t)t.d0 + (uint32_t)t.cx;
  // the word every lane may load when it has no box to read: its own box's
  // (placed in a valid grid), else the table's first word
  const unsigned long long *const e_idle = walk ? t.e + row0 : C.tab.e;
  // box pruning: squared distance from the centre to the neighbour box per
  // axis and offset (-1: max(w, 0), 0: 0, +1: max(L - w, 0)); reach = rw +
  // r_max, plus the skin in iterations that keep the last build's grid (a
  // partner registered in a box may then lie up to the skin outside it)
  const float reach = __fadd_rn(__fadd_rn(rw, s.rmaxf), C.g->reuse ? s.skin_pad : 0.f);
  const float reach2 = __fmul_rn(reach, reach);
  const float wx = fmaxf(o0.x, 0.f), wy = fmaxf(o0.y, 0.f), wz = fmaxf(o0.z, 0.f);
  const float lx = fmaxf(__fsub_rn(Lh, o0.x), 0.f), ly = fmaxf(__fsub_rn(Lh, o0.y), 0.f),
              lz = fmaxf(__fsub_rn(Lh, o0.z), 0.f);
  const float ex[3] = {__fmul_rn(wx, wx), 0.f, __fmul_rn(lx, lx)};
  const float ey[3] = {__fmul_rn(wy, wy), 0.f, __fmul_rn(ly, ly)};
  const float ez[3] = {__fmul_rn(wz, wz), 0.f, __fmul_rn(lz, lz)};
  uint32_t qn = 0;  // queued pairs (warp-uniform)
  __syncwarp();
#pragma unroll
  for (int ph = 0; ph < kPhases; ++ph) {
    // this lane's boxes of the phase: first cell and candidate count
    uint32_t sj[kPhaseBoxes], sn[kPhaseBoxes];
    uint32_t nseg = 0u, ncand = 0u;
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) {
      const int r = ph * 3 + rr;
      int dy = 0, dz = 0, x0 = 0;
      if (r < kRows) stream_row<kSym>(r, dy, dz, x0);
      const bool inrow = r < kRows && walk && dy >= t.ylo && dy <= t.yhi && dz >= t.zlo && dz <= t.zhi;
      const uint32_t rowb = row0 + (uint32_t)(dz * t.d1 + dy) * (uint32_t)t.d0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int dx = x0 + q;
        const int slot = rr * 3 + q;
        sj[slot] = 0u;
        sn[slot] = 0u;
        if (dx > 1 || r >= kRows) continue;  // compile-time
        const bool own = dx == 0 && dy == 0 && dz == 0;
        const float d2 = __fadd_rn(__fadd_rn(ex[dx + 1], ey[dy + 1]), ez[dz + 1]);
        const bool use = inrow && dx >= t.xlo && dx <= t.xhi && (own || !(d2 > reach2));
        const uint32_t bi = (kTorus && t.torus) ? t.box(dx, dy, dz) : rowb + dx;
        const unsigned long long e = __ldg(use ? t.e + bi : e_idle);
        const uint32_t es = ent_start(e), ec = use ? ent_live(e, stamp) : 0u;
        uint32_t j0 = es, cnt = ec;
        if (own && kSym) {
          // cells after the own one (none unless the own cell lies in the box)
          const uint32_t pp = (uint32_t)p;
          cnt = (pp >= es && pp - es < ec) ? es + ec - (pp + 1u) : 0u;
          j0 = pp + 1u;
        }
        sj[slot] = j0;
        sn[slot] = cnt;
        nseg += cnt ? 1u : 0u;
        ncand += cnt;
      }
    }
    // lay the lanes' segments end to end: (candidates << 9 | segments)
    const uint32_t v = (ncand << 9) | nseg;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, incl, d);
      incl += lane >= d ? y : 0u;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    const uint32_t T = tot >> 9, NS = tot & 511u;
    {
      const uint32_t ex0 = incl - v;
      uint32_t pos = ex0 & 511u, off = ex0 >> 9;
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        const int r = ph * 3 + rr;
        if (r >= kRows) continue;
        int dy, dz, x0;
        stream_row<kSym>(r, dy, dz, x0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int dx = x0 + q;
          const int slot = rr * 3 + q;
          if (dx > 1) continue;
          const uint32_t code = (uint32_t)(dx + 1) | ((uint32_t)(dy + 1) << 2) | ((uint32_t)(dz + 1) << 4);
          if (sn[slot]) sh.seg[wid][pos] = make_uint2(sj[slot], off | ((uint32_t)lane << 21) | (code << 26));
          pos += sn[slot] ? 1u : 0u;
          off += sn[slot];
        }
      }
    }
    __syncwarp();
    uint32_t cur = 0u;  // segment of candidate `base`
    const uint32_t last = NS ? NS - 1u : 0u;
    for (uint32_t base = 0u; base < T; base += 32u) {
      const uint32_t idx = cur + 1u + (uint32_t)lane;
      const uint32_t d = (sh.seg[wid][idx < NS ? idx : last].y & kOffMask) - base;
      const uint32_t M = __reduce_or_sync(FULL, (idx < NS && d < 32u) ? (1u << (d & 31u)) : 0u);
      const uint32_t sg = cur + (uint32_t)__popc(M & lm_le);
      cur += (uint32_t)__popc(M);
      const uint32_t c = base + (uint32_t)lane;
      const bool in = c < T;
      const uint2 rec = sh.seg[wid][in ? sg : last];
      const uint32_t j = in ? rec.x + (c - (rec.y & kOffMask)) : rec.x;
      const uint32_t meta = rec.y >> 21;
      const int o = (int)(meta & 31u), code = (int)(meta >> 5);
      const float4 ow = sh.r0[wid][o];
      const float lo = sh.kc[wid][o].x;
      const float fdx = (float)(code & 3) - 1.f, fdy = (float)((code >> 2) & 3) - 1.f, fdz = (float)(code >> 4) - 1.f;
      const float sx = __fmaf_rn(-fdx, lo, ow.x), sy = __fmaf_rn(-fdy, lo, ow.y), sz = __fmaf_rn(-fdz, lo, ow.z);
      const float4 qv = __ldg(&C.c.r0[j]);
      const float ddx = __fsub_rn(sx, qv.x), ddy = __fsub_rn(sy, qv.y), ddz = __fsub_rn(sz, qv.z);
      const float s2 = __fmaf_rn(ddz, ddz, __fmaf_rn(ddy, ddy, __fmul_rn(ddx, ddx)));
      const float Rm = __fadd_rn(sh.rw[wid][o], qv.w);
      const bool hit = in && s2 < __fmul_rn(Rm, Rm) && (kSym || (int64_t)j != p0 + o);
      const unsigned B = __ballot_sync(FULL, hit);
      if (hit) sh.pq[wid][qn + (uint32_t)__popc(B & lm_lt)] = make_uint2(j, meta);
      qn += (uint32_t)__popc(B);
      if (qn >= 32u) {
        stream_flush<kSym>(C, sh, wid, lane, p0, qn, 32u);
        qn -= 32u;
      }
    }
    __syncwarp();  // the next phase rewrites the segments
  }
  if (qn) stream_flush<kSym>(C, sh, wid, lane, p0, qn, qn);
  __syncwarp();
  if (walk) {
    const float4 a = sh.acc[wid][lane];
    if (kSym) {
      if (a.w != 0.f) atomicAdd(&C.c.f32[p], a);
    } else {
      C.c.f32[p] = a;
    }
  }
}

// Static flags of every FP32-path cell (§5.5), for the static-mask mode.
__global__ void __launch_bounds__(kAgentThreads) k_static(DevCtx C) {
  if (C.g->err & ERR_TABLE) return;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= C.g->n_cells) return;
  const int sim = C.c.sim[p];
  const SimConst &sc = C.sc[sim];
  const SimState &s = C.ss[sim];
  if (!s.valid || sc.precision == BDM_PREC_FP64) return;
  int64_t cx, cy, cz;
  unpack_coords(C.c.pkey[p], cx, cy, cz);
  C.c.stat[p] = is_static_cell(C, sc, s, p, cx, cy, cz, C.g->stamp & kStampMask) ? 1 : 0;
}

static inline unsigned int stream_blocks(int64_t n, int t) { return (unsigned int)((n + t - 1) / t); }

template <bool kTorus, bool kOne>
static void launch_stream_mode(const DevCtx &C, cudaStream_t st, int mode, unsigned int nb, int threads) {
  if (mode == kModeSymMasked) k_force32w<kModeSymMasked, kTorus, kOne><<<nb, threads, 0, st>>>(C);
  else if (mode == kModeFull) k_force32w<kModeFull, kTorus, kOne><<<nb, threads, 0, st>>>(C);
  else k_force32w<kModeSym, kTorus, kOne><<<nb, threads, 0, st>>>(C);
}

void launch_force_stream(const DevCtx &C, cudaStream_t st, int mode, int threads, bool torus) {
  if (threads > kStreamThreads) threads = kStreamThreads;
  const unsigned int nb = stream_blocks(C.total_slots, threads);
  if (mode == kModeSymMasked)
    k_static<<<stream_blocks(C.total_slots, kAgentThreads), kAgentThreads, 0, st>>>(C);
  const bool one = C.n_sims == 1;
  if (torus) {
    if (one) launch_stream_mode<true, true>(C, st, mode, nb, threads);
    else launch_stream_mode<true, false>(C, st, mode, nb, threads);
  } else {
    if (one) launch_stream_mode<false, true>(C, st, mode, nb, threads);
    else launch_stream_mode<false, false>(C, st, mode, nb, threads);
  }
}

}  // namespace bdm
