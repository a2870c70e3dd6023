// Shared device structures and helpers of the sm_103a mechanics library.
//
// Data layout (all simulations of a context share each array):
//   storage arrays, indexed by slot: simulation s owns slots
//     [base_s, base_s + cap_s); its agents occupy [base_s, base_s + n_s).
//   cell arrays, indexed by cell position: agents grouped by grid box, the
//     boxes of simulation s contiguous in [cell_base_s, cell_base_s + n_s).
//   box table: one 64-bit word per box (stamp | dirty | count | first
//     cell); simulation s owns entries [table_base_s, table_base_s +
//     table_cap_s).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bdm.h"
#include "ffmath.cuh"

namespace bdm {

// Latched device error bits.
enum : uint32_t {
  ERR_CAPACITY = 1u,   // agent capacity reached while dividing (informational)
  ERR_NONFINITE = 2u,  // NaN or infinity in a position or force
  ERR_TIMEOUT = 4u,    // a bounded retry loop ran out
  ERR_TABLE = 8u,      // box table region too small for the grid
  ERR_COORD = 16u,     // box coordinate beyond 2^21 per axis
  ERR_TORUS = 32u,     // a toroidal space narrower than three boxes per axis
};

// Space boundary conditions (§4.4.11).
enum : int32_t { BOUND_OPEN = 0, BOUND_CLOSED = 1, BOUND_TORUS = 2 };

// Flags per slot.
// FLAG_GHOST: a read-only neighbour (a halo agent owned elsewhere): a
// partner in every other agent's force, but it does not move, grow or
// divide in bdm_step and is never static.
enum : uint8_t { FLAG_CHANGED = 1u, FLAG_STATIC = 2u, FLAG_GHOST = 4u };

// Flags per cell (written by the placement kernel for the force kernel).
enum : uint8_t { CELL_STATIC_ELIGIBLE = 1u };

constexpr int kStages = BDM_NUM_STAGES;
constexpr int kCoordBits = 21;
constexpr uint64_t kCoordMask = (1ull << kCoordBits) - 1ull;

// Per-simulation constants (host-written).
struct SimConst {
  double k, gamma, adherence, max_disp, dt, box_length, growth_rate, divide_volume;
  double box_scale;           // box length = box_scale x largest diameter when box_length is 0
  float kf, gammaf, adherence2f, max_disp2f, max_dispf, dtf;
  int32_t precision, detect_static, sort_interval, grows;
  uint64_t seed;
  int64_t base, cap;
  int64_t table_base, table_cap;
  int32_t boundary;           // BOUND_*
  int32_t exec_ctx;           // BDM_EXEC_COPY or BDM_EXEC_INPLACE
  double bmin, bmax;          // the space of closed and toroidal boundaries, per axis
  double bsize, bhalf;        // bmax - bmin and half of it
};

// Per-simulation state (device-written).
struct SimState {
  int64_t n;                  // agent count
  unsigned long long bmin[3]; // order-preserving keys of the per-axis minimum
  unsigned long long bmax[3]; // ... maximum
  unsigned long long dmax;    // ... largest diameter
  double o[3], L;             // grid of the current iteration
  int64_t dims[3];
  int64_t nboxes;
  float Lh, Ll;               // L as float-float
  float ilh, ill;             // 1/L as float-float
  float marg;                 // conservative margin of the FP32 pair filter
  float rmaxf;                // largest radius of the iteration, rounded up to FP32
  int32_t same_grid;          // grid equals the previous iteration's
  int32_t valid;              // grid fits the table region
  int32_t has_prev;
  int32_t keep_boxes;         // same_grid, and no agent moved since the last build unseen by its flags
  double prev_o[3], prev_L;
  int64_t prev_dims[3];
  int64_t cell_base;
  unsigned long long cell_cursor;  // next unclaimed cell of the build (unordered scan)
  int64_t ncell;              // agents placed in the cells of the last build
  int64_t t;                  // iterations completed
  int64_t it;                 // index of the iteration being computed
  unsigned long long n_static, n_moved;
  unsigned long long updates;  // agent-updates stepped since the agents were set
  double skin;                // grid reuse: how far an agent may leave its box before the grid is rebuilt
  float skin_lo, skin_hi;     // the same bounds on a box-relative offset in FP32, rounded inwards
  float skin_pad;             // the skin rounded up (box pruning of iterations that keep the grid)
};

// Global counters of a context.
struct Globals {
  uint32_t stamp;             // grid timestamp (all simulations, every build)
  uint32_t err;               // latched error bits
  int64_t n_cells;            // agents over all simulations
  int64_t n_new;              // agents created in the current division round
  uint32_t tile_ticket;       // scan tiles claimed in this build (reset by k_params)
  uint32_t test_flags;        // TEST_* hooks (host-set; 0 in normal use)
  uint32_t n_ovf;             // FP64-path agents left to the overflow kernel (reset by k_params)
  uint32_t regrid;            // grid reuse: the next iteration must rebuild the grid
  uint32_t reuse;             // grid reuse: this iteration keeps the last build's grid
  uint32_t reused;            // grid reuse: an iteration since the last build kept its grid
  unsigned long long n_builds; // grid builds of step iterations
  uint32_t ip_count[27];      // in-place context: boxes per colour of this iteration
  uint32_t ip_cursor[27];     //   fill cursors of the colour lists
  uint32_t ip_off[28];        //   start of each colour's list (in DevCtx::ovf)
};

// Test hooks of Globals::test_flags.  TEST_SCAN_TIMEOUT: the ordered scan's
// look-back waits for a tile word that no tile publishes and gives up after
// kTestSpin polls, so that a test sees its bounded wait run out.
// TEST_INPLACE_NARROW (read on the host): the in-place context runs its
// boxes on groups of 8 lanes whatever the population's size.
enum : uint32_t { TEST_SCAN_TIMEOUT = 1u, TEST_INPLACE_NARROW = 2u };

// Slots from which the in-place context runs its boxes on groups of 8 lanes
// (four boxes per warp) rather than a warp per box.
constexpr int64_t kInplaceNarrowSlots = 131072;

struct Agents {               // storage arrays (per slot)
  double *x, *y, *z, *d, *v;
  int32_t *id;                // caller ID
  int32_t *sim;               // owning simulation (every slot of a region)
  uint64_t *pkey;             // packed box coordinates c_x | c_y << 21 | c_z << 42 of the last
                              // step's grid (a step reads them as history, then rewrites them)
  uint32_t *rank;             // position inside the box
  uint8_t *flags;
  uint8_t *nnz;               // non-zero pair forces of the last evaluation (saturating)
};

struct Cells {                // cell arrays (per cell position)
  int32_t *slot;
  int32_t *sim;
  uint64_t *pkey;
  float4 *r0;                 // FP32 path: (w_hi.xyz, r_hi): offset inside the own box
  float4 *r1;                 //            (w_lo.xyz, r_lo)
  double4_32a *r64;               // FP64 path: (x, y, z, r)
  uint8_t *flag;
  float4 *f32;                // net force (FP32 path)
  double4_32a *f64;               // net force (FP64 path)
  uint8_t *nnz;
  uint8_t *stat;
};

// Box table: one 64-bit word per box of the bounding grid,
//   stamp (21 bits) << 43 | dirty << 42 | count (10 bits) << 32 | first cell.
// A box is empty unless its stamp equals the current build's; the host
// clears the table before the stamp counter would wrap.
struct Table {
  unsigned long long *e;
};

constexpr int kStampBits = 21;
constexpr uint32_t kStampMask = (1u << kStampBits) - 1u;
constexpr uint32_t kMaxBoxCount = 1023u;

__host__ __device__ __forceinline__ uint32_t ent_stamp(unsigned long long e) { return (uint32_t)(e >> 43); }
__host__ __device__ __forceinline__ bool ent_dirty(unsigned long long e) { return ((e >> 42) & 1ull) != 0; }
__host__ __device__ __forceinline__ uint32_t ent_count(unsigned long long e) { return (uint32_t)(e >> 32) & 0x3FFu; }
__host__ __device__ __forceinline__ uint32_t ent_start(unsigned long long e) { return (uint32_t)e; }
// agents of a box in the current build (0 for a box of an older build)
__host__ __device__ __forceinline__ uint32_t ent_live(unsigned long long e, uint32_t stamp) {
  return ent_stamp(e) == stamp ? ent_count(e) : 0u;
}

struct DevCtx {
  SimConst *sc;
  SimState *ss;
  Globals *g;
  Agents a;
  Cells c;                    // cells of the last iteration
  Cells q;                    // cells of the last neighbor query
  Table tab;
  int32_t *order;             // simulations in slot-region order (-1 padded)
  unsigned long long *tstat;  // per scan tile: stamp << 34 | state << 32 | sum (look-back)
  uint64_t *qkey;             // per slot: packed box of the last query build (queries only)
  uint8_t *kind;              // agent kinds by ID (slot region base + ID), or NULL: every agent kind 0
  int32_t *ovf;               // FP64 path: cells with more overlapping partners than the row kernel keeps;
                              // in-place context: the box leaders of every colour
  int32_t n_sims;
  int64_t total_slots;
};

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ord_key(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double ord_val(unsigned long long k) {
  unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ void unpack_coords(uint64_t p, int64_t &cx, int64_t &cy, int64_t &cz) {
  cx = (int64_t)(p & kCoordMask);
  cy = (int64_t)((p >> kCoordBits) & kCoordMask);
  cz = (int64_t)((p >> (2 * kCoordBits)) & kCoordMask);
}

__device__ __forceinline__ int64_t linear_box(const SimState &s, int64_t cx, int64_t cy, int64_t cz) {
  return cx + s.dims[0] * (cy + s.dims[1] * cz);
}

// Box coordinate of centre coordinate x on axis a (§4.4.3:
// floor((x - o_a) / L) with IEEE FP64 subtraction, division and floor),
// clamped to the grid.  The FP64 division runs only for undecided
// quotients.
__device__ __forceinline__ uint32_t grid_coord(const SimState &s, double x, int a) {
  const double av = __dsub_rn(x, s.o[a]);
  float ah, al;
  split_ff(av, ah, al);
  int c;
  int64_t cl;
  if (box_coord_ff(ah, al, s.ilh, s.ill, c))
    cl = c;
  else
    cl = (int64_t)floor(__ddiv_rn(av, s.L));
  return (uint32_t)(cl < 0 ? 0 : (cl >= s.dims[a] ? s.dims[a] - 1 : cl));
}

__device__ __forceinline__ void set_err(Globals *g, uint32_t bits) { atomicOr(&g->err, bits); }

// Table index of the stencil box (c + d) of simulation sc: false when it
// lies outside an open grid; wrapped around on a torus (every axis of a
// toroidal grid has at least three boxes, so the 27 boxes are distinct).
__device__ __forceinline__ bool stencil_index(const SimConst &sc, const SimState &s, int64_t cx, int64_t cy,
                                              int64_t cz, int dx, int dy, int dz, int64_t &idx) {
  int64_t x = cx + dx, y = cy + dy, z = cz + dz;
  if (sc.boundary == BOUND_TORUS) {
    x = x < 0 ? x + s.dims[0] : (x >= s.dims[0] ? x - s.dims[0] : x);
    y = y < 0 ? y + s.dims[1] : (y >= s.dims[1] ? y - s.dims[1] : y);
    z = z < 0 ? z + s.dims[2] : (z >= s.dims[2] ? z - s.dims[2] : z);
  } else if (x < 0 || x >= s.dims[0] || y < 0 || y >= s.dims[1] || z < 0 || z >= s.dims[2]) {
    return false;
  }
  idx = sc.table_base + linear_box(s, x, y, z);
  return true;
}

// Coordinate difference a - b; on a torus the minimum image (- size above
// half of it, + size below minus half), IEEE FP64 as the definition orders it.
__device__ __forceinline__ double coord_diff(const SimConst &sc, double a, double b) {
  double d = __dsub_rn(a, b);
  if (sc.boundary == BOUND_TORUS) {
    if (d > sc.bhalf) d = __dsub_rn(d, sc.bsize);
    else if (d < -sc.bhalf) d = __dadd_rn(d, sc.bsize);
  }
  return d;
}

// A new coordinate under the boundary condition: clamped into a closed
// space, wrapped into a toroidal one (the rounding guard keeps it below
// bmax).
__device__ __forceinline__ double bound_apply(const SimConst &sc, double v) {
  if (sc.boundary == BOUND_CLOSED) return v < sc.bmin ? sc.bmin : (v > sc.bmax ? sc.bmax : v);
  if (sc.boundary == BOUND_TORUS) {
    if (v >= sc.bmax) v = __dsub_rn(v, sc.bsize);
    else if (v < sc.bmin) v = __dadd_rn(v, sc.bsize);
    if (v >= sc.bmax) v = sc.bmin;
  }
  return v;
}

// Static check (§5.5): the agent itself is eligible (unchanged in the last
// iteration, at most one non-zero pair force, grid unchanged) and no box of
// its stencil carries a dirty mark of the current build.
__device__ __forceinline__ bool is_static_cell(const DevCtx &C, const SimConst &sc, const SimState &s, int64_t p,
                                          int64_t cx, int64_t cy, int64_t cz, uint32_t stamp) {
  if (!sc.detect_static || !s.same_grid || !(C.c.flag[p] & CELL_STATIC_ELIGIBLE)) return false;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t idx;
        if (!stencil_index(sc, s, cx, cy, cz, dx, dy, dz, idx)) continue;
        const unsigned long long e = C.tab.e[idx];
        if (ent_stamp(e) == stamp && ent_dirty(e)) return false;
      }
  return true;
}

// Grid-stride helpers sized for 152 SMs.
constexpr int kThreads = 256;
// Block size of the one-agent-per-thread passes of the grid build and the
// displacement (measured faster than 256 or 512 on this part).
constexpr int kAgentThreads = 128;

}  // namespace bdm
