// Host-side launchers of the device stages (one translation unit each).
#pragma once

#include "common.cuh"

namespace bdm {

// grid.cu
void launch_bbox(const DevCtx &C, cudaStream_t st, int step = 0);
// Grid reuse: the device decision at the start of a step iteration (sort:
// its re-sort mode), and the force clearing of iterations that keep the grid.
void launch_decide(const DevCtx &C, cudaStream_t st, int sort);
void launch_zero_f32(const DevCtx &C, cudaStream_t st);
void launch_params(const DevCtx &C, cudaStream_t st, int step);
void launch_count(const DevCtx &C, cudaStream_t st, int step);
// The scan needs tstat in the context: scan_tiles(total_slots) words,
// cleared whenever the build stamp restarts.
int64_t scan_tiles(int64_t total_slots);
// ordered: box ranges in the storage order of the leaders (decoupled
// look-back); otherwise in the order the scan's blocks finish
void launch_scan(const DevCtx &C, cudaStream_t st, int step = 1, int ordered = 1);
void launch_place(const DevCtx &C, cudaStream_t st, int step, int zero_f32 = 0);

// force.cu
// FP32 path: variant 0 symmetric half stencil (needs the forces zeroed by
// the placement), 1 deferred walk with rows flattened, 2 direct loop, 3
// deferred walk box by box, 4 as 0 without queue, 5 warp candidate stream
// (force_stream.cu; half stencil, or the full one when a simulation detects
// static agents), 6 as 5 with the static flags computed first and the half
// stencil kept.  The FP64 path runs the row kernel.
constexpr int kForceVariants = 7;
struct ForcePlan {
  int variant;      // variant that runs
  bool zero_f32;    // the placement must zero the FP32 forces (symmetric walks)
};
// any_static: some FP32-path simulation detects static agents
ForcePlan plan_force(int variant, bool any_static);
// any_torus: some FP32-path simulation is toroidal (only variants 5 and 6
// wrap the stencil)
void launch_force(const DevCtx &C, cudaStream_t st, int variant = 0, bool has_fp32 = true, bool has_fp64 = true,
                  bool any_static = false, bool any_torus = false);
// force64.cu: the FP64 path (row kernel, overflow kernel)
void launch_force64(const DevCtx &C, cudaStream_t st);
// force_stream.cu: mode 0 half stencil, 1 full stencil with static skip,
// 2 static flags first, then the half stencil
void launch_force_stream(const DevCtx &C, cudaStream_t st, int mode, int threads, bool torus);
// inplace.cu: S4 + S5 of the in-place execution context, one launch per box colour.
// narrow: groups of 8 lanes per box (large populations), else a warp per box
void launch_inplace(const DevCtx &C, cudaStream_t st, int colours, bool narrow);
// track: grid reuse (cell records follow the moved agents; skin check).
void launch_displace(const DevCtx &C, cudaStream_t st, bool track = false);

// diffusion.cu (soma-clustering slice)
typedef bdm_diffusion_grid DiffGrid;
void launch_diffuse_step(cudaStream_t st, const double *in, double *out, const DiffGrid &g, double nu, double mu,
                         double dt);
void launch_secrete(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const DiffGrid &g, double *u,
                    double quantity);
void launch_chemotaxis(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const DiffGrid &g, const double *u,
                       double weight);
// The same two inside bdm_step: the agent count from the device, launched
// over the simulation's capacity.
void launch_secrete_step(const DevCtx &C, cudaStream_t st, int sim, int kind, int64_t base, int64_t cap,
                         const DiffGrid &g, double *u, double quantity);
void launch_chemotaxis_step(const DevCtx &C, cudaStream_t st, int sim, int kind, int64_t base, int64_t cap,
                            const DiffGrid &g, const double *u, double weight);
// Removal's renumbering applied to the agent kinds (by ID).
void launch_kinds_move(const DevCtx &C, cudaStream_t st, int64_t base, const int64_t *hole, const int64_t *mover,
                       int64_t np);

// sir.cu (epidemiology use case): one step on the query cells of `sim`
void launch_sir_step(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n, int64_t base,
                     const uint8_t *st_in, uint8_t *st_out, double *nxyz, const bdm_sir_params &prm, long long t);

// query.cu
void launch_boxids(const DevCtx &C, cudaStream_t st, int sim, int64_t *out_by_id);
int64_t launch_pairs(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n, double radius,
                     int64_t *counts, int64_t *offsets, int64_t *pairs_dev, int64_t cap, uint32_t *partial,
                     cudaError_t *err);
void launch_gather_agents(const DevCtx &C, cudaStream_t st, int sim, int64_t base, int64_t n, double *xyz,
                          double *diam);
void launch_gather_forces(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n, double *force,
                          int32_t *nnz, uint8_t *stat, int32_t *overlaps = nullptr);
void launch_count_flags(const DevCtx &C, cudaStream_t st, int sim, int64_t cell_base, int64_t n,
                        unsigned long long *counts2);
void launch_set_agents(const DevCtx &C, cudaStream_t st, int sim, int64_t base, int64_t n, int64_t cap,
                       const double *xyz, const double *diam);
void launch_set_ghosts(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const uint8_t *mask);
void launch_update_agents(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, const double *xyz,
                          const double *diam);
// first invalid row into *bad: a position not finite (outside the space of
// a closed or toroidal boundary), a diameter not finite and > 0
void launch_check_input(cudaStream_t st, int64_t n, const double *xyz, const double *diam, unsigned long long *bad,
                        int boundary = BOUND_OPEN, double bmin = 0.0, double bmax = 0.0);

// query.cu: checkpoint state arrays (by caller ID) in device staging memory
int64_t state_array_bytes(int64_t n);
void launch_state_gather(const DevCtx &C, cudaStream_t st, int64_t base, int64_t n, void *staging);
// first invalid row into *bad (set to ~0 by the caller)
void launch_state_check(cudaStream_t st, int64_t n, const void *staging, unsigned long long *bad);
// n rows of arrays laid out for layout_n rows (-1: n)
void launch_state_scatter(const DevCtx &C, cudaStream_t st, int sim, int64_t base, int64_t n, int64_t cap,
                          const void *staging, int64_t layout_n = -1);
// removal: rows movers[k] -> holes[k] of the arrays of n_old agents, then the
// first n_new rows marked changed
void launch_state_remove(cudaStream_t st, void *staging, int64_t n_old, int64_t n_new, const int64_t *holes,
                         const int64_t *movers, int64_t np);

// sort.cu
void launch_cell_order(const DevCtx &C, cudaStream_t st, void *scratch);
void launch_morton(const DevCtx &C, cudaStream_t st, void *scratch, size_t scratch_bytes, int key_bits,
                   int curve = 0);
size_t morton_scratch_bytes(int64_t total_slots);

// growth.cu
void launch_growth(const DevCtx &C, cudaStream_t st, void *scratch, size_t scratch_bytes);
size_t growth_scratch_bytes(int64_t total_slots, int n_sims);

}  // namespace bdm
