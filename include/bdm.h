/*
 * bdm.h -- C ABI of the GB300 (sm_103a) mechanical-interaction step for
 * spherical agents, after the BioDynaMo thesis (arXiv 2503.10796).
 *
 * One iteration, as the thesis's simulation loop runs it (§5.2,
 * Algorithm 8), under the copy execution context (§5.2, "Different
 * Execution Contexts"): all agents see the state at the start of the
 * iteration and the changes are committed at its end.
 *
 *   S0  bounding box and box length: origin o = per-axis minimum of the
 *       centers; box length L = user value, else the largest diameter
 *       (§4.4.3 "Environment"); boxes per axis n_a = floor((max_a-o_a)/L)+1.
 *   S1  box index per agent: c_a = floor((x_a - o_a) / L) in IEEE FP64,
 *       index c_x + n_x (c_y + n_y c_z) (§5.3.1, Fig 5.4B).
 *   S2  grid build with per-box timestamps, so that empty boxes are never
 *       cleared (§5.3.1): count, a contiguous cell range per box (prefix
 *       sum over the box leaders, or ranges claimed by atomics), placement.
 *   S3  Morton re-sort of the agent storage every `sort_interval`
 *       iterations (§5.4.2, Fig 5.4); results never depend on it.
 *   S4  pairwise force over the 27-box stencil, Eq 4.1 / Eq 4.2 (§4.5.1):
 *       delta = r_i + r_j - dist, r = r_i r_j / (r_i + r_j),
 *       F_N = k delta - gamma sqrt(r delta), along (x_i - x_j) / dist.
 *   S5  displacement: none while |F| <= adherence, else dt F with its norm
 *       clamped to max_displacement (§4.5.1; Table D.1 MechanicalForcesOp).
 *   S6  static agents skip S4/S5 (§5.5, conditions (i)-(iv)).
 *   S7  growth and division (Table D.1 GrowthDivision).
 *
 * Conventions.
 *   - Every call returns BDM_OK (0) or a negative BDM_E_* code; the text of
 *     the last error of a context is returned by bdm_last_error().
 *   - Host pointers are owned by the caller; the library copies in and out
 *     and never keeps them.  With BDM_DEVICE_PTRS the pointers are device
 *     pointers, read or written on the context's stream.
 *   - A context is not thread-safe: use it from one host thread.
 *   - Agent IDs are the row indices given to bdm_set_agents (per
 *     simulation); agents created by division get the next IDs, in
 *     ascending parent-ID order.  IDs survive every re-sort.
 *   - bdm_step is asynchronous.  Errors found on the device (capacity,
 *     non-finite values, a bounded wait that ran out) are latched and
 *     reported by the next bdm_sync or bdm_get_* call.
 */
#ifndef BDM_H_
#define BDM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BDM_OK = 0,
  BDM_E_INVAL = -1,     /* bad argument or input value */
  BDM_E_NOMEM = -2,     /* device or host allocation failed */
  BDM_E_CUDA = -3,      /* CUDA runtime error */
  BDM_E_CAPACITY = -4,  /* output buffer, agent capacity or box table too small */
  BDM_E_TIMEOUT = -5,   /* a bounded device wait ran out */
  BDM_E_NONFINITE = -6, /* a position or force became NaN or infinite */
  BDM_E_STATE = -7      /* call not valid in the current state */
};

enum { BDM_PREC_FP64 = 0, BDM_PREC_FP32_FORCE = 1 };

/* Space boundary conditions (§4.4.11).  Open: the space grows with the
 * agents (grid origin = per-axis minimum, as S0 states).  Closed: the space
 * is the cube [bound_min, bound_max] per axis; a new position (displacement,
 * daughter placement) is clamped into it per coordinate.  Toroidal: the
 * space is [bound_min, bound_max) per axis; a new coordinate v becomes
 * v - size when v >= bound_max, v + size when v < bound_min (bound_min if
 * rounding leaves it at bound_max); the grid tiles the space with
 * n = floor(size / L) >= 3 boxes per axis of length size / n from
 * bound_min, stencil boxes wrap around, and coordinate differences are
 * minimum images (dx - size when dx > size / 2, dx + size when
 * dx < -size / 2).  Positions given to a closed or toroidal simulation must
 * lie in its space. */
enum { BDM_BOUNDARY_OPEN = 0, BDM_BOUNDARY_CLOSED = 1, BDM_BOUNDARY_TOROIDAL = 2 };

/* Execution contexts (§5.2).  Copy: every quantity of an iteration is
 * computed from the snapshot at its start and committed after all agents.
 * In-place: an agent's new position is visible to the agents processed
 * after it in the same iteration.  The thesis leaves that order to its
 * scheduler; here it is fixed: boxes by colour (the parity of each box
 * coordinate, plus a third colour for the last box of a toroidal axis with
 * an odd number of boxes; colours ranked x + k_x (y + k_y z)), boxes of a
 * colour in ascending index, agents of a box in ascending ID.  Neighbours
 * are the agents of the 27-box stencil in the grid of the iteration's start,
 * at their current positions; each agent's force (summed in ascending
 * partner ID) and displacement are committed before the next agent.  The
 * in-place context runs the FP64 path without static detection
 * (BDM_E_INVAL otherwise), and all simulations of a context share one
 * context. */
enum { BDM_EXEC_COPY = 0, BDM_EXEC_INPLACE = 1 };

/* flags of bdm_set_agents / bdm_get_agents */
enum { BDM_DEVICE_PTRS = 1 };

/* Per-simulation parameters (thesis Param and Cell attributes). */
typedef struct {
  double k;                /* Eq 4.1 repulsion coefficient (thesis default 2) */
  double gamma;            /* Eq 4.1 adhesion coefficient (thesis default 1) */
  double adherence;        /* an agent moves only if |F| > adherence */
  double max_displacement; /* norm clamp of one iteration's displacement */
  double dt;               /* simulation time step */
  double box_length;       /* grid box length; 0 = largest diameter of each iteration */
  double growth_rate;      /* volume growth per unit time; 0 = no growth */
  double divide_volume;    /* volume at which an agent divides (growth only) */
  int32_t precision;       /* BDM_PREC_FP64 or BDM_PREC_FP32_FORCE */
  int32_t detect_static;   /* 1: skip the force of static agents (§5.5) */
  int32_t sort_interval;   /* Morton re-sort every n iterations; 0 = never */
  int32_t boundary;        /* BDM_BOUNDARY_OPEN (0), _CLOSED or _TOROIDAL */
  uint64_t seed;           /* key of the counter-based generator (division axes) */
  int64_t capacity;        /* agent capacity of this simulation; 0 = count at bdm_set_agents */
  double bound_min;        /* the space of closed and toroidal boundaries, per axis */
  double bound_max;
  int32_t execution_context; /* BDM_EXEC_COPY (0, default) or BDM_EXEC_INPLACE */
  int32_t reserved;        /* 0 */
} bdm_params;

/* Counters of one simulation (bdm_get_stats). */
typedef struct {
  int64_t agents;          /* current agent count */
  int64_t iterations;      /* iterations stepped since bdm_set_agents */
  int64_t static_agents;   /* agents skipped as static in the last iteration */
  int64_t moved_agents;    /* agents with a non-zero displacement in the last iteration */
  double origin_len[4];    /* grid of the last iteration: origin x, y, z and box length */
  int64_t dims[3];         /* boxes per axis of that grid */
  int64_t agent_updates;   /* sum over stepped iterations of the agent count at their start */
  int64_t reserved[3];
} bdm_stats;

typedef struct bdm_ctx bdm_ctx;

/* Create a context on CUDA device `device` for `n_sims` independent
 * simulations whose agent capacities sum to at most `max_agents_total`.
 * `per_sim` holds n_sims parameter sets.  `cuda_stream` is a cudaStream_t
 * to run on (for example a PyTorch stream), or NULL for a stream the
 * context creates.  The context owns all device memory it allocates.
 * Errors: BDM_E_INVAL (n_sims < 1, bad parameters), BDM_E_NOMEM,
 * BDM_E_CUDA. */
int bdm_create(const bdm_params* per_sim, int32_t n_sims, int64_t max_agents_total,
               int32_t device, void* cuda_stream, bdm_ctx** out);

/* Replace the agents of simulation `sim`: n rows of (x, y, z) in `xyz`
 * (n x 3, row-major) and n diameters.  Row i becomes agent ID i.  The
 * iteration counter and all history (static flags) restart.  Errors:
 * BDM_E_INVAL (sim out of range, n < 0, non-finite value, diameter <= 0),
 * BDM_E_CAPACITY (n above the simulation's capacity, or the capacities of
 * all simulations above max_agents_total). */
int bdm_set_agents(bdm_ctx* ctx, int32_t sim, int64_t n, const double* xyz,
                   const double* diameter, int32_t flags);

/* Give the current agents of simulation `sim` new positions and, when
 * `diameter` is not NULL, new diameters: row i of xyz (n x 3, row-major)
 * and of diameter belongs to agent ID i, and n must equal the agent count.
 * Unlike bdm_set_agents this keeps the simulation: storage order, iteration
 * counter and history stay, and agents whose values change count as changed
 * in the next iteration (static detection).  Meant for callers that move
 * agents between steps (coupling to another code).  The thesis has no
 * counterpart.  Errors: BDM_E_INVAL (n differs from the count, non-finite
 * value, diameter <= 0), BDM_E_STATE (no agents set), latched device
 * errors as bdm_sync. */
int bdm_update_agents(bdm_ctx* ctx, int32_t sim, int64_t n, const double* xyz,
                      const double* diameter, int32_t flags);

/* Checkpoint of simulation `sim` for a resume that continues bit for bit
 * (the thesis backs simulations up at an interval, §4.3.5; this is the state
 * one iteration reads).  bdm_get_state writes *size_out and, when cap_bytes
 * is at least that, the state into buf (host memory): a 144-byte header
 * (the magic "BDMSTATE", version 1, the agent count, the iterations done,
 * which are also the counter of the division axes' random numbers, the
 * agent-update counter and the grid of the last iteration) and, by caller
 * ID, positions, diameters, volumes, the box of the last grid, the changed,
 * static and ghost flags and the non-zero pair counts.  BDM_E_CAPACITY (nothing
 * written) when cap_bytes is too small, BDM_E_STATE when no agents are set.
 * bdm_set_state replaces the agents of `sim` by such a state (of this or
 * another context or simulation; the parameters are the receiving
 * simulation's): the next iterations then equal, in the FP64 path bit for
 * bit, those the saved simulation would have run.  Storage order is not part
 * of the state (the next due re-sort sorts again).  Errors: BDM_E_INVAL (not
 * a state of this version, size or header inconsistent, an agent value not
 * finite or a diameter or volume not > 0), BDM_E_CAPACITY (as
 * bdm_set_agents). */
int bdm_get_state(bdm_ctx* ctx, int32_t sim, void* buf, int64_t cap_bytes, int64_t* size_out);
int bdm_set_state(bdm_ctx* ctx, int32_t sim, const void* buf, int64_t size_bytes);

/* Remove the agents `ids` (n_ids distinct caller IDs, host memory) from
 * simulation `sim`, with the swaps of the thesis's parallel removal (§5.3.2,
 * Fig 5.1): of the n' agents left, those with an ID below n' keep it, and
 * the IDs below n' that removed agents held go, in ascending order, to the
 * surviving agents with IDs >= n', in ascending order.  Every survivor
 * counts as changed in the next iteration (the neighbourhoods of the removed
 * agents changed: no agent is static then), the iteration counter and the
 * last grid stay, and bdm_get_forces reports zeros until the next
 * iteration.  Errors: BDM_E_INVAL (an ID out of range or repeated),
 * BDM_E_STATE (no agents set), latched device errors as bdm_sync. */
int bdm_remove_agents(bdm_ctx* ctx, int32_t sim, int64_t n_ids, const int64_t* ids);

/* Mark agents of simulation `sim` as ghosts, read-only neighbours: ghost[i]
 * != 0 (host memory, n = the simulation's agent count, by caller ID) makes
 * agent i a ghost, 0 an ordinary agent.  A ghost is a partner in every other
 * agent's force, but bdm_step does not move, grow or divide it and never
 * counts it static (its own force and nnz are still reported).  This is the
 * halo of a domain decomposition (the aura of the thesis's distributed
 * engine, §6.2): a rank steps its own agents with the agents of the
 * neighbouring ranks within one largest diameter as ghosts, which puts every
 * partner of an owned agent on the rank (Eq 4.1 needs a distance below
 * r_i + r_j); with IDs in the global order the owned agents' FP64 results
 * equal a single domain's bit for bit.  An agent whose flag changes counts
 * as changed.  bdm_set_agents, bdm_set_state and bdm_remove_agents keep or
 * reset the flags with the agents (bdm_set_agents: no ghosts).  Errors:
 * BDM_E_INVAL (n differs from the agent count, NULL mask), BDM_E_STATE (no
 * agents set), latched device errors as bdm_sync. */
int bdm_set_ghosts(bdm_ctx* ctx, int32_t sim, int64_t n, const uint8_t* ghost);

/* Run n_iterations iterations of every simulation (S0-S7), asynchronously
 * on the context's stream.  Errors: BDM_E_STATE (a simulation has no
 * agents set), BDM_E_NOMEM (box table growth failed), BDM_E_CUDA. */
int bdm_step(bdm_ctx* ctx, int32_t n_iterations);

/* Wait for the context's stream and report latched device errors:
 * BDM_E_CAPACITY when a grid outgrew its box table or a box held more than
 * 1023 agents (that iteration's results are then undefined),
 * BDM_E_NONFINITE, BDM_E_TIMEOUT, BDM_E_INVAL when a toroidal space holds
 * fewer than three boxes per axis (the largest diameter grew too large). */
int bdm_sync(bdm_ctx* ctx);

/* Copy the agents of `sim` out in caller-ID order: xyz (cap x 3) and
 * diameter (cap), either may be NULL.  *n_out receives the agent count.
 * Returns BDM_E_CAPACITY, writing nothing, if the count exceeds cap. */
int bdm_get_agents(bdm_ctx* ctx, int32_t sim, int64_t cap, double* xyz, double* diameter,
                   int64_t* n_out, int32_t flags);

/* Unordered neighbor pairs {i, j}, i < j in caller IDs, sorted by (i, j),
 * of the current agents of `sim` (§4.4.3 ForEachNeighbor).  radius >= 0:
 * pairs with squared center distance < radius * radius; radius < 0:
 * overlapping pairs (delta > 0, the pairs that interact in Eq 4.1).  The
 * decision is taken in FP64 exactly as in the definitions above.  A radius
 * above the box length uses a grid of box length = radius.  pairs holds
 * 2 x cap int64 values (may be NULL when cap = 0); *n_out receives the pair
 * count; BDM_E_CAPACITY (nothing written) if it exceeds cap. */
int bdm_neighbors(bdm_ctx* ctx, int32_t sim, double radius, int64_t cap, int64_t* pairs,
                  int64_t* n_out);

/* Grid that the next iteration would build from the current agents of
 * `sim` (S0, S1): box index per caller ID in box_id (cap entries, may be
 * NULL), origin x, y, z and box length in origin_len, boxes per axis in
 * dims.  BDM_E_CAPACITY (nothing written) if the agent count exceeds cap. */
int bdm_get_grid(bdm_ctx* ctx, int32_t sim, int64_t cap, int64_t* box_id, double origin_len[4],
                 int64_t dims[3]);

/* Per-agent results of the last iteration of `sim`, by caller ID: the
 * net force (cap x 3; zero for static agents), the number of non-zero pair
 * forces (saturated at 255), the static flag and the number of overlapping
 * pairs (delta > 0, Eq 4.1; -1 for static agents, which evaluate none).
 * Any output may be NULL.  Agents created in the last iteration report
 * zeros (overlaps -1). */
int bdm_get_forces(bdm_ctx* ctx, int32_t sim, int64_t cap, double* force, int32_t* nnz,
                   uint8_t* is_static, int32_t* overlaps, int64_t* n_out);

/* Caller IDs of `sim` in device storage order (the order that the Morton
 * re-sort arranges). */
int bdm_get_storage_order(bdm_ctx* ctx, int32_t sim, int64_t cap, int64_t* ids, int64_t* n_out);

/* Counters of `sim` after the last iteration. */
int bdm_get_stats(bdm_ctx* ctx, int32_t sim, bdm_stats* out);

/* Per-stage timing.  While enabled, every stage of bdm_step is bracketed by
 * CUDA events on the context's stream; bdm_get_profile returns, for each
 * stage, the number of launches and the summed device time in ms since
 * profiling was enabled, and the stage names in `names` (NULL allowed).
 * Stages: 0 bbox, 1 grid count, 2 grid scan, 3 grid place, 4 force,
 * 5 displace, 6 growth/division, 7 morton sort, 8 substances. */
enum { BDM_NUM_STAGES = 9 };
int bdm_profile(bdm_ctx* ctx, int32_t enable);
int bdm_get_profile(bdm_ctx* ctx, int64_t launches[BDM_NUM_STAGES], double ms[BDM_NUM_STAGES],
                    const char* names[BDM_NUM_STAGES]);

/* Net force on each of n spheres, without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (allocator-free runtimes, programs that hand out
 * every byte of device memory from their own pool and cannot have a library
 * allocate behind their back).  It builds the grid of the given positions
 * and evaluates the force of one iteration exactly as bdm_step does for its
 * first iteration (S0-S4), but it calls no cudaMalloc, cudaFree or
 * allocating library routine: its working memory is one fixed array of
 * about 5 MB in the library's device memory, held by every GPU that loads
 * the library until the process exits.
 *
 * params: one parameter set (growth, static, sort, capacity and
 * execution-context fields are ignored: the first iteration has no static
 * agents, and the forces are those of the iteration's snapshot, as in the
 * copy context).
 * xyz: device pointer, n x 3 doubles, row-major; diameter: device pointer,
 * n doubles; force: device pointer, n x 3 doubles written in row order;
 * nnz: device pointer, n int32 (non-zero pair forces per agent), or NULL.
 * cuda_stream: the stream to run on (NULL: the legacy default stream).
 * The caller owns all four buffers.
 *
 * Limits: n <= 16384, at most 131072 grid boxes and at most 1023 agents in
 * one box; beyond them the call returns BDM_E_CAPACITY (n too large: before
 * any work; the others: after the run, with force contents undefined).
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress while that device is current.  The call waits for
 * its stream to finish (it reads the device error word before it gathers
 * the results), so it cannot be recorded into a CUDA stream capture.
 * All calls on a device share the one array: calls that overlap on the GPU
 * race and give undefined results.
 * Errors: BDM_E_INVAL (NULL pointer, n < 0, bad params), BDM_E_CAPACITY,
 * BDM_E_NONFINITE (a position not finite, or a diameter not finite and
 * > 0), BDM_E_CUDA. */
int bdm_forces_noalloc(const bdm_params* params, int64_t n, const double* xyz, const double* diameter,
                       double* force, int32_t* nnz, void* cuda_stream);

/* Tuning knobs of a context.  None of them changes results beyond the
 * order of floating-point sums over neighbors. */
typedef struct {
  int32_t force_variant;   /* force kernel of the FP32 path (the FP64 path always
                              runs its row kernel): 5 warp candidate stream, the
                              stencil boxes a sphere can reach laid end to end
                              and tested 32 at a time (default; half stencil with
                              each pair's force added to both agents, or the full
                              stencil when a simulation detects static agents);
                              6 as 5, but with static detection the static flags
                              are computed first and the half stencil is kept
                              (static agents' forces are then computed but
                              unused); 0 symmetric half-stencil walk, a lane per
                              agent (1 stands in when a simulation detects static
                              agents); 1 direct walk, rows flattened, pair
                              evaluation deferred; 2 direct loop, pairs evaluated
                              in the walk; 3 as 1 box by box; 4 as 0 with every
                              pair evaluated in the walk (crowded agents) */
  int32_t sort_interval;   /* -1: every simulation's own sort_interval;
                              >= 0: this re-sort interval for all simulations */
  int32_t sort_curve;      /* order the re-sort gives the storage: 0 Morton order of the
                              boxes (default, §5.4.2); 1 row-major box order */
  int32_t box_scale_pct;   /* grid box length in percent of the largest diameter, 100
                              to 400 (0 = 100), for simulations without static
                              detection and without a box_length of their own (a
                              longer box keeps every interaction inside the 27-box
                              stencil, §4.4.3; the static check's stencil would
                              change, so those simulations keep the thesis's rule) */
  int32_t iter_batch;      /* iterations per replayed CUDA graph, 1 to 64 (0 = 1) */
  int32_t test_flags;      /* test hooks, 0 in normal use.  Bit 0: the ordered grid
                              scan's bounded wait looks for a word that nothing writes
                              and gives up after 64 polls per tile, so that the next
                              bdm_sync reports BDM_E_TIMEOUT (that iteration's
                              results are undefined; the context stays usable).
                              Bit 1: the in-place context runs its boxes on groups of
                              8 lanes (its form for 131,072 slots and more) whatever
                              the context's size; results are the same */
  int32_t grid_reuse;      /* 1: incremental grid (the thesis adapts its grid to
                              incremental position updates, §6.2.5): an iteration
                              keeps the last build's grid while every agent stays
                              within the skin (L - largest diameter) / 2 of the box
                              it is registered in, which still puts every
                              interacting pair in neighbouring boxes; the moved
                              agents' cell records are rewritten in place.  The grid
                              is rebuilt when an agent left its skin, on re-sorts,
                              and after any other call that changes agents or the
                              grid.  Needs a box longer than the largest diameter
                              (box_scale_pct > 100 or a box_length) to keep any
                              grid; results are those of a rebuilt grid (FP64 path
                              bit for bit).  Only for contexts without static
                              detection, growth, toroidal boundaries or the
                              in-place context (BDM_E_INVAL otherwise).  0: rebuild
                              every iteration (default, §5.3.1). */
  int32_t reserved;        /* must be 0 */
} bdm_tuning;

int bdm_set_tuning(bdm_ctx* ctx, const bdm_tuning* tuning);
int bdm_get_tuning(bdm_ctx* ctx, bdm_tuning* tuning);

/* Knobs of bdm_autotune. */
enum {
  BDM_TUNE_FORCE = 1,     /* force_variant */
  BDM_TUNE_CURVE = 2,     /* sort_curve */
  BDM_TUNE_INTERVAL = 4,  /* sort_interval */
  BDM_TUNE_BOX = 8,       /* box_scale_pct */
  BDM_TUNE_BATCH = 16,    /* iter_batch */
  BDM_TUNE_ALL = 31
};

/* Autotuner (the thesis proposes automatic tuning of performance
 * parameters such as the sorting frequency, §7.1.7): from the current
 * agents, time the current setting and then, one knob after another, each
 * candidate of the knobs selected in `knobs` (BDM_TUNE_* bits; the others
 * keep their current values): every force-kernel variant, box lengths of
 * 100, 125 and 150% of the largest diameter, both storage curves, re-sort
 * intervals 0 (only if no simulation asked for re-sorting), 5, 10 and 25,
 * and 1, 4 or 10 iterations per graph.  Each trial runs a whole number of
 * re-sort periods after as many untimed iterations, the saved state is
 * restored after each trial, and the setting with the shortest time per
 * iteration is kept; *chosen (may be NULL) receives it.  The agents' state
 * after the call equals the state before it.  Errors: BDM_E_INVAL
 * (iterations < 1, unknown knob bits), BDM_E_STATE, BDM_E_NOMEM, latched
 * device errors. */
int bdm_autotune(bdm_ctx* ctx, int32_t iterations, int32_t knobs, bdm_tuning* chosen);

/* Launch counters of a context since bdm_create: CUDA graphs replayed by
 * bdm_step, the kernels they and bdm_step's own table sizing launched, the
 * iterations the graphs covered (iterations stepped while profiling is
 * enabled launch their kernels one by one and are not counted), and the
 * grid builds of stepped iterations (synchronizes the stream). */
typedef struct {
  int64_t graph_launches;
  int64_t kernels;
  int64_t graph_iterations;
  int64_t grid_builds;     /* grid builds of stepped iterations (with grid_reuse,
                              the iterations that rebuilt the grid) */
  int64_t reserved[4];
} bdm_counters;

int bdm_get_counters(bdm_ctx* ctx, bdm_counters* out);

/* ---- Soma-clustering slice: diffusion, secretion, chemotaxis ----------
 *
 * A diffusion grid of n[0] x n[1] x n[2] FP64 concentrations (§4.5.2),
 * point (i, j, k) stored at i + n[0] (j + n[1] k).  Point (i, j, k) stands
 * for the box [lo + (i, j, k) h, lo + (i + 1, j + 1, k + 1) h) per axis; a
 * position belongs to the box floor((x - lo) / h) (IEEE FP64).  Outside the
 * grid the concentration is zero (substances diffuse out of the space).
 * The concentrations are host memory (copied in and out on every call) or,
 * with BDM_DEVICE_PTRS, device memory read and written on the context's
 * stream.  Errors: BDM_E_INVAL for a NULL grid or array, n < 1 on an axis,
 * more than 2^40 points, h not finite and > 0, lo not finite, or (per call)
 * parameters below; BDM_E_NOMEM when scratch memory cannot be had; a
 * latched device error is reported first. */
typedef struct {
  double lo[3];   /* lower corner of box (0, 0, 0) */
  double h[3];    /* box size per axis */
  int64_t n[3];   /* points per axis */
} bdm_diffusion_grid;

/* Eq 4.3 (§4.5.2): n_steps explicit steps
 *   u' = u (1 - mu dt) + nu dt / hx^2 (u[i+1] - 2u + u[i-1]) + (y) + (z),
 * evaluated term by term in that order.  nu >= 0 (diffusion coefficient),
 * mu >= 0 (decay), dt >= 0, n_steps >= 0, all finite.  Stability
 * (nu dt (1/hx^2 + 1/hy^2 + 1/hz^2) <= 1/2) is the caller's choice. */
int bdm_diffuse(bdm_ctx* ctx, const bdm_diffusion_grid* grid, double* u, double nu, double mu, double dt,
                int32_t n_steps, int32_t flags);

/* Algorithm 6: every agent of simulation `sim` whose center lies inside the
 * grid adds `quantity` (finite) to the concentration of its box.
 * BDM_E_STATE when the simulation has no agents set. */
int bdm_secrete(bdm_ctx* ctx, int32_t sim, const bdm_diffusion_grid* grid, double* u, double quantity,
                int32_t flags);

/* Algorithm 7: every agent of simulation `sim` whose center lies inside the
 * grid moves by weight (finite) times the normalized gradient of its box:
 * g_a = (u[+1] - u[-1]) / (2 h_a) per axis, divided by
 * |g| = sqrt((gx gx + gy gy) + gz gz); no move where |g| = 0.  u is only
 * read.  Moved agents count as changed for static detection.
 * BDM_E_STATE when the simulation has no agents set. */
int bdm_chemotaxis(bdm_ctx* ctx, int32_t sim, const bdm_diffusion_grid* grid, const double* u, double weight,
                   int32_t flags);

/* Agent kinds of simulation `sim` (the cell types of the soma-clustering
 * benchmark, §4.6): kinds[i] in 0..3 for agent ID i (host memory, n = the
 * agent count).  A daughter takes its mother's kind, removal renumbers the
 * kinds with the agents, and bdm_set_agents and bdm_set_state reset every
 * kind to 0 (a state does not hold them).  Errors: BDM_E_INVAL (n differs
 * from the agent count, a kind above 3), BDM_E_STATE, BDM_E_NOMEM. */
int bdm_set_agent_kinds(bdm_ctx* ctx, int32_t sim, int64_t n, const uint8_t* kinds);

/* The same three inside bdm_step (the cell-clustering use case of §4.6):
 * the agents of kind `kind` (0..3) of simulation `sim` keep a substance on
 * `grid`, with initial concentrations u (host memory, or device memory with
 * BDM_DEVICE_PTRS; copied, the caller keeps u).  After the mechanical step
 * of every iteration (forces, displacement, growth), over the agents of that
 * kind and each seeing the result of the one before: they secrete
 * `quantity` into the boxes of their new positions (Algorithm 6), the
 * substance takes one step of Eq 4.3 with the simulation's dt and nu, mu
 * (>= 0), and they move by `weight` along its normalized gradient
 * (Algorithm 7).  Kinds touch neither each other's agents nor substances.
 * grid NULL removes the substance.  Open space only.  Errors: BDM_E_INVAL
 * (bad kind, grid or values, a closed or toroidal simulation), BDM_E_NOMEM.
 * Grid reuse stays correct: agents that chemotaxis moves make the next
 * iteration rebuild the grid. */
int bdm_set_substance(bdm_ctx* ctx, int32_t sim, int32_t kind, const bdm_diffusion_grid* grid, const double* u,
                      double nu, double mu, double quantity, double weight, int32_t flags);

/* The concentrations of the substance of kind `kind` of simulation `sim`
 * (grid order, as u of bdm_set_substance) into u (cap doubles; host, or
 * device with BDM_DEVICE_PTRS); *n_out (may be NULL) receives the point
 * count.  BDM_E_STATE (no substance), BDM_E_CAPACITY (cap too small, nothing
 * written). */
int bdm_get_substance(bdm_ctx* ctx, int32_t sim, int32_t kind, double* u, int64_t cap, int64_t* n_out,
                      int32_t flags);

/* ---- Epidemiology use case (§4.6.3) ------------------------------------
 * Persons are the agents of a simulation (their diameters play no part);
 * each has a state 0 susceptible, 1 infected, 2 recovered, in a uint8
 * array by agent ID (host memory, or device memory with BDM_DEVICE_PTRS).
 * One step, all persons reading the states and positions at its start:
 *   Algorithm 3: a susceptible person draws u0; if u0 < p_infect and any
 *     other person infected at the start of the step lies within radius
 *     (squared distance (dx dx + dy dy) + dz dz below radius * radius), it
 *     becomes infected;
 *   Algorithm 4: an infected person (also one infected in this step) draws
 *     u1 and recovers if u1 < p_recover;
 *   Algorithm 5: every person moves by speed along the normalized vector of
 *     three uniforms in [-1, 1) (no move for the zero vector), and every
 *     coordinate is wrapped into [0, length) (a torus).
 * Uniforms: Philox4x64-10 with key {seed, 1}, counter {ID, t, 0, 0}
 * (words 0, 1: u0, u1) and {ID, t, 1, 0} (words 0-2: movement), each the
 * top 53 bits of a word times 2^-53; t counts steps from t0.
 * Errors: BDM_E_INVAL for a NULL argument, n_steps < 0, t0 < 0, radius,
 * speed or length not finite and >= 0 (length > 0), probabilities outside
 * [0, 1], a state outside {0, 1, 2}; BDM_E_STATE when the simulation has
 * no agents set; BDM_E_NOMEM for scratch memory.  Moved persons count as
 * changed for the mechanics step. */
typedef struct {
  double radius, p_infect, p_recover, speed, length;
  uint64_t seed;
} bdm_sir_params;

int bdm_sir_step(bdm_ctx* ctx, int32_t sim, const bdm_sir_params* params, uint8_t* state, int64_t t0,
                 int32_t n_steps, int32_t flags);

/* Release everything the context owns. */
void bdm_destroy(bdm_ctx* ctx);

/* Text of the last error of ctx (or of the last failed bdm_create when ctx
 * is NULL).  Valid until the next call on the same context. */
const char* bdm_last_error(const bdm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BDM_H_ */
