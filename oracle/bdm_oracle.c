/*
 * bdm_oracle.c -- plain, single-threaded FP64 CPU oracle of the
 * mechanical-interaction step for spherical agents described in the
 * BioDynaMo thesis (arXiv 2503.10796).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library and its binding) never calls it, and it shares no code,
 * header, table or helper with that path.
 *
 * Everything here is written to be checked by eye against the thesis:
 * no blocking, no fusion, no reordering beyond what the text states.
 * Compiled with -O2 -ffp-contract=off so that no multiply-add is fused.
 *
 * One iteration follows the thesis's simulation loop (§5.2, Algorithm 8)
 * under the copy execution context (§5.2, "Different Execution Contexts"):
 * every quantity of iteration t is computed from the snapshot taken at the
 * start of t and committed after all agents were processed.  Sums run over
 * neighbors in ascending agent-ID order, so no storage order can change a
 * result.
 *
 *   1. uniform grid (§4.4.3 "Environment", §5.3.1): origin = per-axis
 *      minimum of the centers, box length = largest diameter (or the user's
 *      value), box of an agent from its center, 27-box search;
 *   2. pairwise force, Eq 4.1 / Eq 4.2 (§4.5.1) with k and gamma;
 *   3. displacement with the adherence threshold and the maximum-
 *      displacement clamp (§4.5.1 last paragraph, Table D.1
 *      MechanicalForcesOp, the simulation_max_displacement parameter);
 *   4. static-agent detection (§5.5, conditions (i)-(iv));
 *   5. growth and division (Table D.1 GrowthDivision, Cell::Divide), with
 *      the counter-based random numbers proposed in §7.1.4;
 *   6. Morton order of grid boxes by the gap algorithm (§5.4.2, Fig 5.4);
 *   7. the space boundary conditions of §4.4.11 (open, closed, toroidal);
 *   8. agent removal with the swap of §5.3.2 (Fig 5.1);
 *   9. the in-place execution context (§5.2), as an alternative to copy.
 *
 * Readings taken where the thesis is silent (each one is listed with the
 * design notes of the repository):
 *   - displacement = dt * F (unit mobility; mass unused);
 *   - adherence is a threshold: no movement while |F| <= adherence;
 *   - the clamp limits the Euclidean norm of the displacement;
 *   - a pair interacts iff delta > 0 (strict); dist == 0 contributes 0;
 *   - radius queries use dist^2 < R^2 (strict), R^2 computed as R*R;
 *   - the grid is rebuilt from the snapshot of every iteration;
 *   - static detection needs the grid of t+1 to equal the grid of t, and
 *     treats an agent as disturbed if a changed agent (moved, grown,
 *     divided or created at t) had its position at t or at t+1 inside the
 *     agent's 27-box stencil;
 *   - growth/division: V += g*dt while V < V_div; an agent whose volume is
 *     >= V_div at the start of t divides after the displacement commit
 *     (daughters V/2, d = cbrt(6V/pi) correctly rounded, mother keeps its
 *     ID and moves by -(d'/4)u, the new agent goes to +(d'/4)u); new IDs are
 *     given in ascending parent-ID order while the count is below capacity;
 *   - boundaries: the space is the cube [bound_min, bound_max] on every
 *     axis.  Closed: every new position (displacement commit, daughter
 *     placement) is clamped into it per coordinate.  Toroidal: every new
 *     coordinate v is wrapped into [bound_min, bound_max): v - size when
 *     v >= bound_max, v + size when v < bound_min, and bound_min if
 *     rounding leaves it at bound_max; the grid tiles the space exactly with
 *     n = floor(size / L) >= 3 boxes per axis of length size / n from
 *     bound_min (n < 3 is an error), neighbour boxes wrap around, and the
 *     difference of two coordinates is taken as the minimum image: dx =
 *     x_i - x_j, then dx - size if dx > size / 2, dx + size if dx <
 *     -size / 2.  Open: the open-space rules above.  An agent pushed by a
 *     non-zero displacement counts as changed also when a wall stops it;
 *   - removal: m agents leave, n' = n - m remain; survivors with an ID
 *     below n' keep it, and the IDs below n' that removed agents held go,
 *     in ascending order, to the survivors with IDs >= n' in ascending
 *     order (the swaps of §5.3.2); every survivor then counts as changed for
 *     one iteration (the removed agents' neighbourhoods changed);
 *   - in-place execution context: an agent's new position is visible to
 *     the agents processed after it in the same iteration.  The thesis
 *     leaves the order to the scheduler; the order taken is: boxes by
 *     colour, then boxes of a colour in ascending box index, then the
 *     agents of a box in ascending ID.  The colour of a box is (c_x mod 2,
 *     c_y mod 2, c_z mod 2), except that on a toroidal axis with an odd
 *     number of boxes the last box of the axis has a third colour (it
 *     touches box 0 across the seam); colours are ranked x + k_x (y + k_y
 *     z), k_a = 2 or 3 colours per axis.  Boxes of one colour never lie in
 *     each other's 27-box stencil, so their order inside the colour does
 *     not matter.  Neighbours are the agents of the stencil in the grid of
 *     the iteration's start, at their current positions; an agent's force
 *     is summed over them in ascending ID and its displacement committed
 *     (under the boundary condition) before the next agent.  Static
 *     detection is not combined with it; growth and division follow the
 *     mechanics as in the copy context.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.141592653589793

typedef struct {
  double k, gamma, adherence, max_displacement, dt, box_length;
  double growth_rate, divide_volume;
  int32_t precision;     /* ignored: the oracle always computes in FP64 */
  int32_t detect_static;
  int32_t sort_interval; /* ignored: storage order never changes results */
  int32_t boundary;      /* 0 open, 1 closed, 2 toroidal (§4.4.11) */
  uint64_t seed;
  int64_t capacity;
  double bound_min, bound_max;  /* the space of closed and toroidal boundaries */
  int32_t execution_context;    /* 0 copy, 1 in-place (§5.2) */
  int32_t reserved;
} orc_params;

enum { ORC_OPEN = 0, ORC_CLOSED = 1, ORC_TORUS = 2 };
enum { ORC_COPY = 0, ORC_INPLACE = 1 };

/* A new coordinate under the boundary condition (§4.4.11). */
static double bound_apply(const orc_params *p, double v) {
  if (p->boundary == ORC_CLOSED) {
    if (v < p->bound_min) return p->bound_min;
    if (v > p->bound_max) return p->bound_max;
    return v;
  }
  if (p->boundary == ORC_TORUS) {
    const double size = p->bound_max - p->bound_min;
    if (v >= p->bound_max) v = v - size;
    else if (v < p->bound_min) v = v + size;
    if (v >= p->bound_max) v = p->bound_min;
    return v;
  }
  return v;
}

/* Coordinate difference a - b, as the minimum image on a torus. */
static double coord_diff(const orc_params *p, double a, double b) {
  double d = a - b;
  if (p && p->boundary == ORC_TORUS) {
    const double size = p->bound_max - p->bound_min, half = 0.5 * size;
    if (d > half) d = d - size;
    else if (d < -half) d = d + size;
  }
  return d;
}

/* ------------------------------------------------------------------------
 * Uniform grid (§4.4.3, §5.3.1).
 * ---------------------------------------------------------------------- */
typedef struct {
  double o[3];      /* origin: per-axis minimum of the agent centers */
  double L;         /* box length */
  int64_t dims[3];  /* boxes per axis: floor((max - o) / L) + 1 */
  int torus;        /* the grid tiles a toroidal space (neighbour boxes wrap) */
  int64_t n;
  int64_t *c;       /* box coordinates, 3 per agent */
  int64_t *box;     /* linear box index c_x + n_x (c_y + n_y c_z) */
  int64_t *sorted;  /* agent IDs ordered by (box, ID) */
  int64_t *sbox;    /* box of sorted[k] */
} grid_t;

typedef struct { int64_t box, id; } box_id_pair;

static int cmp_box_id(const void *a, const void *b) {
  const box_id_pair *p = (const box_id_pair *)a, *q = (const box_id_pair *)b;
  if (p->box != q->box) return p->box < q->box ? -1 : 1;
  if (p->id != q->id) return p->id < q->id ? -1 : 1;
  return 0;
}

static int cmp_i64(const void *a, const void *b) {
  int64_t p = *(const int64_t *)a, q = *(const int64_t *)b;
  return p < q ? -1 : (p > q ? 1 : 0);
}

static void grid_free(grid_t *g) {
  free(g->c); free(g->box); free(g->sorted); free(g->sbox);
  memset(g, 0, sizeof(*g));
}

/* Box length: the user's value, else the largest diameter (§4.4.3). */
static double grid_box_length(int64_t n, const double *d, double box_length) {
  if (box_length > 0.0) return box_length;
  double L = 0.0;
  for (int64_t i = 0; i < n; ++i) if (d[i] > L) L = d[i];
  return L;
}

/* Build the grid over the snapshot (x, y, z).  Open space: origin and
 * extent from the agents.  Toroidal space (bp->boundary): the space from
 * bound_min, n = floor(size / L) >= 3 boxes per axis of length size / n.
 * Returns 0 on success. */
static int grid_build(grid_t *g, int64_t n, const double *x, const double *y,
                      const double *z, double L, const orc_params *bp) {
  memset(g, 0, sizeof(*g));
  g->n = n;
  g->L = L;
  if (n == 0) { g->dims[0] = g->dims[1] = g->dims[2] = 0; return 0; }
  if (!(L > 0.0) || !isfinite(L)) return -1;
  const double *p[3] = {x, y, z};
  if (bp && bp->boundary == ORC_TORUS) {
    const double size = bp->bound_max - bp->bound_min;
    const double nb = floor(size / L);
    if (!(nb >= 3.0) || nb > 2097151.0) return -3;
    g->torus = 1;
    g->L = size / nb;
    for (int a = 0; a < 3; ++a) {
      g->o[a] = bp->bound_min;
      g->dims[a] = (int64_t)nb;
    }
  } else {
    double mx[3];
    for (int a = 0; a < 3; ++a) {
      g->o[a] = p[a][0];
      mx[a] = p[a][0];
      for (int64_t i = 1; i < n; ++i) {
        if (p[a][i] < g->o[a]) g->o[a] = p[a][i];
        if (p[a][i] > mx[a]) mx[a] = p[a][i];
      }
      g->dims[a] = (int64_t)floor((mx[a] - g->o[a]) / L) + 1;
    }
  }
  L = g->L;
  g->c = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)n);
  g->box = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  g->sorted = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  g->sbox = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  box_id_pair *tmp = (box_id_pair *)malloc(sizeof(box_id_pair) * (size_t)n);
  if (!g->c || !g->box || !g->sorted || !g->sbox || !tmp) { free(tmp); grid_free(g); return -2; }
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      int64_t c = (int64_t)floor((p[a][i] - g->o[a]) / L);
      if (g->torus) c = c < 0 ? 0 : (c >= g->dims[a] ? g->dims[a] - 1 : c);  /* rounding at the far face */
      g->c[3 * i + a] = c;
    }
    g->box[i] = g->c[3 * i] + g->dims[0] * (g->c[3 * i + 1] + g->dims[1] * g->c[3 * i + 2]);
    tmp[i].box = g->box[i];
    tmp[i].id = i;
  }
  qsort(tmp, (size_t)n, sizeof(box_id_pair), cmp_box_id);
  for (int64_t k = 0; k < n; ++k) { g->sorted[k] = tmp[k].id; g->sbox[k] = tmp[k].box; }
  free(tmp);
  return 0;
}

/* First index k with sbox[k] >= b. */
static int64_t grid_lower(const grid_t *g, int64_t b) {
  int64_t lo = 0, hi = g->n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (g->sbox[mid] < b) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* Growable list of agent IDs. */
typedef struct { int64_t *v; int64_t n, cap; } idlist;

static void idl_push(idlist *l, int64_t x) {
  if (l->n == l->cap) {
    l->cap = l->cap ? 2 * l->cap : 64;
    l->v = (int64_t *)realloc(l->v, sizeof(int64_t) * (size_t)l->cap);
  }
  l->v[l->n++] = x;
}

/* Stencil box (c + d) of a grid: 0 when it lies outside an open grid;
 * wrapped around on a torus. */
static int stencil_box(const grid_t *g, const int64_t *c, int dx, int dy, int dz, int64_t *b) {
  int64_t cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
  if (g->torus) {
    cx = (cx + g->dims[0]) % g->dims[0];
    cy = (cy + g->dims[1]) % g->dims[1];
    cz = (cz + g->dims[2]) % g->dims[2];
  } else if (cx < 0 || cy < 0 || cz < 0 || cx >= g->dims[0] || cy >= g->dims[1] || cz >= g->dims[2]) {
    return 0;
  }
  *b = cx + g->dims[0] * (cy + g->dims[1] * cz);
  return 1;
}

/* Candidates of agent i: every other agent in the (up to) 27 boxes around
 * i's box that lie inside the grid (§5.3.1; on a torus the 27 boxes wrap
 * around and are distinct, since every axis has at least 3 boxes), in
 * ascending ID order. */
static void grid_candidates(const grid_t *g, int64_t i, idlist *out) {
  out->n = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t b;
        if (!stencil_box(g, &g->c[3 * i], dx, dy, dz, &b)) continue;
        for (int64_t k = grid_lower(g, b); k < g->n && g->sbox[k] == b; ++k)
          if (g->sorted[k] != i) idl_push(out, g->sorted[k]);
      }
  qsort(out->v, (size_t)out->n, sizeof(int64_t), cmp_i64);
}

/* ------------------------------------------------------------------------
 * Pairwise quantities (Eq 4.1, Eq 4.2).
 * ---------------------------------------------------------------------- */
/* Squared center distance, summed as ((dx*dx + dy*dy) + dz*dz); on a
 * torus the differences are minimum images. */
static double sq_dist(const orc_params *p, const double *x, const double *y, const double *z, int64_t i,
                      int64_t j, double *dx, double *dy, double *dz) {
  *dx = coord_diff(p, x[i], x[j]);
  *dy = coord_diff(p, y[i], y[j]);
  *dz = coord_diff(p, z[i], z[j]);
  return ((*dx) * (*dx) + (*dy) * (*dy)) + (*dz) * (*dz);
}

/* Overlap delta = (r_i + r_j) - dist with r = 0.5 * d. */
static double overlap(const double *d, int64_t i, int64_t j, double dist) {
  return (0.5 * d[i] + 0.5 * d[j]) - dist;
}

/* Force on i from j.  Eq 4.2: r = r_i r_j / (r_i + r_j); Eq 4.1:
 * F_N = k delta - gamma sqrt(r delta), directed along (x_i - x_j)/dist
 * (positive F_N pushes i away from j).  Adds to F, counts non-zero F_N in
 * *nnz and adds k delta + gamma sqrt(r delta) to *smag (the magnitude sum
 * used to scale tolerances). */
static void pair_force(const orc_params *p, const double *x, const double *y, const double *z,
                       const double *d, int64_t i, int64_t j, double F[3], int32_t *nnz,
                       double *smag) {
  double dx, dy, dz;
  double s = sq_dist(p, x, y, z, i, j, &dx, &dy, &dz);
  double dist = sqrt(s);
  double delta = overlap(d, i, j, dist);
  if (!(delta > 0.0)) return;
  double ri = 0.5 * d[i], rj = 0.5 * d[j];
  double r = (ri * rj) / (ri + rj);
  double rep = p->k * delta;
  double adh = p->gamma * sqrt(r * delta);
  double fn = rep - adh;
  if (fn != 0.0) *nnz += 1;
  *smag += rep + adh;
  if (dist > 0.0) {
    F[0] += fn * (dx / dist);
    F[1] += fn * (dy / dist);
    F[2] += fn * (dz / dist);
  }
}

/* Displacement from the net force (reading of §4.5.1 / MechanicalForcesOp):
 * zero while |F| <= adherence, else dt*F with its norm clamped to the
 * maximum displacement. */
static void displacement(const orc_params *p, const double F[3], double D[3]) {
  double fn = sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
  D[0] = D[1] = D[2] = 0.0;
  if (!(fn > p->adherence)) return;
  D[0] = p->dt * F[0];
  D[1] = p->dt * F[1];
  D[2] = p->dt * F[2];
  double dn = sqrt((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2]);
  if (dn > p->max_displacement) {
    double s = p->max_displacement / dn;
    D[0] = D[0] * s;
    D[1] = D[1] * s;
    D[2] = D[2] * s;
  }
}

/* ------------------------------------------------------------------------
 * Correctly rounded cube root (diameter from volume).  A library cube root
 * gives the starting point; the result is then moved to the double nearest
 * to the exact cube root by comparing the cubes of the midpoints between
 * adjacent doubles with x in exact integer arithmetic.
 * ---------------------------------------------------------------------- */
typedef struct { uint64_t w[3]; } u192;

static u192 u192_of(uint64_t a) { u192 r = {{a, 0, 0}}; return r; }

static u192 u192_mul(u192 a, uint64_t b) {
  u192 r;
  unsigned __int128 carry = 0;
  for (int k = 0; k < 3; ++k) {
    unsigned __int128 t = (unsigned __int128)a.w[k] * b + carry;
    r.w[k] = (uint64_t)t;
    carry = t >> 64;
  }
  return r;
}

static int u192_bits(u192 a) {
  for (int k = 2; k >= 0; --k)
    if (a.w[k]) return 64 * k + 64 - __builtin_clzll(a.w[k]);
  return 0;
}

static u192 u192_shl(u192 a, int s) {
  u192 r = {{0, 0, 0}};
  int q = s / 64, m = s % 64;
  for (int k = 2; k >= 0; --k) {
    int src = k - q;
    if (src < 0) continue;
    uint64_t v = a.w[src] << m;
    if (m && src - 1 >= 0) v |= a.w[src - 1] >> (64 - m);
    r.w[k] = v;
  }
  return r;
}

static int u192_cmp(u192 a, u192 b) {
  for (int k = 2; k >= 0; --k)
    if (a.w[k] != b.w[k]) return a.w[k] < b.w[k] ? -1 : 1;
  return 0;
}

/* Sign of M^3 2^(3e) - X 2^ex for positive integers M < 2^56, X < 2^54. */
static int cmp_cube(uint64_t M, int e, uint64_t X, int ex) {
  u192 c = u192_mul(u192_mul(u192_of(M), M), M);
  u192 xx = u192_of(X);
  int s = 3 * e - ex;
  if (s >= 0) {
    if (u192_bits(c) + s > 190) return 1;
    c = u192_shl(c, s);
  } else {
    if (u192_bits(xx) - s > 190) return -1;
    xx = u192_shl(xx, -s);
  }
  return u192_cmp(c, xx);
}

/* v = M 2^e with integer M (positive finite v). */
static void split_double(double v, uint64_t *M, int *e) {
  uint64_t b;
  memcpy(&b, &v, 8);
  int E = (int)((b >> 52) & 0x7ff);
  uint64_t f = b & ((1ULL << 52) - 1);
  if (E == 0) { *M = f; *e = -1074; }
  else { *M = f | (1ULL << 52); *e = E - 1075; }
}

/* Midpoint of two adjacent positive doubles a < b as M 2^e. */
static void midpoint(double a, double b, uint64_t *M, int *e) {
  uint64_t Ma, Mb;
  int ea, eb;
  split_double(a, &Ma, &ea);
  split_double(b, &Mb, &eb);
  int m = ea < eb ? ea : eb;
  *M = (Ma << (ea - m)) + (Mb << (eb - m));
  *e = m - 1;
}

double orc_cbrt_rn(double x) {
  if (!(x > 0.0) || isinf(x)) return cbrt(x);
  uint64_t X;
  int ex;
  split_double(x, &X, &ex);
  double y = cbrt(x);
  for (int it = 0; it < 16; ++it) {
    uint64_t M;
    int e;
    double up = nextafter(y, INFINITY);
    midpoint(y, up, &M, &e);
    if (cmp_cube(M, e, X, ex) < 0) { y = up; continue; }
    double dn = nextafter(y, 0.0);
    if (dn > 0.0) {
      midpoint(dn, y, &M, &e);
      if (cmp_cube(M, e, X, ex) > 0) { y = dn; continue; }
    }
    break;
  }
  return y;
}

/* Diameter of a sphere of volume V and volume of a sphere of diameter d. */
static double diameter_of_volume(double V) { return orc_cbrt_rn((6.0 * V) / ORC_PI); }
static double volume_of_diameter(double d) { return (ORC_PI * ((d * d) * d)) / 6.0; }

double orc_diameter_of_volume(double V) { return diameter_of_volume(V); }
double orc_volume_of_diameter(double d) { return volume_of_diameter(d); }

/* ------------------------------------------------------------------------
 * Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), the per-agent
 * counter-based generator proposed in §7.1.4 for reproducible simulations.
 * ---------------------------------------------------------------------- */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    unsigned __int128 p0 = (unsigned __int128)M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Division axis of agent `id` at iteration t: rejection-sample a point of
 * [-1,1)^3 from 53-bit uniforms (counter {id, t, attempt, 0}, key
 * {seed, 0}), accept when 1e-6 < |p|^2 <= 1, and normalise. */
void orc_division_axis(uint64_t seed, int64_t id, int64_t t, double u[3]) {
  for (uint64_t k = 0; k < 1000000; ++k) {
    uint64_t ctr[4] = {(uint64_t)id, (uint64_t)t, k, 0}, key[2] = {seed, 0}, w[4];
    orc_philox4x64_10(ctr, key, w);
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = 2.0 * ((double)(w[a] >> 11) * 0x1.0p-53) - 1.0;
    double s = (p[0] * p[0] + p[1] * p[1]) + p[2] * p[2];
    if (s > 1e-6 && s <= 1.0) {
      double r = sqrt(s);
      u[0] = p[0] / r;
      u[1] = p[1] / r;
      u[2] = p[2] / r;
      return;
    }
  }
  u[0] = 1.0; u[1] = 0.0; u[2] = 0.0;
}

/* ------------------------------------------------------------------------
 * Simulation state (ID order) and one iteration.
 * ---------------------------------------------------------------------- */
typedef struct orc_sim {
  orc_params p;
  int64_t n, cap;
  double *x, *y, *z, *d, *v;
  double *F;            /* force of the last iteration (0 for static agents) */
  double *D;            /* displacement of the last iteration */
  int32_t *nnz;         /* non-zero pair forces of the last evaluation */
  uint8_t *changed;     /* moved, grown, divided or created in the last iteration */
  uint8_t *stat;        /* static in the last iteration */
  int64_t *prev_box;    /* box of each agent in the last iteration's grid */
  int have_prev;
  double prev_o[3], prev_L;
  int64_t prev_dims[3];
  int64_t t;
} orc_sim;

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->x); free(s->y); free(s->z); free(s->d); free(s->v);
  free(s->F); free(s->D); free(s->nnz); free(s->changed); free(s->stat); free(s->prev_box);
  free(s);
}

/* A position inside the space of a closed ([min, max]) or toroidal
 * ([min, max)) boundary; any finite position in open space. */
static int inside_space(const orc_params *p, double v) {
  if (!isfinite(v)) return 0;
  if (p->boundary == ORC_CLOSED) return v >= p->bound_min && v <= p->bound_max;
  if (p->boundary == ORC_TORUS) return v >= p->bound_min && v < p->bound_max;
  return 1;
}

orc_sim *orc_create(const orc_params *p, int64_t n, const double *xyz, const double *d) {
  if (n < 0) return NULL;
  if (p->boundary < ORC_OPEN || p->boundary > ORC_TORUS) return NULL;
  if (p->execution_context != ORC_COPY && p->execution_context != ORC_INPLACE) return NULL;
  if (p->execution_context == ORC_INPLACE && p->detect_static) return NULL;
  if (p->boundary != ORC_OPEN &&
      !(isfinite(p->bound_min) && isfinite(p->bound_max) && p->bound_min < p->bound_max))
    return NULL;
  int64_t cap = p->capacity > n ? p->capacity : n;
  if (cap < 1) cap = 1;
  for (int64_t i = 0; i < n; ++i) {
    if (!inside_space(p, xyz[3 * i]) || !inside_space(p, xyz[3 * i + 1]) || !inside_space(p, xyz[3 * i + 2]))
      return NULL;
    if (!(d[i] > 0.0) || !isfinite(d[i])) return NULL;
  }
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  if (!s) return NULL;
  s->p = *p;
  s->n = n;
  s->cap = cap;
  size_t c = (size_t)cap;
  s->x = (double *)calloc(c, 8); s->y = (double *)calloc(c, 8); s->z = (double *)calloc(c, 8);
  s->d = (double *)calloc(c, 8); s->v = (double *)calloc(c, 8);
  s->F = (double *)calloc(3 * c, 8); s->D = (double *)calloc(3 * c, 8);
  s->nnz = (int32_t *)calloc(c, 4);
  s->changed = (uint8_t *)calloc(c, 1); s->stat = (uint8_t *)calloc(c, 1);
  s->prev_box = (int64_t *)calloc(c, 8);
  if (!s->x || !s->y || !s->z || !s->d || !s->v || !s->F || !s->D || !s->nnz || !s->changed ||
      !s->stat || !s->prev_box) { orc_destroy(s); return NULL; }
  for (int64_t i = 0; i < n; ++i) {
    s->x[i] = xyz[3 * i]; s->y[i] = xyz[3 * i + 1]; s->z[i] = xyz[3 * i + 2];
    s->d[i] = d[i];
    s->v[i] = volume_of_diameter(d[i]);
    s->changed[i] = 1;  /* new agents: nothing is known about them yet */
  }
  return s;
}

int64_t orc_count(const orc_sim *s) { return s->n; }
int64_t orc_iteration(const orc_sim *s) { return s->t; }

void orc_get(const orc_sim *s, double *xyz, double *d, double *v) {
  for (int64_t i = 0; i < s->n; ++i) {
    if (xyz) { xyz[3 * i] = s->x[i]; xyz[3 * i + 1] = s->y[i]; xyz[3 * i + 2] = s->z[i]; }
    if (d) d[i] = s->d[i];
    if (v) v[i] = s->v[i];
  }
}

/* Per-agent record of the last iteration. */
void orc_last(const orc_sim *s, double *F, double *D, int32_t *nnz, uint8_t *stat, uint8_t *changed) {
  for (int64_t i = 0; i < s->n; ++i) {
    if (F) for (int a = 0; a < 3; ++a) F[3 * i + a] = s->F[3 * i + a];
    if (D) for (int a = 0; a < 3; ++a) D[3 * i + a] = s->D[3 * i + a];
    if (nnz) nnz[i] = s->nnz[i];
    if (stat) stat[i] = s->stat[i];
    if (changed) changed[i] = s->changed[i];
  }
}

/* Grid of the current snapshot: box index per agent, origin and box length,
 * boxes per axis. */
int orc_grid(const orc_sim *s, int64_t *box, double origin_len[4], int64_t dims[3]) {
  grid_t g;
  double L = grid_box_length(s->n, s->d, s->p.box_length);
  int rc = grid_build(&g, s->n, s->x, s->y, s->z, L, &s->p);
  if (rc) return rc;
  if (box) for (int64_t i = 0; i < s->n; ++i) box[i] = g.box[i];
  if (origin_len) { origin_len[0] = g.o[0]; origin_len[1] = g.o[1]; origin_len[2] = g.o[2]; origin_len[3] = g.L; }
  if (dims) { dims[0] = g.dims[0]; dims[1] = g.dims[1]; dims[2] = g.dims[2]; }
  grid_free(&g);
  return 0;
}

/* Net force, non-zero pair count and magnitude sum of the agents `ids`
 * (all agents in ID order when ids == NULL) from the current snapshot,
 * evaluated for every agent (no static skipping). */
int orc_forces(const orc_sim *s, const int64_t *ids, int64_t m, double *F, int32_t *nnz, double *smag) {
  grid_t g;
  double L = grid_box_length(s->n, s->d, s->p.box_length);
  int rc = grid_build(&g, s->n, s->x, s->y, s->z, L, &s->p);
  if (rc) return rc;
  idlist cand = {0, 0, 0};
  int64_t count = ids ? m : s->n;
  for (int64_t q = 0; q < count; ++q) {
    int64_t i = ids ? ids[q] : q;
    double f[3] = {0.0, 0.0, 0.0}, sm = 0.0;
    int32_t nz = 0;
    if (i >= 0 && i < s->n) {
      grid_candidates(&g, i, &cand);
      for (int64_t k = 0; k < cand.n; ++k)
        pair_force(&s->p, s->x, s->y, s->z, s->d, i, cand.v[k], f, &nz, &sm);
    }
    if (F) { F[3 * q] = f[0]; F[3 * q + 1] = f[1]; F[3 * q + 2] = f[2]; }
    if (nnz) nnz[q] = nz;
    if (smag) smag[q] = sm;
  }
  free(cand.v);
  grid_free(&g);
  return 0;
}

static int box_in_sorted(const int64_t *v, int64_t n, int64_t b) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (v[mid] < b) lo = mid + 1; else hi = mid;
  }
  return lo < n && v[lo] == b;
}

/* Colour of box coordinates c in the in-place order (k[a] colours per axis). */
static int box_colour(const grid_t *g, const int64_t *c, const int *k) {
  int col[3];
  for (int a = 0; a < 3; ++a)
    col[a] = (k[a] == 3 && c[a] == g->dims[a] - 1) ? 2 : (int)(c[a] % 2);
  return col[0] + k[0] * (col[1] + k[1] * col[2]);
}

/* Forces and displacements under the in-place execution context (§5.2):
 * boxes by colour, boxes of a colour in ascending index, agents of a box in
 * ascending ID; each agent's force from the current positions of the agents
 * of its stencil in the grid g of the iteration's start, its displacement
 * committed at once. */
static void inplace_mechanics(orc_sim *s, const grid_t *g) {
  const orc_params *p = &s->p;
  const int64_t n = s->n;
  int k[3];
  for (int a = 0; a < 3; ++a) k[a] = (g->torus && (g->dims[a] % 2) == 1) ? 3 : 2;
  const int ncol = k[0] * k[1] * k[2];
  idlist cand = {0, 0, 0};
  for (int col = 0; col < ncol; ++col) {
    /* g->sorted lists the agents by (box, ID), boxes in ascending index */
    for (int64_t q = 0; q < n; ++q) {
      const int64_t i = g->sorted[q];
      if (box_colour(g, &g->c[3 * i], k) != col) continue;
      double f[3] = {0.0, 0.0, 0.0}, sm = 0.0;
      int32_t nz = 0;
      grid_candidates(g, i, &cand);
      for (int64_t m = 0; m < cand.n; ++m) pair_force(p, s->x, s->y, s->z, s->d, i, cand.v[m], f, &nz, &sm);
      s->F[3 * i] = f[0]; s->F[3 * i + 1] = f[1]; s->F[3 * i + 2] = f[2];
      s->nnz[i] = nz;
      double *D = &s->D[3 * i];
      displacement(p, f, D);
      s->x[i] = bound_apply(p, s->x[i] + D[0]);
      s->y[i] = bound_apply(p, s->y[i] + D[1]);
      s->z[i] = bound_apply(p, s->z[i] + D[2]);
      s->changed[i] = (uint8_t)(D[0] != 0.0 || D[1] != 0.0 || D[2] != 0.0);
      s->stat[i] = 0;
      s->prev_box[i] = g->box[i];
    }
  }
  free(cand.v);
}

/* One iteration (§5.2 Algorithm 8 under the copy execution context, or the
 * in-place one). */
static int orc_iterate(orc_sim *s) {
  const orc_params *p = &s->p;
  int64_t n = s->n;
  grid_t g;
  double L = grid_box_length(n, s->d, p->box_length);
  int rc = grid_build(&g, n, s->x, s->y, s->z, L, p);
  if (rc) return rc;

  /* Static detection (§5.5): the conditions must have held in the last
   * iteration.  Agents that changed at t-1 disturb every box that holds
   * their position of t-1 or of t. */
  uint8_t *stat = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  int same_grid = s->have_prev && g.o[0] == s->prev_o[0] && g.o[1] == s->prev_o[1] &&
                  g.o[2] == s->prev_o[2] && g.L == s->prev_L && g.dims[0] == s->prev_dims[0] &&
                  g.dims[1] == s->prev_dims[1] && g.dims[2] == s->prev_dims[2];
  if (p->detect_static && same_grid && n > 0) {
    int64_t *dirty = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)n);
    int64_t nd = 0;
    for (int64_t j = 0; j < n; ++j)
      if (s->changed[j]) { dirty[nd++] = g.box[j]; dirty[nd++] = s->prev_box[j]; }
    qsort(dirty, (size_t)nd, sizeof(int64_t), cmp_i64);
    for (int64_t i = 0; i < n; ++i) {
      if (s->changed[i] || s->nnz[i] > 1) continue;
      int disturbed = 0;
      for (int dz = -1; dz <= 1 && !disturbed; ++dz)
        for (int dy = -1; dy <= 1 && !disturbed; ++dy)
          for (int dx = -1; dx <= 1 && !disturbed; ++dx) {
            int64_t b;
            if (!stencil_box(&g, &g.c[3 * i], dx, dy, dz, &b)) continue;
            if (box_in_sorted(dirty, nd, b)) disturbed = 1;
          }
      stat[i] = (uint8_t)!disturbed;
    }
    free(dirty);
  }

  if (p->execution_context == ORC_INPLACE) {
    inplace_mechanics(s, &g);
  } else {
    /* Forces and displacements from the snapshot. */
    idlist cand = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
      double f[3] = {0.0, 0.0, 0.0}, sm = 0.0;
      if (stat[i]) {
        s->D[3 * i] = s->D[3 * i + 1] = s->D[3 * i + 2] = 0.0;
        s->F[3 * i] = s->F[3 * i + 1] = s->F[3 * i + 2] = 0.0;
        continue;  /* static: keeps its nnz, does not move */
      }
      int32_t nz = 0;
      grid_candidates(&g, i, &cand);
      for (int64_t k = 0; k < cand.n; ++k) pair_force(p, s->x, s->y, s->z, s->d, i, cand.v[k], f, &nz, &sm);
      s->F[3 * i] = f[0]; s->F[3 * i + 1] = f[1]; s->F[3 * i + 2] = f[2];
      s->nnz[i] = nz;
      displacement(p, f, &s->D[3 * i]);
    }
    free(cand.v);

    /* Commit (copy execution context), under the boundary condition. */
    for (int64_t i = 0; i < n; ++i) {
      s->x[i] = bound_apply(p, s->x[i] + s->D[3 * i]);
      s->y[i] = bound_apply(p, s->y[i] + s->D[3 * i + 1]);
      s->z[i] = bound_apply(p, s->z[i] + s->D[3 * i + 2]);
      s->changed[i] = (uint8_t)(s->D[3 * i] != 0.0 || s->D[3 * i + 1] != 0.0 || s->D[3 * i + 2] != 0.0);
      s->stat[i] = stat[i];
      s->prev_box[i] = g.box[i];
    }
  }
  free(stat);

  /* Growth and division (GrowthDivision; new agents visible next
   * iteration, §5.2). */
  if (p->growth_rate > 0.0 && p->divide_volume > 0.0) {
    double dv = p->growth_rate * p->dt;
    int64_t n0 = n;
    for (int64_t i = 0; i < n0; ++i) {
      if (s->v[i] < p->divide_volume) {
        s->v[i] = s->v[i] + dv;
        s->d[i] = diameter_of_volume(s->v[i]);
        s->changed[i] = 1;
      } else if (s->n < s->cap) {
        double vh = 0.5 * s->v[i];
        double dh = diameter_of_volume(vh);
        double u[3];
        orc_division_axis(p->seed, i, s->t, u);
        double off = 0.25 * dh;
        int64_t j = s->n++;
        s->x[j] = bound_apply(p, s->x[i] + off * u[0]);
        s->y[j] = bound_apply(p, s->y[i] + off * u[1]);
        s->z[j] = bound_apply(p, s->z[i] + off * u[2]);
        s->x[i] = bound_apply(p, s->x[i] - off * u[0]);
        s->y[i] = bound_apply(p, s->y[i] - off * u[1]);
        s->z[i] = bound_apply(p, s->z[i] - off * u[2]);
        s->v[i] = vh; s->v[j] = vh;
        s->d[i] = dh; s->d[j] = dh;
        s->changed[i] = 1; s->changed[j] = 1;
        s->nnz[j] = 0; s->stat[j] = 0;
        s->F[3 * j] = s->F[3 * j + 1] = s->F[3 * j + 2] = 0.0;
        s->D[3 * j] = s->D[3 * j + 1] = s->D[3 * j + 2] = 0.0;
        /* The new agent was never in a grid: its "previous box" is its
         * mother's, which lies in the same or a neighboring box. */
        s->prev_box[j] = g.box[i];
      }
    }
  }

  s->have_prev = 1;
  s->prev_o[0] = g.o[0]; s->prev_o[1] = g.o[1]; s->prev_o[2] = g.o[2];
  s->prev_L = g.L;
  s->prev_dims[0] = g.dims[0]; s->prev_dims[1] = g.dims[1]; s->prev_dims[2] = g.dims[2];
  s->t += 1;
  grid_free(&g);
  return 0;
}

/* Remove the m agents `ids` (distinct, in range; returns -1 otherwise and
 * changes nothing).  The swaps of §5.3.2 (Fig 5.1): with n' = n - m, a
 * removed agent below n' leaves a hole, and the holes, in ascending order,
 * take the survivors at or above n', in ascending order; agents below n'
 * that survive keep their ID.  Every survivor counts as changed for the
 * next iteration. */
int orc_remove(orc_sim *s, int64_t m, const int64_t *ids) {
  int64_t n = s->n;
  if (m < 0 || m > n) return -1;
  uint8_t *gone = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t k = 0; k < m; ++k) {
    if (ids[k] < 0 || ids[k] >= n || gone[ids[k]]) { free(gone); return -1; }
    gone[ids[k]] = 1;
  }
  const int64_t nn = n - m;
  int64_t hole = 0, mover = nn;
  for (;;) {
    while (hole < nn && !gone[hole]) ++hole;
    while (mover < n && gone[mover]) ++mover;
    if (hole >= nn || mover >= n) break;
    /* the survivor `mover` takes the ID `hole` */
    s->x[hole] = s->x[mover]; s->y[hole] = s->y[mover]; s->z[hole] = s->z[mover];
    s->d[hole] = s->d[mover]; s->v[hole] = s->v[mover];
    for (int a = 0; a < 3; ++a) { s->F[3 * hole + a] = s->F[3 * mover + a]; s->D[3 * hole + a] = s->D[3 * mover + a]; }
    s->nnz[hole] = s->nnz[mover];
    s->stat[hole] = s->stat[mover];
    s->prev_box[hole] = s->prev_box[mover];
    ++hole;
    ++mover;
  }
  s->n = nn;
  for (int64_t i = 0; i < nn; ++i) s->changed[i] = 1;
  free(gone);
  return 0;
}

/* New positions of the current agents (xyz by ID, n x 3), as an operation
 * after the mechanical step of an iteration (chemotaxis): an agent whose
 * position changes counts as changed for static detection; its box of the
 * last grid stays.  Returns -1 (nothing changed) on a position outside the
 * space of a closed or toroidal boundary. */
int orc_set_positions(orc_sim *s, const double *xyz) {
  for (int64_t i = 0; i < s->n; ++i)
    for (int a = 0; a < 3; ++a)
      if (!inside_space(&s->p, xyz[3 * i + a])) return -1;
  for (int64_t i = 0; i < s->n; ++i) {
    const double nx = xyz[3 * i], ny = xyz[3 * i + 1], nz = xyz[3 * i + 2];
    if (nx != s->x[i] || ny != s->y[i] || nz != s->z[i]) {
      s->x[i] = nx; s->y[i] = ny; s->z[i] = nz;
      s->changed[i] = 1;
    }
  }
  return 0;
}

int orc_step(orc_sim *s, int32_t iterations) {
  for (int32_t it = 0; it < iterations; ++it) {
    int rc = orc_iterate(s);
    if (rc) return rc;
  }
  return 0;
}

/* ------------------------------------------------------------------------
 * Neighbor queries (§4.4.3 ForEachNeighbor, tutorial "environment"):
 * unordered pairs {i, j}, i < j, in ascending (i, j) order.  radius >= 0:
 * dist^2 < radius^2; radius < 0: overlapping pairs (delta > 0).  A radius
 * above the box length uses a grid whose box length is the radius.
 * Returns the number of pairs; writes at most `cap` of them.
 * ---------------------------------------------------------------------- */
int64_t orc_neighbors(const orc_sim *s, double radius, int64_t cap, int64_t *pairs) {
  grid_t g;
  double L = grid_box_length(s->n, s->d, s->p.box_length);
  if (radius > L) L = radius;
  if (grid_build(&g, s->n, s->x, s->y, s->z, L, &s->p)) return -1;
  double R2 = radius * radius;
  idlist cand = {0, 0, 0};
  int64_t count = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    grid_candidates(&g, i, &cand);
    for (int64_t k = 0; k < cand.n; ++k) {
      int64_t j = cand.v[k];
      if (j <= i) continue;
      double dx, dy, dz;
      double sq = sq_dist(&s->p, s->x, s->y, s->z, i, j, &dx, &dy, &dz);
      int hit = radius >= 0.0 ? (sq < R2) : (overlap(s->d, i, j, sqrt(sq)) > 0.0);
      if (!hit) continue;
      if (count < cap && pairs) { pairs[2 * count] = i; pairs[2 * count + 1] = j; }
      count++;
    }
  }
  free(cand.v);
  grid_free(&g);
  return count;
}

/* ------------------------------------------------------------------------
 * Morton order (§5.4.2, Fig 5.4).
 * ---------------------------------------------------------------------- */
/* Interleave box coordinates: bit b of axis a goes to bit b*dim + a
 * (x is the least significant, Fig 5.4C). */
uint64_t orc_interleave(int dim, const int64_t *c) {
  uint64_t code = 0;
  for (int b = 0; b < 64 / dim; ++b)
    for (int a = 0; a < dim; ++a)
      code |= (uint64_t)((c[a] >> b) & 1) << (b * dim + a);
  return code;
}

typedef struct {
  int dim;
  const int64_t *dims;
  int64_t counter, offset;
  int found_gap;
  int64_t n, cap;
  int64_t *out_counter, *out_offset;
} gap_state;

/* Depth-first traversal of the implicit 2^dim-ary tree over the
 * power-of-two cube of side `size` at corner `lo` (Fig 5.4D). */
static void gap_visit(gap_state *st, const int64_t *lo, int64_t size) {
  int empty = 0, complete = 1;
  for (int a = 0; a < st->dim; ++a) {
    if (lo[a] >= st->dims[a]) empty = 1;
    if (lo[a] + size > st->dims[a]) complete = 0;
  }
  int64_t leaves = 1;
  for (int a = 0; a < st->dim; ++a) leaves *= size;
  if (empty) {
    st->offset += leaves;
    st->found_gap = 1;
    return;
  }
  if (complete) {
    if (st->found_gap) {
      if (st->n < st->cap) { st->out_counter[st->n] = st->counter; st->out_offset[st->n] = st->offset; }
      st->n++;
      st->found_gap = 0;
    }
    st->counter += leaves;
    return;
  }
  int64_t half = size / 2;
  for (int child = 0; child < (1 << st->dim); ++child) {
    int64_t clo[3];
    for (int a = 0; a < st->dim; ++a) clo[a] = lo[a] + (((child >> a) & 1) ? half : 0);
    gap_visit(st, clo, half);
  }
}

/* Gap table of a dim-dimensional grid: entries (box counter, offset) such
 * that the k-th box in Morton order has code k + offset of the last entry
 * whose counter <= k.  Returns the number of entries. */
int64_t orc_morton_gaps(int dim, const int64_t *dims, int64_t cap, int64_t *counter, int64_t *offset) {
  int64_t mx = 1;
  for (int a = 0; a < dim; ++a) {
    if (dims[a] <= 0) return 0;
    if (dims[a] > mx) mx = dims[a];
  }
  int64_t size = 1;
  while (size < mx) size *= 2;
  gap_state st = {dim, dims, 0, 0, 1, 0, cap, counter, offset};
  int64_t lo[3] = {0, 0, 0};
  gap_visit(&st, lo, size);
  return st.n;
}

/* Morton codes of all boxes of the grid, in Morton order (Fig 5.4E). */
int64_t orc_morton_sequence(int dim, const int64_t *dims, int64_t *codes) {
  int64_t nb = 1;
  for (int a = 0; a < dim; ++a) nb *= dims[a];
  int64_t ng = orc_morton_gaps(dim, dims, 0, NULL, NULL);
  int64_t *gc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng > 0 ? ng : 1));
  int64_t *go = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng > 0 ? ng : 1));
  orc_morton_gaps(dim, dims, ng, gc, go);
  int64_t e = 0;
  for (int64_t k = 0; k < nb; ++k) {
    while (e + 1 < ng && gc[e + 1] <= k) e++;
    codes[k] = k + go[e];
  }
  free(gc);
  free(go);
  return nb;
}

/* Agents of the current snapshot in Morton order of their grid box, ties
 * by ID (§5.4.2: agents stored in increasing Morton order of their box).
 * Written as its plain definition, a sort by (interleaved code, ID); the
 * gap algorithm above is checked to enumerate the same box order. */
int orc_morton_agent_order(const orc_sim *s, int64_t *ids) {
  grid_t g;
  double L = grid_box_length(s->n, s->d, s->p.box_length);
  int rc = grid_build(&g, s->n, s->x, s->y, s->z, L, &s->p);
  if (rc) return rc;
  box_id_pair *tmp = (box_id_pair *)malloc(sizeof(box_id_pair) * (size_t)(s->n > 0 ? s->n : 1));
  for (int64_t i = 0; i < s->n; ++i) {
    tmp[i].box = (int64_t)orc_interleave(3, &g.c[3 * i]);
    tmp[i].id = i;
  }
  qsort(tmp, (size_t)s->n, sizeof(box_id_pair), cmp_box_id);
  for (int64_t i = 0; i < s->n; ++i) ids[i] = tmp[i].id;
  free(tmp);
  grid_free(&g);
  return 0;
}
