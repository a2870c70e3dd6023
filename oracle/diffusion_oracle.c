/*
 * diffusion_oracle.c -- plain, single-threaded FP64 CPU oracle of the
 * soma-clustering slice of the BioDynaMo thesis (arXiv 2503.10796):
 * extracellular diffusion (§4.5.2, Eq 4.3), substance secretion
 * (Algorithm 6) and chemotaxis (Algorithm 7).
 *
 * TEST INFRASTRUCTURE ONLY, like bdm_oracle.c: only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it, and it
 * shares no code with the CUDA path.  Compiled with -O2 -ffp-contract=off.
 *
 * The diffusion grid: n[0] x n[1] x n[2] points, point (i, j, k) stored at
 * i + n0 (j + n1 k).  Point (i, j, k) stands for the box
 * [lo + (i, j, k) h, lo + (i + 1, j + 1, k + 1) h); a position belongs to
 * the box floor((x - lo) / h) per axis (IEEE FP64 subtraction, division
 * and floor).
 *
 * Readings taken where the thesis is silent or leaves a choice (each one is
 * listed with the design notes of the repository):
 *   - boundary: substances diffuse out of the space (§4.5.2), read as a
 *     concentration of zero at every point outside the grid;
 *   - Eq 4.3 is evaluated term by term in the order it is printed:
 *     u (1 - mu dt) + cx (u[i+1] - 2u + u[i-1]) + cy (...) + cz (...), with
 *     cx = nu dt / hx^2 computed as (nu * dt) / (hx * hx), and
 *     u[i+1] - 2u + u[i-1] as (u[i+1] - 2u) + u[i-1];
 *   - secretion (Algorithm 6) adds the quantity to the box that holds the
 *     agent's center, agents in ascending ID order; agents outside the
 *     grid secrete nothing;
 *   - the gradient at a box is the central difference of its neighbours,
 *     (u[i+1] - u[i-1]) / (2 h) per axis (zero outside the grid); the
 *     normalized gradient is g / |g| with |g| = sqrt((gx gx + gy gy) +
 *     gz gz), and zero where |g| = 0;
 *   - chemotaxis (Algorithm 7) moves every agent inside the grid by
 *     weight * normalized gradient of its box, all agents reading the same
 *     grid; agents outside do not move.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int64_t point_index(const int64_t n[3], int64_t i, int64_t j, int64_t k) {
  return i + n[0] * (j + n[1] * k);
}

/* Concentration at (i, j, k), zero outside the grid. */
static double value_at(const double *u, const int64_t n[3], int64_t i, int64_t j, int64_t k) {
  if (i < 0 || j < 0 || k < 0 || i >= n[0] || j >= n[1] || k >= n[2]) return 0.0;
  return u[point_index(n, i, j, k)];
}

/* Box of a position, 0 when it lies inside the grid, -1 otherwise. */
static int box_of(const double lo[3], const double h[3], const int64_t n[3], const double x[3], int64_t b[3]) {
  for (int a = 0; a < 3; ++a) {
    double q = floor((x[a] - lo[a]) / h[a]);
    if (!(q >= 0.0) || !(q < (double)n[a])) return -1;
    b[a] = (int64_t)q;
  }
  return 0;
}

/* Eq 4.3: `steps` explicit time steps of the grid u in place. */
int orc_diffuse(const int64_t n[3], const double h[3], double nu, double mu, double dt, int32_t steps,
                double *u) {
  if (n[0] < 1 || n[1] < 1 || n[2] < 1 || steps < 0) return -1;
  const int64_t total = n[0] * n[1] * n[2];
  double *next = (double *)malloc(sizeof(double) * (size_t)total);
  if (!next) return -2;
  const double keep = 1.0 - mu * dt;
  const double cx = (nu * dt) / (h[0] * h[0]);
  const double cy = (nu * dt) / (h[1] * h[1]);
  const double cz = (nu * dt) / (h[2] * h[2]);
  for (int32_t s = 0; s < steps; ++s) {
    for (int64_t k = 0; k < n[2]; ++k)
      for (int64_t j = 0; j < n[1]; ++j)
        for (int64_t i = 0; i < n[0]; ++i) {
          const double c = value_at(u, n, i, j, k);
          const double lx = (value_at(u, n, i + 1, j, k) - 2.0 * c) + value_at(u, n, i - 1, j, k);
          const double ly = (value_at(u, n, i, j + 1, k) - 2.0 * c) + value_at(u, n, i, j - 1, k);
          const double lz = (value_at(u, n, i, j, k + 1) - 2.0 * c) + value_at(u, n, i, j, k - 1);
          next[point_index(n, i, j, k)] = ((c * keep + cx * lx) + cy * ly) + cz * lz;
        }
    memcpy(u, next, sizeof(double) * (size_t)total);
  }
  free(next);
  return 0;
}

/* Algorithm 6: every agent inside the grid adds `quantity` to its box, in
 * ascending ID order.  xyz: n x 3. */
int orc_secrete(const double lo[3], const double h[3], const int64_t ng[3], double *u, int64_t n,
                const double *xyz, double quantity) {
  for (int64_t id = 0; id < n; ++id) {
    int64_t b[3];
    if (box_of(lo, h, ng, xyz + 3 * id, b)) continue;
    u[point_index(ng, b[0], b[1], b[2])] += quantity;
  }
  return 0;
}

/* Normalized central-difference gradient of box b. */
static void normalized_gradient(const double h[3], const int64_t ng[3], const double *u, const int64_t b[3],
                                double g[3]) {
  const int64_t i = b[0], j = b[1], k = b[2];
  g[0] = (value_at(u, ng, i + 1, j, k) - value_at(u, ng, i - 1, j, k)) / (2.0 * h[0]);
  g[1] = (value_at(u, ng, i, j + 1, k) - value_at(u, ng, i, j - 1, k)) / (2.0 * h[1]);
  g[2] = (value_at(u, ng, i, j, k + 1) - value_at(u, ng, i, j, k - 1)) / (2.0 * h[2]);
  const double norm = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
  for (int a = 0; a < 3; ++a) g[a] = norm > 0.0 ? g[a] / norm : 0.0;
}

/* The normalized gradient at each of n positions (zero outside the grid). */
int orc_gradient(const double lo[3], const double h[3], const int64_t ng[3], const double *u, int64_t n,
                 const double *xyz, double *grad) {
  for (int64_t id = 0; id < n; ++id) {
    int64_t b[3];
    double g[3] = {0.0, 0.0, 0.0};
    if (!box_of(lo, h, ng, xyz + 3 * id, b)) normalized_gradient(h, ng, u, b, g);
    grad[3 * id] = g[0];
    grad[3 * id + 1] = g[1];
    grad[3 * id + 2] = g[2];
  }
  return 0;
}

/* Algorithm 7: every agent inside the grid moves by weight times the
 * normalized gradient of its box; the grid is read, not changed. */
int orc_chemotaxis(const double lo[3], const double h[3], const int64_t ng[3], const double *u, int64_t n,
                   double *xyz, double weight) {
  for (int64_t id = 0; id < n; ++id) {
    int64_t b[3];
    if (box_of(lo, h, ng, xyz + 3 * id, b)) continue;
    double g[3];
    normalized_gradient(h, ng, u, b, g);
    for (int a = 0; a < 3; ++a) xyz[3 * id + a] = xyz[3 * id + a] + g[a] * weight;
  }
  return 0;
}
