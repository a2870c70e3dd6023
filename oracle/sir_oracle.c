/*
 * sir_oracle.c -- plain, single-threaded FP64 CPU oracle of the thesis's
 * epidemiology use case (§4.6.3): susceptible / infected / recovered agents
 * with the infection (Algorithm 3), recovery (Algorithm 4) and random
 * movement (Algorithm 5) behaviours, in a cube with toroidal boundaries.
 *
 * TEST INFRASTRUCTURE ONLY, like bdm_oracle.c: only the test suite may load
 * it, and it shares no code with the CUDA path.  Compiled with -O2
 * -ffp-contract=off.
 *
 * Random numbers: Philox4x64-10 (the counter-based generator of §7.1.4,
 * implemented in bdm_oracle.c), key {seed, 1}, counter {ID, t, draw, 0};
 * a 53-bit uniform in [0, 1) from the top 53 bits of a word.  Draw 0 gives
 * the infection uniform (word 0) and the recovery uniform (word 1); draw 1
 * gives the three movement uniforms (words 0-2).  Results therefore do not
 * depend on the order in which agents are processed.
 *
 * Readings taken where the thesis leaves a choice (each one is listed with
 * the design notes of the repository):
 *   - copy execution context: every agent reads the positions and states of
 *     the other agents at the start of the step; an agent's own behaviours
 *     run in the order infection, recovery, movement and see its own
 *     updates (an agent infected in a step may recover in the same step);
 *   - infection: a susceptible agent draws one uniform; below the infection
 *     probability, it becomes infected if any other agent infected at the
 *     start of the step lies within the infection radius (squared distance
 *     below radius * radius, plain Euclidean distance inside the cube);
 *   - movement: Algorithm 5 prints the L2 norm of a random vector where a
 *     direction is meant; read as the normalized vector of three uniforms
 *     in [-1, 1) (no move for the zero vector), times the speed; each
 *     coordinate is then wrapped into [0, L) by fmod and + L when negative.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

enum { SIR_S = 0, SIR_I = 1, SIR_R = 2 };

typedef struct {
  double radius, p_infect, p_recover, speed, length;
  uint64_t seed;
} orc_sir_params;

static double unit53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

static void draw(uint64_t seed, int64_t id, int64_t t, uint64_t k, uint64_t w[4]) {
  uint64_t ctr[4] = {(uint64_t)id, (uint64_t)t, k, 0}, key[2] = {seed, 1};
  orc_philox4x64_10(ctr, key, w);
}

static double wrap(double v, double L) {
  double r = fmod(v, L);
  if (r < 0.0) r = L + r;
  return r;
}

/* Any agent j != i infected in the snapshot within the radius of i. */
static int infected_neighbor(int64_t n, const double *xyz, const uint8_t *state, int64_t i, double r2) {
  for (int64_t j = 0; j < n; ++j) {
    if (j == i || state[j] != SIR_I) continue;
    double dx = xyz[3 * j] - xyz[3 * i], dy = xyz[3 * j + 1] - xyz[3 * i + 1], dz = xyz[3 * j + 2] - xyz[3 * i + 2];
    if ((dx * dx + dy * dy) + dz * dz < r2) return 1;
  }
  return 0;
}

/* `steps` steps from step index t0; xyz (n x 3) and state (n) in place. */
int orc_sir_step(const orc_sir_params *p, int64_t n, double *xyz, uint8_t *state, int64_t t0, int32_t steps) {
  double *nx = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  uint8_t *ns = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
  if (!nx || !ns) { free(nx); free(ns); return -2; }
  const double r2 = p->radius * p->radius;
  for (int32_t s = 0; s < steps; ++s) {
    const int64_t t = t0 + s;
    for (int64_t i = 0; i < n; ++i) {
      uint64_t w[4];
      draw(p->seed, i, t, 0, w);
      uint8_t st = state[i];
      if (st == SIR_S && unit53(w[0]) < p->p_infect && infected_neighbor(n, xyz, state, i, r2)) st = SIR_I;
      if (st == SIR_I && unit53(w[1]) < p->p_recover) st = SIR_R;
      ns[i] = st;
      uint64_t m[4];
      draw(p->seed, i, t, 1, m);
      double v[3];
      for (int a = 0; a < 3; ++a) v[a] = 2.0 * unit53(m[a]) - 1.0;
      const double norm = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
      for (int a = 0; a < 3; ++a) {
        double x = xyz[3 * i + a];
        if (norm > 0.0) x = x + (v[a] / norm) * p->speed;
        nx[3 * i + a] = wrap(x, p->length);
      }
    }
    memcpy(xyz, nx, sizeof(double) * 3 * (size_t)n);
    memcpy(state, ns, (size_t)n);
  }
  free(nx);
  free(ns);
  return 0;
}
