// Host build of the kernels' float-float and bit-construction arithmetic
// (paper_2503_10796_gb300/csrc/ffmath.cuh), checked against IEEE arithmetic
// and exact identities.  Built with g++ -ffp-contract=off, so that every
// float and double operation rounds as the device intrinsics do.
//
// Prints one line per check: "<name> <cases> <failures>" and exits non-zero
// when any check fails.
#include <cmath>
#include <cstdio>
#include <random>
#include <string>

#include "ffmath.cuh"

using namespace bdm;

static long failures_total = 0;

static void report(const char *name, long cases, long failures) {
  std::printf("%s %ld %ld\n", name, cases, failures);
  failures_total += failures;
}

// floor((x - o) / L) in IEEE FP64 (§4.4.3), against the float-float quotient
// where it decides; undecided cases fall back to that division on the GPU.
static void check_box_coord(std::mt19937_64 &rng, long max_span, const char *name) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long cases = 0, failures = 0, undecided = 0, random_cases = 0, random_undecided = 0;
  for (int trial = 0; trial < 3000; ++trial) {
    const double L = std::exp(std::log(1e-3) + U(rng) * std::log(1e6));
    const double o = (U(rng) - 0.5) * 1e5 * L;
    const long span = 1 + (long)(U(rng) * (double)max_span);
    float ilh, ill;
    split_ff(1.0 / L, ilh, ill);
    for (int k = 0; k < 400; ++k) {
      double x = o + (double)(long)(U(rng) * (double)span) * L;
      int u = (int)(U(rng) * 7) - 3;
      for (; u > 0; --u) x = std::nextafter(x, INFINITY);
      for (; u < 0; ++u) x = std::nextafter(x, -INFINITY);
      if (k % 4 == 0) x = o + U(rng) * (double)span * L;
      if (x < o) x = o;
      const double av = x - o;
      const long want = (long)std::floor(av / L);
      float ah, al;
      split_ff(av, ah, al);
      int got = 0;
      ++cases;
      const bool random = k % 4 == 0;
      random_cases += random ? 1 : 0;
      if (!box_coord_ff(ah, al, ilh, ill, got)) {
        ++undecided;
        random_undecided += random ? 1 : 0;
        continue;
      }
      if ((long)got != want) {
        if (failures < 5)
          std::printf("  box: L=%.17g o=%.17g x=%.17g want %ld got %d\n", L, o, x, want, got);
        ++failures;
      }
    }
  }
  // near-boundary centres (three in four cases here) need the FP64
  // division; centres drawn at random almost never do
  std::printf("%s undecided %ld of %ld; random centres %ld of %ld\n", name, undecided, cases, random_undecided,
              random_cases);
  report(name, cases, failures);
  report((std::string(name) + "_random_fallback_over_1pct").c_str(), random_cases,
         random_undecided * 100 > random_cases ? 1 : 0);
}

// hi + lo equals a to 2^-48 of |a|; hi carries at most 24 significant bits
// and is a truncation of a (same sign, not larger in magnitude).
static void check_split(std::mt19937_64 &rng) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long cases = 0, failures = 0;
  for (int k = 0; k < 200000; ++k) {
    const double a = (U(rng) - 0.5) * std::exp((U(rng) - 0.5) * 80.0);  // the integer branch
    float hi, lo;
    split_ff(a, hi, lo);
    ++cases;
    const double err = std::fabs(((double)hi + (double)lo) - a);
    const bool trunc = std::fabs((double)hi) <= std::fabs(a) && (hi == 0.0f || (hi > 0) == (a > 0));
    if (!(err <= std::ldexp(std::fabs(a), -48)) || !trunc) ++failures;
  }
  report("split_ff", cases, failures);
}

static void check_bits(std::mt19937_64 &rng) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long cases = 0, failures = 0;
  for (int k = 0; k < 200000; ++k) {
    const float f = (float)((U(rng) - 0.5) * std::exp((U(rng) - 0.5) * 150.0));
    const double d = (U(rng) - 0.5) * std::exp((U(rng) - 0.5) * 1300.0);
    const uint32_t c = (uint32_t)(U(rng) * 4294967295.0);
    ++cases;
    if (f2d(f) != (double)f) ++failures;
    if (half_of(d) != d * 0.5) ++failures;
    if (neg_u32_to_double(c) != -(double)c) ++failures;
  }
  if (neg_u32_to_double(0u) != 0.0 || !std::signbit(neg_u32_to_double(0u))) ++failures;
  report("bit_construction", cases, failures);
}

// two_sum and two_prod are error-free: the pair equals the exact result.
static void check_eft(std::mt19937_64 &rng) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long cases = 0, failures = 0;
  for (int k = 0; k < 200000; ++k) {
    const float a = (float)((U(rng) - 0.5) * std::exp((U(rng) - 0.5) * 40.0));
    const float b = (float)((U(rng) - 0.5) * std::exp((U(rng) - 0.5) * 40.0));
    float s, e, p, q;
    two_sum(a, b, s, e);
    two_prod(a, b, p, q);
    ++cases;
    if ((double)s + (double)e != (double)a + (double)b) ++failures;
    if ((double)p + (double)q != (double)a * (double)b) ++failures;
  }
  report("error_free_transformations", cases, failures);
}

// ff_add_float: a float-float box-relative offset moved by FP32
// displacements stays within a few ulps of its low part of the exact sum
// (long double reference), over 100 updates in a row.
static void check_ff_add(std::mt19937_64 &rng) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  long cases = 0, failures = 0;
  for (int k = 0; k < 20000; ++k) {
    const double L = 8.0 + 10.0 * U(rng);
    float h, l;
    split_ff((U(rng) * 1.4 - 0.2) * L, h, l);
    long double exact = (long double)h + (long double)l;
    for (int t = 0; t < 100; ++t) {
      const float d = (float)((U(rng) - 0.5) * 0.2);
      float rh, rl;
      ff_add_float(h, l, d, rh, rl);
      exact += (long double)d;
      h = rh;
      l = rl;
      ++cases;
      const long double err = ((long double)h + (long double)l) - exact;
      const double tol = std::ldexp(L, -44);
      if (!(std::fabs((double)err) <= tol)) ++failures;
      // the leading part is the float nearest the value (to one ulp)
      if (std::fabs((double)l) > std::ldexp(std::fabs((double)h) + 1e-30, -23) + std::ldexp(L, -60)) ++failures;
    }
  }
  report("ff_add_float", cases, failures);
}

int main() {
  std::mt19937_64 rng(20250314);
  check_box_coord(rng, 2000, "box_coord_narrow");
  check_box_coord(rng, 30000, "box_coord_wide");
  check_box_coord(rng, 2000000, "box_coord_2M");
  check_split(rng);
  check_bits(rng);
  check_eft(rng);
  check_ff_add(rng);
  return failures_total ? 1 : 0;
}
