// Float-float and bit-construction arithmetic of the mechanics kernels.
//
// Every function here is plain IEEE arithmetic with round-to-nearest and
// no contraction.  On the device it uses the CUDA round-to-nearest
// intrinsics; compiled for the host (no FMA contraction), the same source
// gives the same bits, so that the box-index logic and the record splits can
// be checked on the CPU against IEEE division and exact arithmetic.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define BDM_HD __host__ __device__ __forceinline__
#else
#define BDM_HD inline
#endif

namespace bdm {

// ---------------------------------------------------------------------------
// Round-to-nearest operations and bit casts.
// ---------------------------------------------------------------------------
BDM_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

BDM_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

BDM_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

BDM_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

BDM_HD float u32_to_float_rn(unsigned int u) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(u);
#else
  return (float)u;
#endif
}

BDM_HD int float_to_int_rz(float f) {
#ifdef __CUDA_ARCH__
  return __float2int_rz(f);
#else
  return (int)f;
#endif
}

BDM_HD float double_to_float_rn(double d) {
#ifdef __CUDA_ARCH__
  return __double2float_rn(d);
#else
  return (float)d;
#endif
}

BDM_HD double d_sub(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}

BDM_HD double d_mul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}

BDM_HD unsigned long long bits_of(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long b;
  std::memcpy(&b, &d, sizeof b);
  return b;
#endif
}

BDM_HD double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
#endif
}

BDM_HD unsigned int bits_of(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned int u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}

BDM_HD float float_of(unsigned int u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}

BDM_HD int leading_zeros(unsigned int v) {
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return v ? __builtin_clz(v) : 32;
#endif
}

// ---------------------------------------------------------------------------
// Error-free transformations in FP32 (Knuth two-sum, fma two-product).
// ---------------------------------------------------------------------------
BDM_HD void two_sum(float a, float b, float &s, float &e) {
  s = f_add(a, b);
  const float bb = f_sub(s, a);
  e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}

BDM_HD void fast_two_sum(float a, float b, float &s, float &e) {
  s = f_add(a, b);
  e = f_sub(b, f_sub(s, a));
}

BDM_HD void two_prod(float a, float b, float &p, float &e) {
  p = f_mul(a, b);
  e = f_fma(a, b, -p);
}

// float-float (h, l) plus a float d, renormalized: the error of the result
// is one rounding of the low part (about 2^-48 of the value).
BDM_HD void ff_add_float(float h, float l, float d, float &rh, float &rl) {
  float s, e;
  two_sum(h, d, s, e);
  two_sum(s, f_add(l, e), rh, rl);
}

// 2^k as a float for -126 <= k <= 127.
BDM_HD float pow2f(int k) { return float_of((unsigned int)(k + 127) << 23); }

// Split a finite double into hi + lo floats (hi: leading 24 significant bits,
// truncated; lo: the remaining 29 bits rounded to 24).  Integer operations
// only, except for zero, tiny or huge magnitudes.
BDM_HD void split_ff(double a, float &hi, float &lo) {
  const unsigned long long b = bits_of(a);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  if (e >= 1023 - 126 + 52 && e <= 1023 + 127) {
    const unsigned int hb = sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)((b >> 29) & 0x7FFFFF);
    hi = float_of(hb);
    const float l = f_mul(u32_to_float_rn((unsigned int)(b & 0x1FFFFFFF)), pow2f(e - 1075));
    lo = sign ? -l : l;
  } else if (a == 0.0) {
    hi = 0.0f;
    lo = 0.0f;
  } else {
    hi = double_to_float_rn(a);
    lo = double_to_float_rn(d_sub(a, (double)hi));
  }
}

// -c as a double for 0 <= c < 2^32, built from its bits (the FP64 pipe of
// this part is 1/64 of the FP32 rate; conversions would use it).
BDM_HD double neg_u32_to_double(uint32_t c) {
  if (c == 0u) return -0.0;
  const int e = 31 - leading_zeros(c);
  const unsigned long long m = ((unsigned long long)c << (52 - e)) & 0xFFFFFFFFFFFFFull;
  return double_of(0x8000000000000000ull | ((unsigned long long)(1023 + e) << 52) | m);
}

// d / 2, exact: the exponent field decremented for normal values whose half
// is normal, an FP64 multiply otherwise.
BDM_HD double half_of(double d) {
  const unsigned long long b = bits_of(d);
  const unsigned e = (unsigned)((b >> 52) & 0x7FF);
  if (e > 1u && e < 0x7FFu) return double_of(b - (1ull << 52));
  return d_mul(0.5, d);
}

// Exact float -> double conversion with integer operations for normal
// values.
BDM_HD double f2d(float f) {
  const unsigned int u = bits_of(f);
  const unsigned int e = (u >> 23) & 0xFF;
  if (e == 0 || e == 0xFF) return (double)f;
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e + (1023 - 127)) << 52) |
                               ((unsigned long long)(u & 0x7FFFFF) << 29);
  return double_of(b);
}

// floor(fl64(a / L)) for a >= 0, exactly as IEEE FP64 division and floor
// give it, from float-float operands: (ah, al) approximates a and (ilh, ill)
// is 1/L to 2^-47 relative.  p + e = ah ilh + ah ill + al ilh, with
// |e| < 5 p 2^-24 (the product's rounding and the two tails, each below
// 2^-23 of its head).  A fraction of p at least p 2^-20 + 2^-10 away from 0
// and 1 decides at once; otherwise the fraction corrected by e decides
// unless it lies within p 2^-36 + 2^-40 of the integer (far above the
// remaining error, about p 2^-44, and the FP64 rounding of x - o and of the
// quotient).  False: undecided, the caller divides in FP64.
BDM_HD bool box_coord_ff(float ah, float al, float ilh, float ill, int &out) {
  float p, e;
  two_prod(ah, ilh, p, e);
  e = f_add(e, f_add(f_mul(ah, ill), f_mul(al, ilh)));
  const float c = floorf(p);
  const float g = f_sub(p, c);  // exact: fractional bits of p
  const int ci = float_to_int_rz(c);
  const float mg = f_fma(p, 0x1p-20f, 0x1p-10f);
  if (g >= mg && g <= 1.0f - mg) {
    out = ci;
    return true;
  }
  const float m = f_fma(p, 0x1p-36f, 0x1p-40f);
  if (g < 0.5f) {
    const float t = f_add(g, e);
    if (t >= m) { out = ci; return true; }
    if (t <= -m) { out = ci - 1; return true; }
  } else {
    const float t = f_add(f_sub(g, 1.0f), e);
    if (t <= -m) { out = ci; return true; }
    if (t >= m) { out = ci + 1; return true; }
  }
  return false;
}

}  // namespace bdm
