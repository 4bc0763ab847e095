// kc_device.cuh -- device-side arithmetic shared by the chi-square, gradient,
// prediction and Kepler-only kernels.
//
// Notation follows Ford (2008): P period, K semi-amplitude, e eccentricity,
// w argument of pericentre, M0 mean anomaly at the epoch t0, M mean anomaly,
// E eccentric anomaly, f true anomaly, gamma systemic offset.
//
// Costs that shape this file (GB300, per SM per clock, measured): FP32 FMA
// 128 lanes; sin/cos/rcp (MUFU) 16; float rounding (cvt.rni) 16; FP64 FMA
// and double<->float conversion about 2.  So the hot loops use FP32 FMA
// only, MUFU where its error is later corrected, integer-pipe bit
// manipulation instead of conversion instructions, and FP64 only once per
// (system, planet).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kc {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kInvTwoPi = 0.15915494309189533576888376337251;
constexpr float kTwoPiF = 6.28318530717958647692f;

// Fixed step counts (Sec. 4.3 caps the loop so the GPU is never trapped; a
// fixed count also keeps warps branch-uniform).  The single-precision solve
// starts from Mikkola's cubic approximation, within 3.6e-3 rad of the root
// for every e < 1, and takes one Halley step with accurate sin/cos (5.1e-9
// in exact arithmetic, under the float rounding of E).  The double-precision
// solve polishes that solution with one Halley step in double.
//
// Eccentricity up to which one double-precision step suffices (the
// workloads draw e <= 0.95): above it the single-precision seed's error
// grows like 1e-7 / (1 - e cos E) near pericentre and the double-precision
// solve takes two steps.  Kernels choose once per warp (any_high_e), so
// that the usual case keeps one straight-line body with no branch per
// planet.
constexpr float kEccFast = 0.95f;

// ------------------------------------------------ conversions (integer pipe)

// All of them are branch-free: on GB300 a conversion with a rarely taken
// double-precision fallback branch measured three times the latency of the
// same code without it, and these conversions sit on the critical path of
// every kernel's prologue.  Values outside the normal float range follow
// flush-to-zero rules (results below 2^-126 become a signed zero, above the
// float range a signed infinity; NaN stays NaN), like the .ftz arithmetic
// of the kernels.

// Float bits of the double with high word hi and low word lo, rounded to
// nearest even; m and rest are the 23 kept and 29 dropped fraction bits.
__device__ __forceinline__ unsigned d2f_bits(unsigned hi, unsigned lo, unsigned &m,
                                             unsigned &rest, unsigned &up) {
  const unsigned ex = (hi >> 20) & 0x7ffu;
  const unsigned sign = hi & 0x80000000u;
  m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  rest = lo & 0x1fffffffu;
  up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  unsigned f = ((sign | ((ex - 896u) << 23) | m) + up);
  const unsigned special = (ex == 2047u && (((hi & 0xfffffu) | lo) != 0u)) ? 0x7fc00000u
                                                                           : (sign | 0x7f800000u);
  f = ex < 897u ? sign : f;
  f = ex > 1150u ? special : f;
  return f;
}

// double -> float, round to nearest even, by bit manipulation.
__device__ __forceinline__ float d2f(double x) {
  unsigned m, rest, up;
  return __uint_as_float(d2f_bits((unsigned)__double2hiint(x), (unsigned)__double2loint(x), m,
                                  rest, up));
}

// float -> double, exact, by bit manipulation.
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  const unsigned sign = b & 0x80000000u;
  unsigned hi = sign | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  unsigned lo = b << 29;
  hi = ex == 0u ? sign : hi;
  lo = ex == 0u ? 0u : lo;
  hi = ex == 255u ? (sign | 0x7ff00000u | ((b & 0x7fffffu) >> 3)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// x = hi + lo with hi = RN(x), lo = RN(x - hi): a double as a pair of floats
// (48 significant bits), by bit manipulation.  lo is zero when x lies
// outside [2^-74, 2^127) (there only hi is kept).
__device__ __forceinline__ void split_d(double x, float &hi, float &lo) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned ex = (h >> 20) & 0x7ffu;
  unsigned m, rest, up;
  hi = __uint_as_float(d2f_bits(h, l, m, rest, up));
  // x - hi = (rest - up 2^29) 2^(ex - 1075), |.| <= 2^28 units
  const int r = (int)rest - (int)(up << 29);
  const float scale = __uint_as_float(((ex - 948u) & 0xffu) << 23);   // 2^(ex - 1075)
  float lo_abs = __int2float_rn(r) * scale;
  lo_abs = (ex - 949u > 201u) ? 0.0f : lo_abs;
  lo = (h & 0x80000000u) ? -lo_abs : lo_abs;
}

// ------------------------------------------------ FP32 building blocks

// Nearest integer of |x| < 2^22 with two FP32 adds (1.5 * 2^23 shifts the
// fraction out of the significand); cvt.rni runs on the 16-lane pipe.
constexpr float kRoundMagic = 12582912.0f;

__device__ __forceinline__ float round_small(float x) {
  return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic);
}

// MUFU approximations (relative error ~2^-22 for the reciprocal, square
// root reciprocal and base-2 exponential and logarithm).
__device__ __forceinline__ float rsqrt_fast(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// One MUFU operation, where x * rsqrt(x) takes two (x > 0 here).
__device__ __forceinline__ float sqrt_fast(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_fast(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/x in double for x in the normal float range: the single-precision
// MUFU reciprocal (relative error < 2^-22, converted on the integer pipe)
// and one Newton step in double, r (2 - x r), whose error is the square of
// the seed's: below 2^-44 relative, always on the low side.  Two FP64
// operations instead of the four of an IEEE-exact reciprocal; the FP64 path
// uses it where that error is far below its 1e-12 target (the Danby step's
// correction, which is itself tiny, and 1/(1 - e cos E) of the velocity).
__device__ __forceinline__ double rcp_f64(double x) {
  const double r = f2d(rcp_fast(d2f(x)));
  return fma(r, fma(-x, r, 1.0), r);
}

// sin and cos for |x| <= 3 pi / 2 (the starting values of the
// single-precision Kepler solve lie within pi + 0.1): x = k pi + r with
// k = round(x / pi) in {-1, 0, 1} and pi split into two floats (the first
// product exact), so sin x = (-1)^k sin r and cos x = (-1)^k cos r with one
// shared sign and no exchange of sin and cos; sin r and cos r on
// [-pi/2, pi/2] by minimax polynomials of degree 9 and 10 (Remez fits of the
// absolute error, 4.6e-9 and 2.4e-10; minimax_sincos.py prints the
// coefficients).  Largest error over |x| <= pi + 0.1 in a float emulation:
// 1.3e-7 (sin) and 1.1e-7 (cos), about one ulp of 1, most of it the rounding
// of r near |r| = pi/2; 17 FMA-pipe and 3 integer operations, where a
// reduction by pi/2 would also select the quadrant and exchange sin and cos
// (6 integer operations more).
constexpr float kInvPiF = 0.318309886183790672f;          // RN(1/pi)
constexpr float kPiHiF = 3.14159274101257324219f;         // RN(pi)
constexpr float kPiLoF = -8.74227800037248566e-8f;        // pi - kPiHiF
constexpr float kSinC3 = -0.166666570965f;
constexpr float kSinC5 = 0.00833301729157f;
constexpr float kSinC7 = -0.000198066152016f;
constexpr float kSinC9 = 2.6000547683e-6f;
constexpr float kCosC2 = -0.499999995496f;
constexpr float kCosC4 = 0.0416666407281f;
constexpr float kCosC6 = -0.00138884035082f;
constexpr float kCosC8 = 2.47618862485e-5f;
constexpr float kCosC10 = -2.60771053559e-7f;

__device__ __forceinline__ void sincos_pi(float x, float &s, float &c) {
  const float k = __fmaf_rn(x, kInvPiF, kRoundMagic);
  const unsigned sgn = __float_as_uint(k) << 31;            // k odd: both negate
  const float kf = __fsub_rn(k, kRoundMagic);
  float r = __fmaf_rn(-kf, kPiHiF, x);
  r = __fmaf_rn(-kf, kPiLoF, r);
  const float u = r * r;
  float ps = __fmaf_rn(u, kSinC9, kSinC7);
  ps = __fmaf_rn(u, ps, kSinC5);
  ps = __fmaf_rn(u, ps, kSinC3);
  const float sr = __fmaf_rn(r * u, ps, r);
  float pc = __fmaf_rn(u, kCosC10, kCosC8);
  pc = __fmaf_rn(u, pc, kCosC6);
  pc = __fmaf_rn(u, pc, kCosC4);
  pc = __fmaf_rn(u, pc, kCosC2);
  const float cr = __fmaf_rn(u, pc, 1.0f);
  s = __uint_as_float(__float_as_uint(sr) ^ sgn);
  c = __uint_as_float(__float_as_uint(cr) ^ sgn);
}

// sin and cos in double precision for |x| <= 8: the same Cody & Waite
// reduction (pi/2 as two doubles) and the Taylor series of sin to r^17
// (truncation 8e-20 at pi/4) and of cos to r^16 (2e-18).  No branches, so
// the FP64-pipe cost is fixed: 3 + 9 + 9 operations.
constexpr double kRoundMagicD = 6755399441055744.0;           // 1.5 * 2^52
constexpr double kTwoOverPiD = 0.6366197723675814;
constexpr double kPiO2HiD = 1.5707963267948966;               // RN(pi/2)
constexpr double kPiO2LoD = 6.123233995736766e-17;            // pi/2 - hi

__device__ __forceinline__ void sincos_f64(double x, double &s, double &c) {
  const double k = fma(x, kTwoOverPiD, kRoundMagicD);
  const unsigned q = (unsigned)__double2loint(k);             // low bits: q mod 4
  const double qf = k - kRoundMagicD;
  double r = fma(-qf, kPiO2HiD, x);
  r = fma(-qf, kPiO2LoD, r);
  const double r2 = r * r;
  double ps = fma(r2, 1.0 / 355687428096000.0, -1.0 / 1307674368000.0);   // 1/17!, -1/15!
  ps = fma(r2, ps, 1.0 / 6227020800.0);                                    // 1/13!
  ps = fma(r2, ps, -1.0 / 39916800.0);                                     // -1/11!
  ps = fma(r2, ps, 1.0 / 362880.0);                                        // 1/9!
  ps = fma(r2, ps, -1.0 / 5040.0);
  ps = fma(r2, ps, 1.0 / 120.0);
  ps = fma(r2, ps, -1.0 / 6.0);
  const double sr = fma(r * r2, ps, r);
  double pc = fma(r2, 1.0 / 20922789888000.0, -1.0 / 87178291200.0);     // 1/16!, -1/14!
  pc = fma(r2, pc, 1.0 / 479001600.0);                                     // 1/12!
  pc = fma(r2, pc, -1.0 / 3628800.0);                                      // -1/10!
  pc = fma(r2, pc, 1.0 / 40320.0);
  pc = fma(r2, pc, -1.0 / 720.0);
  pc = fma(r2, pc, 1.0 / 24.0);
  pc = fma(r2, pc, -0.5);
  const double cr = fma(r2, pc, 1.0);
  // quadrant swap and signs on the integer halves (keeps them off the FP64 pipe)
  const bool swap = q & 1u;
  const int sh = __double2hiint(sr), sl = __double2loint(sr);
  const int ch = __double2hiint(cr), cl = __double2loint(cr);
  const int s_hi = swap ? ch : sh, s_lo = swap ? cl : sl;
  const int c_hi = swap ? sh : ch, c_lo = swap ? sl : cl;
  s = __hiloint2double(s_hi ^ (int)((q & 2u) << 30), s_lo);
  c = __hiloint2double(c_hi ^ (int)(((q + 1u) & 2u) << 30), c_lo);
}

// ------------------------------------------------ compensated sums

// Knuth's TwoSum: s + err == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  err = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Kahan (1965) compensated sum as described in Sec. 4.4: the running value
// is big - small, where small carries the rounding error of the last add.
struct Kahan {
  float big, small;
};

__device__ __forceinline__ void kahan_add(Kahan &k, float x) {
  const float y = __fsub_rn(x, k.small);
  const float t = __fadd_rn(k.big, y);
  k.small = __fsub_rn(__fsub_rn(t, k.big), y);
  k.big = t;
}

// a += b for two compensated sums (TwoSum on the big parts).
__device__ __forceinline__ void kahan_merge(Kahan &a, const Kahan &b) {
  float s, err;
  two_sum(a.big, b.big, s, err);
  a.big = s;
  a.small = __fsub_rn(__fadd_rn(a.small, b.small), err);
}

__device__ __forceinline__ float kahan_value(const Kahan &k) {
  return __fsub_rn(k.big, k.small);
}

// ------------------------------------------------ Kepler's equation (Sec. 4.3)

// One quartic Danby step for f(E) = E - e sin E - M given s = sin E,
// c = cos E, in double (the second double-precision step above kEccFast).
// The three nested divisions of Eqs. 8-10 fold into one: with
// f' = 1 - e c, f'' = e s, f''' = e c, h = f f''/2, D2 = f'^2 - h,
//   delta2 = -f f'/D2,
//   delta3 = -f / (f' + delta2 f''/2 + delta2^2 f'''/6)
//          = -f D2^2 / (f' [D2 (D2 - h) + f^2 f' f'''/6]),
// algebraically identical to Danby's delta3 (Eq. 10 as printed mixes
// delta1 and delta2).  Returns delta3.
__device__ __forceinline__ double danby_delta_f64(double E, double M, double e, double s,
                                                  double c) {
  const double es = e * s;
  const double f = (E - M) - es;
  const double f1 = fma(-e, c, 1.0);
  const double h = 0.5 * f * es;
  const double D2 = fma(f1, f1, -h);
  const double Q = fma(f * f * f1, (e * (1.0 / 6.0)) * c, D2 * (D2 - h));
  return -(f * D2 * D2) * rcp_f64(f1 * Q);
}

// Starting value of Mikkola (1987, "A cubic approximation for Kepler's
// equation"): with a = (1 - e)/(4 e + 1/2) and b = (M/2)/(4 e + 1/2), the
// real root z = cbrt(b + sign(b) sqrt(b^2 + a^3)) gives s = z - a/z, which
// is corrected by -0.078 s^5/(1 + e); then E0 = M + e (3 s - 4 s^3).  For M
// in [-pi, pi] it lies within 3.6e-3 rad of the root for every 0 <= e < 1
// (exact arithmetic, dense grid in (M, e) including |M| down to 1e-9),
// where the paper's M + 0.85 e sign(sin M) is up to 0.84 rad off near
// pericentre.  The cube root is exp2(log2|t|/3) on MUFU (|t| >= a^(3/2),
// above 1e-12 for float e < 1); the accuracy of the approximations only
// moves the start.  The constants that depend on e only are formed once
// per (system, planet) where the kernel can (kepler_start_setup).
//
// The per-planet part of Mikkola's start, formed once per (system, planet)
// instead of at every evaluation: r = 1/(4 e + 1/2), bs = r/2 (b = M bs),
// a = (1 - e) r, a3 = a^3 and the quintic correction's factor
// corr = -0.078/(1 + e).
struct StartF {
  float bs, a, a3, corr;
};

__device__ __forceinline__ StartF kepler_start_setup(float e) {
  const float r = 1.0f / __fmaf_rn(4.0f, e, 0.5f);
  StartF m;
  m.bs = 0.5f * r;
  m.a = (1.0f - e) * r;
  m.a3 = m.a * m.a * m.a;
  m.corr = -0.078f / (1.0f + e);
  return m;
}

// Mikkola's start from the hoisted constants.  The start is odd in M
// (sign(b) = sign(M)), so it is formed on |b|: |t| = |b| + sqrt(b^2 + a^3),
// z = |t|^(1/3) >= sqrt(a), s = z - a/z >= 0, the quintic correction
// s (1 + corr s^4), and the sign of M applied once before
// E0 = M + e s (3 - 4 s^2).
__device__ __forceinline__ float kepler_start_h(float M, float e, const StartF &m) {
  const float b = M * m.bs;
  const float w = __fmaf_rn(b, b, m.a3);
  const float tabs = fabsf(b) + sqrt_fast(w);           // w >= a^3 > 0
  const float z = ex2_fast(lg2_fast(tabs) * (1.0f / 3.0f));
  float s = __fmaf_rn(-m.a, rcp_fast(z), z);
  const float s2 = s * s;
  s = s * __fmaf_rn(m.corr, s2 * s2, 1.0f);
  const float ss = copysignf(s, M);
  return __fmaf_rn(e, ss * __fmaf_rn(-4.0f, s * s, 3.0f), M);
}

// Halley's step -f f' / (f'^2 - f f''/2) for f(E) = E - e sin E - M,
// f' = 1 - e cos E, f'' = e sin E, given s = sin E and c = cos E.  From
// Mikkola's start its cubic convergence lands within 5.1e-9 rad of the root
// for every e < 1 (exact arithmetic), below the float rounding of E.
__device__ __forceinline__ float halley_delta_h(float E, float M, float e, float s, float c) {
  const float es = e * s;
  const float f = (E - M) - es;
  const float f1 = __fmaf_rn(-e, c, 1.0f);
  const float den = __fmaf_rn(f * es, -0.5f, f1 * f1);
  return -(f * f1) * rcp_fast(den);
}

// Kepler's equation in single precision from the hoisted start constants:
// Mikkola's start, sin/cos to about an ulp there (sincos_pi, FMA pipe), one
// Halley step, and sin/cos of the returned E from that evaluation by the
// angle-addition expansion to second order in the step (|delta| < 3.6e-3,
// truncation < 8e-9).  No branch on e: the same straight-line code for
// every eccentricity.
__device__ __forceinline__ float kepler_f32_h(float M, float e, const StartF &m, float &sE,
                                              float &cE) {
  const float E = kepler_start_h(M, e, m);
  float s, c;
  sincos_pi(E, s, c);
  const float d = halley_delta_h(E, M, e, s, c);
  const float hd2 = 0.5f * d * d;
  sE = __fmaf_rn(d, c, __fmaf_rn(-hd2, s, s));
  cE = __fmaf_rn(-d, s, __fmaf_rn(-hd2, c, c));
  return E + d;
}

// The start constants for one evaluation, where every (M, e) has its own e
// (the Kepler-only solver; the FP64 path's single-precision first solve):
// approximate reciprocals instead of divisions, the same values up to
// their rounding.
__device__ __forceinline__ StartF kepler_start_consts(float e) {
  const float r = rcp_fast(__fmaf_rn(4.0f, e, 0.5f));
  StartF m;
  m.bs = 0.5f * r;
  m.a = (1.0f - e) * r;
  m.a3 = m.a * m.a * m.a;
  m.corr = -0.078f * rcp_fast(1.0f + e);
  return m;
}

__device__ __forceinline__ float kepler_f32(float M, float e, float &sE, float &cE) {
  return kepler_f32_h(M, e, kepler_start_consts(e), sE, cE);
}

// Warp-uniform choice of the double-precision solver's HI variant: true if
// any lane holds an eccentricity above kEccFast.  All lanes of `mask` must
// call it.
__device__ __forceinline__ bool any_high_e(bool mine, unsigned mask = 0xffffffffu) {
  return __any_sync(mask, mine) != 0;
}

// Calls body(HiTag<true>) or body(HiTag<false>): the observation loops of
// the double-precision kernels are compiled twice, once without the
// high-eccentricity branch.
template <bool B>
struct HiTag {
  static constexpr bool value = B;
};
template <typename F>
__device__ __forceinline__ void with_high_e(bool hi, F &&body) {
  if (hi)
    body(HiTag<true>{});
  else
    body(HiTag<false>{});
}

// Table-driven sin/cos in double (the table method of Tang, 1989-1991):
// x = k (2 pi/N) + b with k the nearest integer to x N/(2 pi) (chosen in
// single precision from x as a float, kf), b reduced in double with 2 pi/N
// split into two doubles, |b| <= pi/N + 1e-5; sin b and cos b by Taylor
// series to b^5 and b^6 (truncation below 1e-17 at N = 256); then
// sin x = S_k cos b + C_k sin b, cos x = C_k cos b - S_k sin b with
// (S_k, C_k) = (sin, cos)(2 pi k/N) from a table in shared memory
// (sincos_table_build).  The series' last terms, b^5/120 < 2.4e-12 and
// b^6/720 < 4.9e-15, enter the combination through one single-precision
// term each (error below 1e-18): 11 FP64 operations against 21 for
// sincos_f64.
constexpr int kSinTabN = 256;
constexpr double kTabStepHi = 0.02454369260617026;      // RN(2 pi/256)
constexpr double kTabStepLo = 9.567553118338697e-19;    // 2 pi/256 - hi
constexpr float kTabInvStepF = 40.74366543152521f;      // 256/(2 pi)

__device__ __forceinline__ void sincos_table_build(double2 *tab, int tid, int nthreads) {
  for (int i = tid; i < kSinTabN; i += nthreads) {
    double s, c;
    sincos_f64(fma((double)i, kTabStepHi, (double)i * kTabStepLo), s, c);
    tab[i] = make_double2(s, c);
  }
}

// xf: x rounded to float (the FP64 path evaluates sin/cos at its
// single-precision Kepler solution, or within a float ulp of it).
__device__ __forceinline__ void sincos_tab(double x, float xf, const double2 *tab, double &s,
                                           double &c) {
  const float kf = rintf(xf * kTabInvStepF);
  const double kd = f2d(kf);
  double b = fma(-kd, kTabStepHi, x);
  b = fma(-kd, kTabStepLo, b);
  const double b2 = b * b;
  const double sb3 = fma(b * b2, -1.0 / 6.0, b);                  // sin b to b^3
  const double cb4 = fma(b2, fma(b2, 1.0 / 24.0, -0.5), 1.0);     // cos b to b^4
  const double2 sc = tab[(int)kf & (kSinTabN - 1)];
  const float bf = d2f(b), b2f = bf * bf;
  const float sb5 = b2f * b2f * bf * (1.0f / 120.0f);             // b^5/120
  const float cb6 = -(b2f * b2f * b2f) * (1.0f / 720.0f);         // -b^6/720
  const float Sf = d2f(sc.x), Cf = d2f(sc.y);
  s = fma(sc.x, cb4, fma(sc.y, sb3, f2d(__fmaf_rn(Sf, cb6, Cf * sb5))));
  c = fma(sc.y, cb4, fma(-sc.x, sb3, f2d(__fmaf_rn(Cf, cb6, -(Sf * sb5)))));
}

// Halley's step -2 f f' / (2 f'^2 - f f'') = -f f' / (f'^2 - f e sin E / 2)
// for f(E) = E - e sin E - M, in double: 8 FP64 operations (13 FLOPs)
// against 26 FLOPs for Danby's quartic step.  From the single-precision
// solution (within 7e-7 of the root for e <= kEccFast, M rounded to float
// included) its cubic error is below double rounding (5e-16 |f'| at worst in
// a float emulation of the seed over 4e5 (M, e)).  f = (E - M) - e sin E
// takes one rounding (of E - M) with the product inside the FMA.  The term
// h = f e sin E / 2 is below 4e-7 f' (|f| ~ f' |E - root| < 7e-7 f'), at most
// 7e-6 of f'^2 (f' >= 1 - e >= 0.05): formed in single precision from
// ef = e and sf, the seed's sine (within 1e-6 of sin E), its error moves the
// step by less than 1e-11 of itself.
__device__ __forceinline__ double halley_delta_f64(double E, double M, double e, double s,
                                                   double c, float ef, float sf) {
  const double f = fma(-e, s, E - M);
  const double f1 = fma(-e, c, 1.0);
  const double h = f2d(0.5f * d2f(f) * (ef * sf));
  return -(f * f1) * rcp_f64(fma(f1, f1, -h));
}

// Kepler's equation in double precision.  The single-precision solve
// (kepler_f32) seeds one double-precision Halley step, which lands on the
// double root; sin/cos of the result follow by angle addition to second
// order in that last step.  HI and e > kEccFast: two quartic steps in
// double instead (the seed's error grows like 1e-7 / (1 - e cos E)).  The
// single-precision work costs little here: one FP64 instruction takes as
// long on GB300's FP64 pipe as ~76 FP32 issues.
// With a table (tab != nullptr, sincos_table_build), sin/cos come from
// sincos_tab.
template <bool HI = true>
__device__ __forceinline__ double kepler_f64(double M, double e, double &sE, double &cE,
                                             const double2 *tab = nullptr) {
  const float Mf = d2f(M), ef = d2f(e);
  float sf, cf;
  const float Ef = kepler_f32(Mf, ef, sf, cf);
  const bool high = HI && ef > kEccFast;
  double E = f2d(Ef);
  double s, c;
  if (tab)
    sincos_tab(E, Ef, tab, s, c);
  else
    sincos_f64(E, s, c);
  double d;
  if (high) {
    E += danby_delta_f64(E, M, e, s, c);
    if (tab)
      sincos_tab(E, d2f(E), tab, s, c);
    else
      sincos_f64(E, s, c);
    d = danby_delta_f64(E, M, e, s, c);
  } else {
    d = halley_delta_f64(E, M, e, s, c, ef, sf);
  }
  // d^2/2 < 2.5e-13 (|d| < 7e-7 in the Halley step, far smaller in the
  // second quartic step): single precision leaves it below 1e-19 absolute
  const float df = d2f(d);
  const double hd2 = f2d(0.5f * df * df);
  sE = fma(d, c, fma(-hd2, s, s));
  cE = fma(-d, s, fma(-hd2, c, c));
  return E + d;
}

// ------------------------------------------------ per-planet constants

// Double-precision constants of one planet.  The phase of the mean anomaly
// at time t is (t - t_ref) * (inv_P + inv_P_lo) + c0 cycles (Eqs. 4/6 with
// the epoch moved from t0 to a reference time t_ref of the observations):
// inv_P + inv_P_lo = 1/P to ~1e-32 relative, and c0 in [-1/2, 1/2] holds
// frac((t_ref - t0)/P) + M0/(2 pi).  A and B give the velocity in the
// eccentric-anomaly form of Eq. 3:
//   v = (A cos E - B sin E) / (1 - e cos E),
//   A = K cos w (1-e)(1+e), B = K sqrt((1-e)(1+e)) sin w,
// which equals K [cos(w + f) + e cos w] with cos f = (cos E - e)/D,
// sin f = sqrt(1-e^2) sin E / D, D = 1 - e cos E (the e cos w term and the
// -e of cos f combine: (cos E - e) + e D = (1 - e^2) cos E); (1-e)(1+e)
// limits round-off for small e, as Sec. 4.4 advises.
struct PlanetD {
  double inv_P, inv_P_lo, c0, e, A, B, beta;
  float inv_P_f, inv_P_lo_f;    // the same in single precision, for the phase's helpers
};

// Single-precision constants of one planet for the mixed path: 1/P and the
// phase offset as float pairs (the "pair of single" arithmetic of Sec. 5;
// the low parts stored times 2 pi, the scale the mean anomaly needs them
// in), e and the velocity constants.
struct PlanetF {
  float n_hi, n_lo2pi, c_hi, c_lo2pi, e, A, B, C;
};

// Parameter checks on the bit patterns (integer pipe, no FP64 compares):
// finite P > 0; K, w, M0 finite; 0 <= e < 1 (-0 counts as 0).
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}

__device__ __forceinline__ bool planet_valid(double P, double K, double e, double w, double M0) {
  const long long pb = __double_as_longlong(P), eb = __double_as_longlong(e);
  const long long emag = eb & 0x7fffffffffffffffll;
  const bool p_ok = pb > 0 && pb < 0x7ff0000000000000ll;            // +0 < P < +inf
  const bool e_ok = (eb >= 0 || emag == 0) && emag < 0x3ff0000000000000ll;   // [0, 1)
  return p_ok && e_ok && finite_bits(K) && finite_bits(w) && finite_bits(M0);
}

// 1/P as a double-double n + nl (|nl| < 2^-52 n): single-precision seed and
// two Newton steps in double (no double division).
__device__ __forceinline__ void recip_dd(double P, double &n, double &nl) {
  double r = f2d(rcp_fast(d2f(P)));
  double err = fma(-P, r, 1.0);
  r = fma(r, err, r);
  err = fma(-P, r, 1.0);
  r = fma(r, err, r);
  n = r;
  nl = fma(-P, r, 1.0) * r;          // (1 - P n)/P to first order
}

// frac(d * (n + nl)) + m reduced to [-1/2, 1/2], ~1e-16 absolute error: d*n
// keeps its exact FMA remainder, so the fraction survives d/P ~ 1e6.
__device__ __forceinline__ double phase_cycles(double d, double n, double nl, double m) {
  const double p = __dmul_rn(d, n);         // kept apart from p - floor(p)
  const double pe = fma(d, n, -p);
  const double q = fma(d, nl, pe);
  double c = (p - floor(p)) + q + m;
  c -= rint(c);
  return c;
}

__device__ __forceinline__ void recip_checked(double P, double &n, double &nl) {
  if (P > 0.0 && P < 1e300) {
    recip_dd(P, n, nl);
  } else {
    n = 1.0 / P;       // invalid system: the result is NaN anyway
    nl = 0.0;
  }
}

__device__ __forceinline__ PlanetD planet_setup_f64(const double *p, double dref) {
  const double P = p[0], K = p[1], e = p[2], w = p[3], M0 = p[4];
  PlanetD q;
  double n, nl;
  recip_checked(P, n, nl);
  q.inv_P = n;
  q.inv_P_lo = nl;
  q.inv_P_f = d2f(n);
  q.inv_P_lo_f = d2f(nl);
  q.c0 = phase_cycles(dref, n, nl, M0 * kInvTwoPi);
  q.e = e;
  double sw, cw;
  sincos(w, &sw, &cw);
  const double b2 = (1.0 - e) * (1.0 + e);
  q.beta = sqrt(b2);
  q.A = K * cw * b2;
  q.B = K * q.beta * sw;
  return q;
}

// ------------------------------------------------ float expansions (setup)

// a b = p + err exactly (the FMA remainder).
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &err) {
  p = __fmul_rn(a, b);
  err = __fmaf_rn(a, b, -p);
}

// s + err == a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &err) {
  s = __fadd_rn(a, b);
  err = __fsub_rn(b, __fsub_rn(s, a));
}

// hi + lo += x, the rounding error of the leading add kept exactly.
__device__ __forceinline__ void expansion_add(float &hi, float &lo, float x) {
  float s, err;
  two_sum(hi, x, s, err);
  hi = s;
  lo = __fadd_rn(lo, err);
}

// x = x0 + x1 + x2 exactly (24 + 24 + 5 significant bits) by bit
// manipulation, for x = 0 or 2^-74 <= |x| < 2^127 (elsewhere x1 = x2 = 0 and
// x0 follows the flush-to-zero rules of d2f).
__device__ __forceinline__ void split3_d(double x, float &x0, float &x1, float &x2) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned ex = (h >> 20) & 0x7ffu;
  unsigned m, rest, up;
  x0 = __uint_as_float(d2f_bits(h, l, m, rest, up));
  // x - x0 = r 2^(ex - 1075) with |r| <= 2^28: r = RN24(r) + (a 5-bit rest)
  const int r = (int)rest - (int)(up << 29);
  const float r1 = __int2float_rn(r);
  const int r2 = r - __float2int_rz(r1);                   // exact, |r2| <= 16
  const float scale = __uint_as_float(((ex - 948u) & 0xffu) << 23);   // 2^(ex - 1075)
  const bool in_range = ex - 949u <= 201u;
  const float y1 = in_range ? r1 * scale : 0.0f;
  const float y2 = in_range ? __int2float_rn(r2) * scale : 0.0f;
  const bool neg = (h & 0x80000000u) != 0u;
  x1 = neg ? -y1 : y1;
  x2 = neg ? -y2 : y2;
}

struct Split3 {
  float x0, x1, x2;
};

__device__ __forceinline__ Split3 split3(double x) {
  Split3 r;
  split3_d(x, r.x0, r.x1, r.x2);
  return r;
}

// a - b as a float pair hi + lo (about 2^-48 relative) from exact splits of
// the doubles a and b: no FP64 instruction.
__device__ __forceinline__ void sub_ds(const Split3 &a, const Split3 &b, float &hi, float &lo) {
  float h, l;
  two_sum(a.x0, -b.x0, h, l);
  expansion_add(h, l, a.x1);
  expansion_add(h, l, -b.x1);
  expansion_add(h, l, a.x2);
  expansion_add(h, l, -b.x2);
  fast_two_sum(h, l, hi, lo);
}

constexpr float kInvTwoPiHi = 0.15915493667125702f;       // RN(1/(2 pi))
constexpr float kInvTwoPiLo = 6.4206382432985265e-09f;    // 1/(2 pi) - hi

// The same quantities in double-double arithmetic, for periods or epochs
// outside the range of the float-expansion code below (out of line).
static __device__ __noinline__ void phase_setup_wide(double P, double M0, double t_ref, double t0,
                                              float &n_hi, float &n_lo, float &c_hi,
                                              float &c_lo) {
  double n, nl;
  recip_checked(P, n, nl);
  float nlo2;
  split_d(n, n_hi, nlo2);
  n_lo = nlo2 + d2f(nl);
  split_d(phase_cycles(t_ref - t0, n, nl, M0 * kInvTwoPi), c_hi, c_lo);
}

// 1/P and the phase offset of the mixed path in float expansions (no FP64
// instruction: the FP64 pipe runs at 1/64 of the FP32 rate).  With exact
// three-float splits P = P0 + P1 + P2, t_ref = r0 + r1 + r2, t0 = e0 + e1 + e2:
//   1/P = n_hi + n_lo: r = 1/P0 (MUFU), x = 1 - P r carried from the exact
//     product P0 r (|x| < 2^-21), 1/P = r (1 + x + x^2); relative error
//     about 2^-45, below 1e-9 cycles over 3e4 periods;
//   frac((t_ref - t0)/P): D0 = RN(r0 - e0), k = the integer nearest to
//     D0 n_hi, and the remainder rho = (t_ref - t0) - k P summed from the
//     split terms, products by FMA remainders and sums by TwoSum, starting
//     with the cancelling pair D0 - k P0 so that the running sum stays of
//     the size of P; then rho (n_hi + n_lo) with |rho/P| < 3: error about
//     1e-14 cycles.
// Valid for 2^-20 <= P <= 2^40 d and |t_ref - t0| < 2^24 P; outside that
// range the double-double code of the FP64 path is used (rare).
__device__ __forceinline__ void phase_setup_ds(double P, double M0, double t_ref, double t0,
                                               float &n_hi, float &n_lo, float &c_hi,
                                               float &c_lo) {
  const Split3 Ps = split3(P), tr = split3(t_ref), te = split3(t0);
  float D0, D1;
  two_sum(tr.x0, -te.x0, D0, D1);
  if (!(Ps.x0 >= 0x1p-20f && Ps.x0 <= 0x1p40f && fabsf(D0) < 0x1p24f * Ps.x0)) {
    phase_setup_wide(P, M0, t_ref, t0, n_hi, n_lo, c_hi, c_lo);
    return;
  }
  const float r = rcp_fast(Ps.x0);
  float pr, pre;
  two_prod(Ps.x0, r, pr, pre);
  const float x = __fmaf_rn(-Ps.x1, r, __fsub_rn(__fsub_rn(1.0f, pr), pre));  // 1 - pr exact
  fast_two_sum(r, r * __fmaf_rn(x, x, x), n_hi, n_lo);
  // rho = (t_ref - t0) - k P
  const float k = rintf(D0 * n_hi);
  float a0, a0e, a1, a1e, a2, a2e;
  two_prod(k, Ps.x0, a0, a0e);
  two_prod(k, Ps.x1, a1, a1e);
  two_prod(k, Ps.x2, a2, a2e);
  float hi, lo;
  two_sum(D0, -a0, hi, lo);
  expansion_add(hi, lo, D1);
  expansion_add(hi, lo, -a0e);
  expansion_add(hi, lo, tr.x1);
  expansion_add(hi, lo, -te.x1);
  expansion_add(hi, lo, -a1);
  expansion_add(hi, lo, tr.x2);
  expansion_add(hi, lo, -te.x2);
  expansion_add(hi, lo, -a1e);
  expansion_add(hi, lo, -a2);
  expansion_add(hi, lo, -a2e);
  float rh, rl;
  fast_two_sum(hi, lo, rh, rl);
  // cycles = rho (n_hi + n_lo) + M0/(2 pi), reduced to [-1/2, 1/2]
  float u, ue;
  two_prod(rh, n_hi, u, ue);
  const float t_small = __fmaf_rn(rh, n_lo, __fmaf_rn(rl, n_hi, ue));
  float mh0, ml0;
  split_d(M0, mh0, ml0);
  float mh, me;
  two_prod(mh0, kInvTwoPiHi, mh, me);
  const float ml = __fmaf_rn(mh0, kInvTwoPiLo, __fmaf_rn(ml0, kInvTwoPiHi, me));
  float sc, se;
  two_sum(u, mh, sc, se);
  sc = __fsub_rn(sc, rintf(sc));                            // exact
  fast_two_sum(sc, __fadd_rn(__fadd_rn(t_small, ml), se), c_hi, c_lo);
}

// Single-precision constants of one planet for the mixed path.
// t_ref: the reference time the observation times are taken from; t0: the
// epoch of M0.
__device__ __forceinline__ PlanetF planet_setup_mixed(const double *p, double t_ref, double t0) {
  const double P = p[0], K = p[1], e = p[2], w = p[3], M0 = p[4];
  PlanetF q;
  float n_lo, c_lo;
  phase_setup_ds(P, M0, t_ref, t0, q.n_hi, n_lo, q.c_hi, c_lo);
  q.n_lo2pi = n_lo * kTwoPiF;
  q.c_lo2pi = c_lo * kTwoPiF;
  const float ef = d2f(e);
  q.e = ef;
  // sin/cos of w to single-precision rounding although w itself is double:
  // w = w_hi + w_lo, sin w ~ sin w_hi + w_lo cos w_hi (|w_lo| < 1e-6 |w|).
  float w_hi, w_lo;
  split_d(w, w_hi, w_lo);
  float sw, cw;
  sincosf(w_hi, &sw, &cw);
  const float sw1 = __fmaf_rn(w_lo, cw, sw);
  cw = __fmaf_rn(-w_lo, sw, cw);
  sw = sw1;
  const float Kf = d2f(K);
  const float beta = sqrtf((1.0f - ef) * (1.0f + ef));
  q.A = Kf * cw;
  q.B = Kf * beta * sw;
  q.C = Kf * ef * cw;
  return q;
}

// ------------------------------------------------ mean anomaly (Eqs. 4, 6)

// Mixed path.  tau = tau_hi + tau_lo = t - t_ref as a float pair.  The
// product tau * (n_hi + n_lo) keeps its exact FMA remainder, so its
// fractional part is good to ~1e-11 cycles although tau/P reaches 1e4
// (valid for |tau/P| < 2^22).  The low part of the phase is formed already
// scaled by 2 pi, 2 pi (pe + tau_lo n_hi) + tau_hi (2 pi n_lo) + 2 pi c_lo,
// and enters the final FMA M = 2 pi u + lo, one rounding.  Result in
// [-pi, pi] up to rounding.
__device__ __forceinline__ float mean_anomaly_mixed(float tau_hi, float tau_lo, const PlanetF &q) {
  const float p = __fmul_rn(tau_hi, q.n_hi);  // kept apart from p - round(p)
  const float pe = __fmaf_rn(tau_hi, q.n_hi, -p);
  const float lo = __fmaf_rn(__fmaf_rn(tau_lo, q.n_hi, pe), kTwoPiF,
                             __fmaf_rn(tau_hi, q.n_lo2pi, q.c_lo2pi));
  const float fp = __fsub_rn(p, round_small(p));              // exact
  float u = __fadd_rn(fp, q.c_hi);
  u = __fsub_rn(u, round_small(u));                           // exact
  return __fmaf_rn(u, kTwoPiF, lo);
}

// Pure single precision (the paper's all-float variant, for comparisons):
// tau = t - t0 as one float, so the phase loses ~|tau/P| 2^-24 cycles.
__device__ __forceinline__ float mean_anomaly_single(float tau, const PlanetF &q) {
  float x = __fmaf_rn(tau, q.n_hi, q.c_hi);
  x = __fsub_rn(x, rintf(x));
  return x * kTwoPiF;
}

// The phase tau/P + c0 with four FP64 instructions (the FP64 pipe runs at
// 1/64 of the FP32 rate): the integer part n of tau/P is taken from single
// precision (exact as a double; it may be off by one or more, which only
// widens the range of u), u = tau inv_P - n in one FMA (exact product and
// difference, one rounding: error below 2^-54 |u| cycles), u + c0 rounds
// once more, and the nearest integer of that (from its single-precision
// value, exact as a double) is removed exactly.  The low part of 1/P,
// tau inv_P_lo (below 1e-13 cycles for tau < 6000 d), enters the final FMA
// scaled by 2 pi in single precision.  M lies in [-pi, pi] up to the
// single-precision rounding of u + c0 near +-1/2 (a few 1e-7 rad).
__device__ __forceinline__ double mean_anomaly_f64(double tau, const PlanetD &q) {
  const float tf = d2f(tau);
  const double n = f2d(rintf(tf * q.inv_P_f));
  double u = fma(tau, q.inv_P, -n) + q.c0;
  u -= f2d(rintf(d2f(u)));
  const float lo2pi = (tf * q.inv_P_lo_f) * kTwoPiF;
  return fma(u, kTwoPi, f2d(lo2pi));
}

// ------------------------------------------------ velocity (Eq. 3)

__device__ __forceinline__ float velocity_mixed(const PlanetF &q, float sE, float cE) {
  const float D = __fmaf_rn(-q.e, cE, 1.0f);
  const float num = __fmaf_rn(q.A, cE - q.e, -(q.B * sE));
  return __fmaf_rn(num, rcp_fast(D), q.C);
}

// The same velocity with the e cos w term folded: A e = K cos w e = C, so
// A (cos E - e) - B sin E = A cos E - (B sin E + C), two FMAs.
__device__ __forceinline__ float velocity_h(const PlanetF &q, float sE, float cE) {
  const float D = __fmaf_rn(-q.e, cE, 1.0f);
  const float num = __fmaf_rn(q.A, cE, -__fmaf_rn(q.B, sE, q.C));
  return __fmaf_rn(num, rcp_fast(D), q.C);
}

// V + v for one planet (the planet sum's addition inside the last FMA).
__device__ __forceinline__ double velocity_add_f64(const PlanetD &q, double sE, double cE,
                                                   double V) {
  const double D = fma(-q.e, cE, 1.0);
  return fma(fma(q.A, cE, -(q.B * sE)), rcp_f64(D), V);
}

// ------------------------------------------------ DE-MC proposal

// floor(f) clamped to 0 .. hi (NaN to 0): an index inside the range for any
// draw, also outside [0, 1).
__device__ __forceinline__ int64_t demc_clamp_index(double f, int64_t hi) {
  f = floor(f);
  return f >= 0.0 ? (f < (double)hi ? (int64_t)f : hi) : 0;
}

// The two partners of draw pair (u1, u2) in [0, 1): distinct, uniform over
// the ordered pairs of the m chains from pfirst (m >= 2, checked by the host).
__device__ __forceinline__ void demc_partners(double u1, double u2, int64_t pfirst, int64_t m,
                                              int64_t &r1, int64_t &r2) {
  const int64_t k1 = demc_clamp_index(u1 * (double)m, m - 1);
  int64_t k2 = demc_clamp_index(u2 * (double)(m - 1), m - 2);
  k2 += k2 >= k1 ? 1 : 0;
  r1 = pfirst + k1;
  r2 = pfirst + k2;
}

// Parameter p of chain i's proposal,
// x*_p = x_ip + gamma (x_r1,p - x_r2,p) + (eps_scale_p |x_ip|) z,
// with explicit roundings so that the result does not depend on FMA
// contraction (the proposal kernel and the fused chi2 prologue agree bit for
// bit).
__device__ __forceinline__ double demc_proposal(const double *states, int npar, int64_t i,
                                                int64_t r1, int64_t r2, int p, double gamma,
                                                double eps_scale, double z) {
  const double xi = states[i * npar + p];
  const double d = __dsub_rn(states[r1 * npar + p], states[r2 * npar + p]);
  const double eps = __dmul_rn(__dmul_rn(eps_scale, fabs(xi)), z);
  return __dadd_rn(__dadd_rn(xi, __dmul_rn(gamma, d)), eps);
}

// ------------------------------------------------ warp helpers

__device__ __forceinline__ float shfl_xor(float x, int m) {
  return __shfl_xor_sync(0xffffffffu, x, m);
}
__device__ __forceinline__ double shfl_xor(double x, int m) {
  return __shfl_xor_sync(0xffffffffu, x, m);
}

}  // namespace kc
