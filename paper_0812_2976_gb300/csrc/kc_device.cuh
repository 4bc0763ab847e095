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

// Fixed Danby iteration counts (Sec. 4.3 caps the loop so the GPU is never
// trapped; a fixed count also keeps warps branch-uniform).  From the paper's
// starting guess E0 = M + 0.85 e sign(sin M), three quartic steps bring
// |E - e sin E - M| to single-precision rounding for e <= 0.95 (worst error
// after two steps 7e-4, after three 1e-13 in exact arithmetic).
constexpr int kItersF32 = 3;

// ------------------------------------------------ conversions (integer pipe)

// double -> float, round to nearest even, by bit manipulation.  Exact IEEE
// result for normal float results; zero, subnormal, huge and non-finite
// inputs take the conversion instruction (rare).
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 897u > 253u) return __double2float_rn(x);   // ex outside [897, 1150]
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  unsigned f = (hi & 0x80000000u) | ((ex - 896u) << 23) | m;
  f += (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  return __uint_as_float(f);
}

// float -> double, exact, by bit manipulation (normal inputs).
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  if (ex - 1u > 253u) return (double)f;                // zero, subnormal, inf, nan
  const unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// x = hi + lo with hi = RN(x), lo = RN(x - hi): a double as a pair of floats
// (48 significant bits), by bit manipulation.
__device__ __forceinline__ void split_d(double x, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const unsigned ex = (h >> 20) & 0x7ffu;
  if (ex - 949u > 201u) {             // outside [949, 1150]: tiny, huge, zero, nan
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
    return;
  }
  const unsigned m = ((h & 0xfffffu) << 3) | (l >> 29);
  const unsigned rest = l & 0x1fffffffu;
  const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
  const unsigned sign = h & 0x80000000u;
  hi = __uint_as_float((sign | ((ex - 896u) << 23) | m) + up);
  // x - hi = (rest - up 2^29) 2^(ex - 1075), |.| <= 2^28 units
  const int r = (int)rest - (int)(up << 29);
  const float scale = __uint_as_float((ex - 948u) << 23);   // 2^(ex - 1075)
  const float lo_abs = __int2float_rn(r) * scale;
  lo = sign ? -lo_abs : lo_abs;
}

// ------------------------------------------------ FP32 building blocks

// Nearest integer of |x| < 2^22 with two FP32 adds (1.5 * 2^23 shifts the
// fraction out of the significand); cvt.rni runs on the 16-lane pipe.
constexpr float kRoundMagic = 12582912.0f;

__device__ __forceinline__ float round_small(float x) {
  return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic);
}

// MUFU approximations (absolute error ~2^-20.5 for sin/cos on the ranges
// used here, ~1 ulp relative for rcp).
__device__ __forceinline__ float sin_fast(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_fast(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/x in double for normal, finite x: the MUFU double-precision seed and
// two Newton steps (error ~1 ulp).  IEEE division costs more FP64-pipe
// instructions, which are the bound of the FP64 path.
__device__ __forceinline__ double rcp_f64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// sin and cos to about one ulp for |x| <= 8, on the FMA pipe.
// Cody & Waite (1980) reduction x = q pi/2 + r, |r| <= pi/4, with pi/2 split
// into two floats (q <= 5, so q * hi is exact inside the FMA), then the
// Taylor series of sin to r^9 (truncation 1.8e-9 at pi/4) and of cos to
// r^10 (1.1e-10), and the quadrant's swap and signs.
constexpr float kTwoOverPi = 0.636619772367581343f;
constexpr float kPiO2Hi = 1.57079637050628662109375f;      // RN(pi/2)
constexpr float kPiO2Lo = -4.37113900018624283e-8f;        // pi/2 - kPiO2Hi

__device__ __forceinline__ void sincos_accurate(float x, float &s, float &c) {
  const float k = __fmaf_rn(x, kTwoOverPi, kRoundMagic);
  const unsigned q = __float_as_uint(k);                    // low bits: q mod 4
  const float qf = __fsub_rn(k, kRoundMagic);
  float r = __fmaf_rn(-qf, kPiO2Hi, x);
  r = __fmaf_rn(-qf, kPiO2Lo, r);
  const float r2 = r * r;
  float ps = __fmaf_rn(r2, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = __fmaf_rn(r2, ps, 1.0f / 120.0f);
  ps = __fmaf_rn(r2, ps, -1.0f / 6.0f);
  const float sr = __fmaf_rn(r * r2, ps, r);
  float pc = __fmaf_rn(r2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = __fmaf_rn(r2, pc, -1.0f / 720.0f);
  pc = __fmaf_rn(r2, pc, 1.0f / 24.0f);
  pc = __fmaf_rn(r2, pc, -0.5f);
  const float cr = __fmaf_rn(r2, pc, 1.0f);
  const bool swap = q & 1u;
  const float s0 = swap ? cr : sr;
  const float c0 = swap ? sr : cr;
  s = __uint_as_float(__float_as_uint(s0) ^ ((q & 2u) << 30));
  c = __uint_as_float(__float_as_uint(c0) ^ (((q + 1u) & 2u) << 30));
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

// ------------------------------------------------ Danby step (Eqs. 7-10)

// One quartic Danby step for f(E) = E - e sin E - M given s = sin E,
// c = cos E.  The three nested divisions of Eqs. 8-10 fold into one:
// with f' = 1 - e c, f'' = e s, f''' = e c, h = f f''/2, D2 = f'^2 - h,
//   delta2 = -f f'/D2,
//   delta3 = -f / (f' + delta2 f''/2 + delta2^2 f'''/6)
//          = -f D2^2 / (f' [D2 (D2 - h) + f^2 f' f'''/6]),
// algebraically identical to Danby's delta3 (Eq. 10 as printed mixes
// delta1 and delta2).  Returns delta3.
__device__ __forceinline__ float danby_delta_f32(float E, float M, float e, float s, float c) {
  const float es = e * s;
  const float f = (E - M) - es;
  const float f1 = __fmaf_rn(-e, c, 1.0f);
  const float h = 0.5f * f * es;
  const float D2 = __fmaf_rn(f1, f1, -h);
  const float f3_6 = (e * (1.0f / 6.0f)) * c;
  const float Q = __fmaf_rn(f * f * f1, f3_6, D2 * (D2 - h));
  return -(f * D2 * D2) * rcp_fast(f1 * Q);
}

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

// Paper's starting guess (Sec. 4.3): E0 = M + 0.85 e sign(sin M); M is
// reduced to [-pi, pi] so sign(sin M) = sign(M), with sign(0) = +1.
__device__ __forceinline__ float kepler_start(float M, float e) {
  return M + (M >= 0.0f ? 0.85f : -0.85f) * e;
}

// Kepler's equation in single precision: three Danby steps from the paper's
// start.  Steps one and two take sin/cos from MUFU; their error (~1e-6)
// only perturbs the iterate, which the next quartic step corrects, so only
// the last step needs sin/cos to an ulp.  sin/cos of the returned E come from
// the last evaluation by the angle-addition expansion to second order in the
// last step (|delta| < 1e-3, truncation < 2e-10).
__device__ __forceinline__ float kepler_f32(float M, float e, float &sE, float &cE) {
  float E = kepler_start(M, e);
#pragma unroll
  for (int it = 0; it < kItersF32 - 1; ++it) {
    E += danby_delta_f32(E, M, e, sin_fast(E), cos_fast(E));
  }
  float s, c;
  sincos_accurate(E, s, c);
  const float d = danby_delta_f32(E, M, e, s, c);
  const float hd2 = 0.5f * d * d;
  sE = __fmaf_rn(d, c, __fmaf_rn(-hd2, s, s));
  cE = __fmaf_rn(-d, s, __fmaf_rn(-hd2, c, c));
  return E + d;
}

// Kepler's equation in double precision.  The single-precision solve (all
// three steps on MUFU sin/cos; error below 2e-5 for e <= 0.95) seeds one
// double-precision Danby step, whose quartic convergence lands on the
// double root; sin/cos of the result follow by angle addition to second
// order in that last step.
__device__ __forceinline__ double kepler_f64(double M, double e, double &sE, double &cE) {
  const float Mf = d2f(M), ef = d2f(e);
  float Ef = kepler_start(Mf, ef);
#pragma unroll
  for (int it = 0; it < kItersF32; ++it)
    Ef += danby_delta_f32(Ef, Mf, ef, sin_fast(Ef), cos_fast(Ef));
  const double E = f2d(Ef);
  double s, c;
  sincos_f64(E, s, c);
  const double d = danby_delta_f64(E, M, e, s, c);
  const double hd2 = 0.5 * d * d;
  sE = fma(d, c, fma(-hd2, s, s));
  cE = fma(-d, s, fma(-hd2, c, c));
  return E + d;
}

// ------------------------------------------------ per-planet constants

// Double-precision constants of one planet.  The phase of the mean anomaly
// at time t is (t - t_ref) * (inv_P + inv_P_lo) + c0 cycles (Eqs. 4/6 with
// the epoch moved from t0 to a reference time t_ref of the observations):
// inv_P + inv_P_lo = 1/P to ~1e-32 relative, and c0 in [-1/2, 1/2] holds
// frac((t_ref - t0)/P) + M0/(2 pi).  A, B, C give the velocity in the
// eccentric-anomaly form of Eq. 3:
//   v = [A (cos E - e) - B sin E] / (1 - e cos E) + C,
//   A = K cos w, B = K sqrt((1-e)(1+e)) sin w, C = K e cos w,
// which equals K [cos(w + f) + e cos w] with cos f = (cos E - e)/D,
// sin f = sqrt(1-e^2) sin E / D, D = 1 - e cos E; (1-e)(1+e) limits
// round-off for small e, as Sec. 4.4 advises.
struct PlanetD {
  double inv_P, inv_P_lo, c0, e, A, B, C, beta;
};

// Single-precision constants of one planet for the mixed path: 1/P and the
// phase offset as float pairs (the "pair of single" arithmetic of Sec. 5),
// e and the velocity constants.
struct PlanetF {
  float n_hi, n_lo, c_hi, c_lo, e, A, B, C;
};

__device__ __forceinline__ bool planet_valid(double P, double K, double e, double w, double M0) {
  return isfinite(P) && P > 0.0 && isfinite(K) && isfinite(e) && e >= 0.0 && e < 1.0 &&
         isfinite(w) && isfinite(M0);
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
  q.c0 = phase_cycles(dref, n, nl, M0 * kInvTwoPi);
  q.e = e;
  double sw, cw;
  sincos(w, &sw, &cw);
  q.beta = sqrt((1.0 - e) * (1.0 + e));
  q.A = K * cw;
  q.B = K * q.beta * sw;
  q.C = K * e * cw;
  return q;
}

__device__ __forceinline__ PlanetF planet_setup_mixed(const double *p, double dref) {
  const double P = p[0], K = p[1], e = p[2], w = p[3], M0 = p[4];
  PlanetF q;
  double n, nl;
  recip_checked(P, n, nl);
  float nlo2;
  split_d(n, q.n_hi, nlo2);
  q.n_lo = nlo2 + d2f(nl);
  const double c = phase_cycles(dref, n, nl, M0 * kInvTwoPi);
  split_d(c, q.c_hi, q.c_lo);
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
// (valid for |tau/P| < 2^22).  Result in [-pi, pi] up to rounding.
__device__ __forceinline__ float mean_anomaly_mixed(float tau_hi, float tau_lo, const PlanetF &q) {
  const float p = __fmul_rn(tau_hi, q.n_hi);  // kept apart from p - round(p)
  const float pe = __fmaf_rn(tau_hi, q.n_hi, -p);
  const float lo = __fmaf_rn(tau_hi, q.n_lo, __fmaf_rn(tau_lo, q.n_hi, pe)) + q.c_lo;
  const float fp = __fsub_rn(p, round_small(p));              // exact
  float u = __fadd_rn(fp, q.c_hi);
  u = __fsub_rn(u, round_small(u));                           // exact
  return (u + lo) * kTwoPiF;
}

__device__ __forceinline__ double mean_anomaly_f64(double tau, const PlanetD &q) {
  const double p = __dmul_rn(tau, q.inv_P);
  const double pe = fma(tau, q.inv_P, -p);
  const double lo = fma(tau, q.inv_P_lo, pe);
  double u = (p - rint(p)) + q.c0;
  u -= rint(u);
  u += lo;
  u -= rint(u);
  return u * kTwoPi;
}

// ------------------------------------------------ velocity (Eq. 3)

__device__ __forceinline__ float velocity_mixed(const PlanetF &q, float sE, float cE) {
  const float D = __fmaf_rn(-q.e, cE, 1.0f);
  const float num = __fmaf_rn(q.A, cE - q.e, -(q.B * sE));
  return __fmaf_rn(num, rcp_fast(D), q.C);
}

__device__ __forceinline__ double velocity_f64(const PlanetD &q, double sE, double cE) {
  const double D = fma(-q.e, cE, 1.0);
  return fma(fma(q.A, cE - q.e, -(q.B * sE)), rcp_f64(D), q.C);
}

// ------------------------------------------------ warp helpers

__device__ __forceinline__ float shfl_xor(float x, int m) {
  return __shfl_xor_sync(0xffffffffu, x, m);
}
__device__ __forceinline__ double shfl_xor(double x, int m) {
  return __shfl_xor_sync(0xffffffffu, x, m);
}

}  // namespace kc
