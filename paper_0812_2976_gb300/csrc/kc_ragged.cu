// kc_ragged.cu -- ragged batches: systems with their own planet count and
// their own observations, evaluated by one persistent kernel that takes
// whole systems from a device work queue, replayed as a CUDA graph.
//
// The paper evaluates uniform batches (every model of one star shares the
// observations, Sec. 4.1).  A ragged batch (n_obs 16..1024, n_pl 1..6 per
// system) varies the work per system by ~400x, so a static split of
// systems over threads leaves most SMs idle at the end.  Here:
//  - a plan orders the systems by planet count, then by decreasing work
//    (n_pl * n_obs), and keeps that order on the device: big systems start
//    first, the smallest fill the tail, and warps running together mostly
//    share one unrolled body;
//  - each warp of a persistent grid takes the next system from an atomic
//    counter and evaluates it with its 32 lanes over the observations, the
//    planet count being warp-uniform so the planet loop is fully unrolled
//    for that count;
//  - the observations, fixed for the plan (Sec. 4.1 treats them as
//    constants for every model), are converted once per plan to the form the
//    kernel reads (float pairs for the mixed path).
// The per-planet arithmetic is that of the uniform kernels (kc_device.cuh).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "kc_device.cuh"
#include "kc_internal.h"
#include "kc_ragged.h"

namespace kc {

namespace {

__device__ inline double nan_r() { return __longlong_as_double(0x7ff8000000000000ll); }

// KC_DEBUG checks of a ragged system's descriptors (always true in a normal
// build): its observation range inside the plan's observations, its planet
// count, its parameter range inside the packed parameters.
__device__ __forceinline__ bool ragged_obs_ok(const RaggedDev &d, int64_t s, int64_t o0,
                                              int64_t o1) {
  return dbg_ok(d.invalid, 0 <= o0 && o0 <= o1 && o1 <= d.n_obs_total, kDbgObsOff, s);
}

__device__ __forceinline__ bool ragged_system_ok(const RaggedDev &d, int64_t s, int J,
                                                 int64_t o0, int64_t o1) {
  if (!dbg_ok(d.invalid, J >= 1 && J <= KC_MAX_PLANETS, kDbgPlanets, s)) return false;
  if (!ragged_obs_ok(d, s, o0, o1)) return false;
  const int64_t p0 = d.par_off[s];
  return dbg_ok(d.invalid, 0 <= p0 && p0 + 5 * J + 1 <= d.n_par_total, kDbgParOff, s);
}

__device__ inline double system_gamma_r(const double *p, int J) {
  bool ok = finite_bits(p[5 * J]);
  for (int j = 0; j < J; ++j)
    ok = ok && planet_valid(p[5 * j], p[5 * j + 1], p[5 * j + 2], p[5 * j + 3], p[5 * j + 4]);
  return ok ? p[5 * J] : nan_r();
}

// ------------------------------------------------------------ observation prep

// One warp per system: tau = t - t_ref (t_ref = the system's first
// observation) and v as float pairs, w = 1/(sigma^2 + jitter^2), t - t0.
__global__ void prep_obs_mixed(RaggedDev d, const double *__restrict__ t,
                               const double *__restrict__ v, const double *__restrict__ sigma,
                               double jitter2, float4 *__restrict__ oa, float2 *__restrict__ ob,
                               double *__restrict__ t_ref) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < d.n_sys; s += nwarp) {
    const int64_t o0 = d.obs_off[s], o1 = d.obs_off[s + 1];
    if (!ragged_obs_ok(d, s, o0, o1)) continue;
    const double tr = o1 > o0 ? t[o0] : d.t0;
    if (lane == 0) t_ref[s] = tr;
    // no FP64 instruction: differences from exact three-float splits
    const Split3 tr3 = split3(tr), te3 = split3(d.t0);
    const float jit2 = d2f(jitter2);
    for (int64_t k = o0 + lane; k < o1; k += 32) {
      const Split3 tk = split3(t[k]);
      float th, tl, vh, vl;
      sub_ds(tk, tr3, th, tl);
      split_d(v[k], vh, vl);
      oa[k] = make_float4(th, tl, vh, vl);
      const float sg = d2f(sigma[k]);
      const float var = __fmaf_rn(sg, sg, jit2);
      ob[k] = make_float2(var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000),
                          (tk.x0 - te3.x0) + (tk.x1 - te3.x1));
    }
  }
}

__global__ void prep_obs_f64(RaggedDev d, const double *__restrict__ t,
                             const double *__restrict__ v, const double *__restrict__ sigma,
                             double jitter2, ObsR64 *__restrict__ od,
                             double *__restrict__ t_ref) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < d.n_sys; s += nwarp) {
    const int64_t o0 = d.obs_off[s], o1 = d.obs_off[s + 1];
    if (!ragged_obs_ok(d, s, o0, o1)) continue;
    const double tr = o1 > o0 ? t[o0] : d.t0;
    if (lane == 0) t_ref[s] = tr;
    for (int64_t k = o0 + lane; k < o1; k += 32) {
      const double var = fma(sigma[k], sigma[k], jitter2);
      od[k] = ObsR64{t[k] - tr, v[k], var > 0.0 ? 1.0 / var : nan_r(), t[k] - d.t0};
    }
  }
}

// FP64 model velocities of a ragged batch, one warp per system.
__global__ void predict_ragged_kernel(const double *__restrict__ params,
                                      const int64_t *__restrict__ par_off,
                                      const int32_t *__restrict__ n_pl,
                                      const double *__restrict__ t,
                                      const int64_t *__restrict__ obs_off, int64_t n_sys,
                                      double t0, double *__restrict__ v_out,
                                      unsigned long long *words) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < n_sys; s += nwarp) {
    const int64_t o0 = obs_off[s], o1 = obs_off[s + 1];
    if (o1 <= o0) continue;
    const int J = n_pl[s];
    // the caller's arrays (no totals known here): ordered offsets, a planet
    // count in range
    if (!dbg_ok(words, o0 >= 0 && par_off[s] >= 0, kDbgObsOff, s) ||
        !dbg_ok(words, J >= 1 && J <= KC_MAX_PLANETS, kDbgPlanets, s))
      continue;
    const double *p = params + par_off[s];
    const double tr = t[o0];
    const double gam = system_gamma_r(p, J);
    for (int64_t k = o0 + lane; k < o1; k += 32) {
      double V = gam;
      for (int j = 0; j < J; ++j) {
        const PlanetD q = planet_setup_f64(p + 5 * j, tr - t0);
        double sE, cE;
        kepler_f64(mean_anomaly_f64(t[k] - tr, q), q.e, sE, cE);
        V = velocity_add_f64(q, sE, cE, V);
      }
      v_out[k] = V;
    }
  }
}

// ------------------------------------------------------------ per-system bodies

struct RPlanetF {
  PlanetF base;
  float K, cw, sw, beta, n2, ibeta;   // ibeta = 1/beta
  StartF m;                           // the e-only constants of Mikkola's start
};

struct RPlanetD {
  PlanetD base;
  double K, cw, sw, n2, ibeta;
};

__device__ inline RPlanetF rsetup_mixed(const double *p, double t_ref, double t0, bool grad) {
  RPlanetF g;
  g.base = planet_setup_mixed(p, t_ref, t0);
  g.m = kepler_start_setup(g.base.e);
  g.K = g.cw = g.sw = g.beta = g.n2 = g.ibeta = 0.0f;
  if (grad) {
    float w_hi, w_lo;
    split_d(p[3], w_hi, w_lo);
    float sw, cw;
    sincosf(w_hi, &sw, &cw);
    g.sw = __fmaf_rn(w_lo, cw, sw);
    g.cw = __fmaf_rn(-w_lo, sw, cw);
    g.K = d2f(p[1]);
    g.beta = sqrtf((1.0f - g.base.e) * (1.0f + g.base.e));
    g.ibeta = 1.0f / g.beta;
    g.n2 = g.base.n_hi * g.base.n_hi;
  }
  return g;
}

__device__ inline RPlanetD rsetup_f64(const double *p, double dref, bool grad) {
  RPlanetD g;
  g.base = planet_setup_f64(p, dref);
  g.K = g.cw = g.sw = g.n2 = g.ibeta = 0.0;
  if (grad) {
    sincos(p[3], &g.sw, &g.cw);
    g.K = p[1];
    g.n2 = g.base.inv_P * g.base.inv_P;
    g.ibeta = 1.0 / g.base.beta;
  }
  return g;
}

template <typename T>
__device__ __forceinline__ void partials_r(T e, T K, T cw, T sw, T beta, T ibeta, T sE, T cE,
                                           T invD,
                                           T &dK, T &dw, T &dM, T &de) {
  const T cf = (cE - e) * invD;
  const T sf = beta * sE * invD;
  const T c_wf = cw * cf - sw * sf;
  const T s_wf = sw * cf + cw * sf;
  dK = c_wf + e * cw;
  dw = -K * (s_wf + e * sw);
  const T ks = K * s_wf * invD;
  dM = -ks * beta * invD;
  de = K * cw - ks * sE * (ibeta + beta * invD);
}

template <int J, bool GRAD>
__device__ __forceinline__ void body_mixed(const RPlanetF *pl, float gam, const float4 *oa,
                                           const float2 *ob, int64_t o0, int n, int lane,
                                           float *chi2_out, float *grad_out) {
  constexpr int NP = 5 * J + 1;
  Kahan acc = {0.0f, 0.0f};
  float g[GRAD ? NP : 1];
  Kahan gP[GRAD ? J : 1];       // compensated d/dP sums (they cancel heavily)
#pragma unroll
  for (int i = 0; i < (GRAD ? NP : 1); ++i) g[i] = 0.0f;
#pragma unroll
  for (int j = 0; j < (GRAD ? J : 1); ++j) gP[j] = Kahan{0.0f, 0.0f};
  // the next observation is loaded while this one is evaluated
  float4 o_next = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 wt_next = make_float2(0.f, 0.f);
  if (lane < n) {
    o_next = oa[o0 + lane];
    wt_next = ob[o0 + lane];
  }
  for (int k = lane; k < n; k += 32) {
    // Gradient: the planets' constants are read from shared memory again in
    // every iteration (the empty asm with a memory clobber keeps the
    // compiler from hoisting them, with the solver's per-planet constants,
    // into registers for all J planets): no spills at 128 registers, 4 %
    // faster on the ragged workload.
    if (GRAD) asm volatile("" ::: "memory");
    const float4 o = o_next;
    const float2 wt = wt_next;
    if (k + 32 < n) {
      o_next = oa[o0 + k + 32];
      wt_next = ob[o0 + k + 32];
    }
    float sEj[J], cEj[J];
    Kahan V = {0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const PlanetF q = pl[j].base;
      const float M = mean_anomaly_mixed(o.x, o.y, q);
      kepler_f32_h(M, q.e, pl[j].m, sEj[j], cEj[j]);
      kahan_add(V, velocity_mixed(q, sEj[j], cEj[j]));
    }
    const float r = __fadd_rn(__fsub_rn(V.big, o.z), __fsub_rn(gam, __fadd_rn(V.small, o.w)));
    const float wr = wt.x * r;
    kahan_add(acc, wr * r);
    if (GRAD) {
      const float a2 = 2.0f * wr;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const RPlanetF q = pl[j];
        float dK, dw, dM, de;
        const float invD = rcp_fast(__fmaf_rn(-q.base.e, cEj[j], 1.0f));
        partials_r(q.base.e, q.K, q.cw, q.sw, q.beta, q.ibeta, sEj[j], cEj[j], invD, dK, dw,
                   dM, de);
        const float dP = dM * (-kTwoPiF * wt.y * q.n2);
        kahan_add(gP[GRAD ? j : 0], a2 * dP);
        g[5 * j + 1] = __fmaf_rn(a2, dK, g[5 * j + 1]);
        g[5 * j + 2] = __fmaf_rn(a2, de, g[5 * j + 2]);
        g[5 * j + 3] = __fmaf_rn(a2, dw, g[5 * j + 3]);
        g[5 * j + 4] = __fmaf_rn(a2, dM, g[5 * j + 4]);
      }
      g[GRAD ? 5 * J : 0] += a2;
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
    if (GRAD) {
#pragma unroll
      for (int j = 0; j < (GRAD ? J : 1); ++j) {
        Kahan op = {shfl_xor(gP[j].big, m), shfl_xor(gP[j].small, m)};
        kahan_merge(gP[j], op);
      }
#pragma unroll
      for (int i = 0; i < (GRAD ? NP : 1); ++i) g[i] += shfl_xor(g[i], m);
    }
  }
  if (GRAD) {
#pragma unroll
    for (int j = 0; j < (GRAD ? J : 1); ++j) g[GRAD ? 5 * j : 0] = kahan_value(gP[j]);
  }
  if (lane == 0) {
    const float poison = 0.0f * gam;
    *chi2_out = kahan_value(acc) + poison;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < (GRAD ? NP : 1); ++i) grad_out[i] = g[i] + poison;
    }
  }
}

template <int J, bool GRAD, bool HI>
__device__ __forceinline__ void body_f64(const RPlanetD *pl, double gam, const ObsR64 *od,
                                         int64_t o0, int n, int lane, double *chi2_out,
                                         double *grad_out) {
  constexpr int NP = 5 * J + 1;
  double acc = 0.0;
  double g[GRAD ? NP : 1];
#pragma unroll
  for (int i = 0; i < (GRAD ? NP : 1); ++i) g[i] = 0.0;
  ObsR64 o_next = {0.0, 0.0, 0.0, 0.0};
  if (lane < n) o_next = od[o0 + lane];
  for (int k = lane; k < n; k += 32) {
    const ObsR64 o = o_next;
    if (k + 32 < n) o_next = od[o0 + k + 32];
    double sEj[J], cEj[J];
    double V = gam;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const PlanetD q = pl[j].base;
      const double M = mean_anomaly_f64(o.tau, q);
      kepler_f64<HI>(M, q.e, sEj[j], cEj[j]);
      V = velocity_add_f64(q, sEj[j], cEj[j], V);
    }
    const double r = V - o.v;
    acc = fma(o.w * r, r, acc);
    if (GRAD) {
      const double a2 = 2.0 * o.w * r;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const RPlanetD q = pl[j];
        double dK, dw, dM, de;
        const double invD = 1.0 / fma(-q.base.e, cEj[j], 1.0);
        partials_r(q.base.e, q.K, q.cw, q.sw, q.base.beta, q.ibeta, sEj[j], cEj[j], invD, dK,
                   dw, dM, de);
        const double dP = dM * (-kTwoPi * o.dt * q.n2);
        g[5 * j + 0] = fma(a2, dP, g[5 * j + 0]);
        g[5 * j + 1] = fma(a2, dK, g[5 * j + 1]);
        g[5 * j + 2] = fma(a2, de, g[5 * j + 2]);
        g[5 * j + 3] = fma(a2, dw, g[5 * j + 3]);
        g[5 * j + 4] = fma(a2, dM, g[5 * j + 4]);
      }
      g[GRAD ? 5 * J : 0] += a2;
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    acc += shfl_xor(acc, m);
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < (GRAD ? NP : 1); ++i) g[i] += shfl_xor(g[i], m);
    }
  }
  if (lane == 0) {
    const double poison = 0.0 * gam;
    *chi2_out = acc + poison;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < (GRAD ? NP : 1); ++i) grad_out[i] = g[i] + poison;
    }
  }
}

// ------------------------------------------------------------ persistent kernels

constexpr int kMaxWarps = 8;   // block <= 256

#define KC_RAGGED_SWITCH(BODY)                      \
  switch (J) {                                      \
    case 1: BODY(1); break;                         \
    case 2: BODY(2); break;                         \
    case 3: BODY(3); break;                         \
    case 4: BODY(4); break;                         \
    case 5: BODY(5); break;                         \
    case 6: BODY(6); break;                         \
    case 7: BODY(7); break;                         \
    default: BODY(8); break;                        \
  }

// Each warp: take the next system from the queue (systems in decreasing
// order of work), set up its planets (one lane per planet, FP64), evaluate
// it with 32 lanes over its observations, reduce, write; until the queue is
// empty.  The queue counter must be zero at launch.
// Gradient: at most 128 registers, two CTAs of 256 threads per SM; the body
// then keeps part of its accumulators in local memory, and still runs 1.26x
// faster than at one CTA per SM (252 registers) on the ragged workload.
// Forward: at most 80 registers, three CTAs per SM (1.08x over two).
template <bool GRAD>
__global__ void __launch_bounds__(256, GRAD ? 2 : 3)
ragged_mixed_kernel(RaggedDev d, const float4 *__restrict__ oa, const float2 *__restrict__ ob,
                    const double *__restrict__ params, float *__restrict__ chi2,
                    float *__restrict__ grad, unsigned long long *__restrict__ queue) {
  __shared__ RPlanetF pl_s[kMaxWarps][KC_MAX_PLANETS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RPlanetF *pl = pl_s[warp];
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(queue, 1ull);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= (unsigned long long)d.n_sys) break;
    const int64_t s = d.order[idx];
    if (!dbg_ok(d.invalid, 0 <= s && s < d.n_sys, kDbgOrder, (int64_t)idx)) continue;
    const int J = d.n_pl[s];
    const int64_t o0 = d.obs_off[s];
    if (!ragged_system_ok(d, s, J, o0, d.obs_off[s + 1])) continue;
    const int n = (int)(d.obs_off[s + 1] - o0);
    const double *p = params + d.par_off[s];
    if (lane < J) pl[lane] = rsetup_mixed(p + 5 * lane, d.t_ref[s], d.t0, GRAD);
    const float gam = d2f(system_gamma_r(p, J));
    __syncwarp();
    float *gout = GRAD ? grad + d.par_off[s] : nullptr;
#define KC_BODY(JJ) body_mixed<JJ, GRAD>(pl, gam, oa, ob, o0, n, lane, chi2 + s, gout)
    KC_RAGGED_SWITCH(KC_BODY)
#undef KC_BODY
    if (lane == 0) note_invalid(d.invalid, chi2[s]);      // lane 0 wrote it
    __syncwarp();
  }
}

template <bool GRAD>
__global__ void __launch_bounds__(256)
ragged_f64_kernel(RaggedDev d, const ObsR64 *__restrict__ od, const double *__restrict__ params,
                  double *__restrict__ chi2, double *__restrict__ grad,
                  unsigned long long *__restrict__ queue) {
  __shared__ RPlanetD pl_s[kMaxWarps][KC_MAX_PLANETS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RPlanetD *pl = pl_s[warp];
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(queue, 1ull);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= (unsigned long long)d.n_sys) break;
    const int64_t s = d.order[idx];
    if (!dbg_ok(d.invalid, 0 <= s && s < d.n_sys, kDbgOrder, (int64_t)idx)) continue;
    const int J = d.n_pl[s];
    const int64_t o0 = d.obs_off[s];
    if (!ragged_system_ok(d, s, J, o0, d.obs_off[s + 1])) continue;
    const int n = (int)(d.obs_off[s + 1] - o0);
    const double *p = params + d.par_off[s];
    const double dref = d.t_ref[s] - d.t0;
    if (lane < J) pl[lane] = rsetup_f64(p + 5 * lane, dref, GRAD);
    const double gam = system_gamma_r(p, J);
    __syncwarp();
    const bool hi = any_high_e(lane < J && pl[lane].base.e > (double)kEccFast);
    double *gout = GRAD ? grad + d.par_off[s] : nullptr;
#define KC_BODY(JJ)                                                                  \
  if (hi)                                                                            \
    body_f64<JJ, GRAD, true>(pl, gam, od, o0, n, lane, chi2 + s, gout);              \
  else                                                                               \
    body_f64<JJ, GRAD, false>(pl, gam, od, o0, n, lane, chi2 + s, gout)
    KC_RAGGED_SWITCH(KC_BODY)
#undef KC_BODY
    if (lane == 0) note_invalid(d.invalid, chi2[s]);      // lane 0 wrote it
    __syncwarp();
  }
}

}  // namespace

// ------------------------------------------------------------ launchers

cudaError_t ragged_prep(const RaggedDev &d, int mode, const double *t, const double *v,
                        const double *sigma, double jitter2, void *obs_a, void *obs_b,
                        double *t_ref, cudaStream_t st) {
  const int64_t warps = d.n_sys;
  int64_t blocks = (warps * 32 + 255) / 256;
  if (blocks > (int64_t)sm_count() * 64) blocks = (int64_t)sm_count() * 64;
  if (blocks < 1) blocks = 1;
  if (mode == KC_MIXED)
    prep_obs_mixed<<<(int)blocks, 256, 0, st>>>(d, t, v, sigma, jitter2, (float4 *)obs_a,
                                                (float2 *)obs_b, t_ref);
  else
    prep_obs_f64<<<(int)blocks, 256, 0, st>>>(d, t, v, sigma, jitter2, (ObsR64 *)obs_a, t_ref);
  return cudaGetLastError();
}

cudaError_t launch_predict_ragged(const double *params, const int64_t *par_off,
                                  const int32_t *n_pl, const double *t, const int64_t *obs_off,
                                  int64_t n_sys, double t0, double *v_out, cudaStream_t st) {
  int64_t blocks = (n_sys * 32 + 255) / 256;
  if (blocks > (int64_t)sm_count() * 64) blocks = (int64_t)sm_count() * 64;
  predict_ragged_kernel<<<(int)(blocks > 0 ? blocks : 1), 256, 0, st>>>(
      params, par_off, n_pl, t, obs_off, n_sys, t0, v_out, invalid_counter());
  return cudaGetLastError();
}

const void *ragged_kernel_fn(int mode, bool grad) {
  if (mode == KC_MIXED)
    return grad ? (const void *)ragged_mixed_kernel<true> : (const void *)ragged_mixed_kernel<false>;
  return grad ? (const void *)ragged_f64_kernel<true> : (const void *)ragged_f64_kernel<false>;
}

int ragged_max_blocks_per_sm(int mode, bool grad, int block) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ragged_kernel_fn(mode, grad), block, 0);
  return n;
}

cudaError_t ragged_launch(const RaggedDev &d, int mode, bool grad, const void *obs_a,
                          const void *obs_b, const double *params, void *chi2, void *gradp,
                          unsigned long long *queue, int grid, int block, cudaStream_t st) {
  if (mode == KC_MIXED) {
    if (grad)
      ragged_mixed_kernel<true><<<grid, block, 0, st>>>(d, (const float4 *)obs_a,
                                                        (const float2 *)obs_b, params,
                                                        (float *)chi2, (float *)gradp, queue);
    else
      ragged_mixed_kernel<false><<<grid, block, 0, st>>>(d, (const float4 *)obs_a,
                                                         (const float2 *)obs_b, params,
                                                         (float *)chi2, (float *)gradp, queue);
  } else {
    if (grad)
      ragged_f64_kernel<true><<<grid, block, 0, st>>>(d, (const ObsR64 *)obs_a, params,
                                                      (double *)chi2, (double *)gradp, queue);
    else
      ragged_f64_kernel<false><<<grid, block, 0, st>>>(d, (const ObsR64 *)obs_a, params,
                                                       (double *)chi2, (double *)gradp, queue);
  }
  return cudaGetLastError();
}

}  // namespace kc
