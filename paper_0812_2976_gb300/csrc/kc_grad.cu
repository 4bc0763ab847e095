// kc_grad.cu -- adjoint of the fused chi-square: d chi2 / d(P, K, e, w, M0)
// for every planet and d chi2 / d gamma, for every system.
//
// Sec. 6 of the paper proposes evaluating partial derivatives of the
// goodness-of-fit statistic in parallel for derivative-based searches.  This
// kernel does it in the same pass as chi2, without storing anything per
// observation: per (observation, planet) it solves Kepler's equation (the
// same fixed-count solver as the forward kernel), keeps sin E and cos E
// in registers until the residual r_k of the observation is known, then adds
// 2 w_k r_k dv/dtheta to per-thread accumulators.  The derivatives follow
// from implicit differentiation of Kepler's equation,
//   dE = (dM + sin E de)/D,  D = 1 - e cos E,
// and of the true anomaly, df/dE = beta/D, df/de|E = sin E/(beta D) with
// beta = sqrt(1 - e^2):
//   dv/dK  = cos(w+f) + e cos w
//   dv/dw  = -K [sin(w+f) + e sin w]
//   dv/dM0 = -K sin(w+f) beta / D^2
//   dv/de  = K cos w - K sin(w+f) (sin E / D) (1/beta + beta/D)
//   dv/dP  = dv/dM0 * (-2 pi (t - t0) / P^2)     (frac() jumps ignored)
//   dV/dgamma = 1.
// Each system is handled by G <= 32 consecutive threads (one warp segment),
// combined by shuffles.
#include <cmath>

#include "kc_device.cuh"
#include "kc_internal.h"
#include "kc_tcgen05.cuh"

namespace kc {

namespace {

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Planet constants for the gradient, single precision.
// ibeta = 1/beta, once per planet: the partials need it per observation.
struct GradPlanetF {
  PlanetF base;    // phase and velocity constants of the forward path
  float K, cw, sw, beta, n2, ibeta;   // n2 = (1/P)^2
  StartF m;        // the e-only constants of Mikkola's start
};

struct GradPlanetD {
  PlanetD base;
  double K, cw, sw, n2, ibeta;
};

__device__ inline GradPlanetF grad_setup_mixed(const double *p, double t_ref, double t0) {
  GradPlanetF g;
  g.base = planet_setup_mixed(p, t_ref, t0);
  float w_hi, w_lo;
  split_d(p[3], w_hi, w_lo);
  float sw, cw;
  sincosf(w_hi, &sw, &cw);
  g.sw = __fmaf_rn(w_lo, cw, sw);
  g.cw = __fmaf_rn(-w_lo, sw, cw);
  g.K = d2f(p[1]);
  const float e = g.base.e;
  g.beta = sqrtf((1.0f - e) * (1.0f + e));
  g.ibeta = 1.0f / g.beta;
  const float n = g.base.n_hi;
  g.n2 = n * n;
  g.m = kepler_start_setup(e);
  return g;
}

__device__ inline GradPlanetD grad_setup_f64(const double *p, double dref) {
  GradPlanetD g;
  g.base = planet_setup_f64(p, dref);
  sincos(p[3], &g.sw, &g.cw);
  g.K = p[1];
  g.n2 = g.base.inv_P * g.base.inv_P;
  g.ibeta = 1.0 / g.base.beta;
  return g;
}

__device__ inline double nan_d() { return __longlong_as_double(0x7ff8000000000000ll); }

__device__ inline double system_gamma_g(const double *p, int J) {
  bool ok = finite_bits(p[5 * J]);
  for (int j = 0; j < J; ++j)
    ok = ok && planet_valid(p[5 * j], p[5 * j + 1], p[5 * j + 2], p[5 * j + 3], p[5 * j + 4]);
  return ok ? p[5 * J] : nan_d();
}

// Free jitter of a system whose parameters end with (gamma, sigma_j).
__device__ inline double system_jitter_g(const double *p, int J) {
  const double sj = p[5 * J + 1];
  return finite_bits(sj) ? sj : nan_d();
}

constexpr double kLn2PiG = 1.8378770664093454836;      // ln(2 pi)

__device__ inline double inv_variance_g(double sigma, double jitter2) {
  const double var = fma(sigma, sigma, jitter2);
  return (var > 0.0) ? 1.0 / var : nan_d();
}

template <typename T>
struct Partials {
  T dP, dK, de, dw, dM;
};

// Partials of one planet's velocity from sin E, cos E and 1/D,
// D = 1 - e cos E (shared by both precisions).
template <typename T>
__device__ __forceinline__ void velocity_partials(T e, T K, T cw, T sw, T beta, T ibeta, T sE, T cE,
                                                  T invD, Partials<T> &d) {
  const T cf = (cE - e) * invD;           // cos f
  const T sf = beta * sE * invD;          // sin f
  const T c_wf = cw * cf - sw * sf;       // cos(w + f)
  const T s_wf = sw * cf + cw * sf;       // sin(w + f)
  d.dK = c_wf + e * cw;
  d.dw = -K * (s_wf + e * sw);
  const T ks = K * s_wf * invD;
  d.dM = -ks * beta * invD;
  d.de = K * cw - ks * sE * (ibeta + beta * invD);
}

struct MixedGradLayout {
  size_t pl, gam, sj, obs, w, total;
  __host__ __device__ MixedGradLayout(int ST, int J, int obs_tile) {
    pl = 0;
    gam = pl + sizeof(GradPlanetF) * ST * J;
    sj = gam + sizeof(float) * ST;
    obs = align_up(sj + sizeof(float) * ST, 16);
    w = obs + sizeof(float4) * obs_tile;
    total = align_up(w + sizeof(float2) * obs_tile, 16);
  }
};

struct ObsGD {
  double tau, v, w, dt;    // dt = t - t0
};

struct F64GradLayout {
  size_t tab, pl, gam, sj, obs, total;
  __host__ __device__ F64GradLayout(int ST, int J, int obs_tile) {
    tab = 0;                                          // sin/cos table, 4 KB
    pl = tab + sizeof(double2) * kSinTabN;
    gam = pl + sizeof(GradPlanetD) * ST * J;
    sj = gam + sizeof(double) * ST;
    obs = align_up(sj + sizeof(double) * ST, 16);
    total = align_up(obs + sizeof(ObsGD) * obs_tile, 16);
  }
};

// ------------------------------------------------------------ mixed

// NLL = true: the free-jitter negative log-likelihood (see kc_fwd.cu) and
// its gradient, including d nll / d sigma_j = sigma_j sum_k w_k (1 - w_k r_k^2)
// (the planet and gamma terms carry w_k r_k instead of 2 w_k r_k).
template <int J, bool NLL = false>
__global__ void __launch_bounds__(256, 2)
grad_mixed_kernel(UniformArgs a, int G, int obs_tile, float *__restrict__ chi2_out,
                  float *__restrict__ grad_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NP = 5 * J + 1 + (NLL ? 1 : 0);
  const int block = blockDim.x;
  const int ST = block / G;
  const MixedGradLayout L(ST, J, obs_tile);
  GradPlanetF *pl_s = reinterpret_cast<GradPlanetF *>(smem + L.pl);
  float *gam_s = reinterpret_cast<float *>(smem + L.gam);
  float *sj_s = reinterpret_cast<float *>(smem + L.sj);
  float4 *obs_s = reinterpret_cast<float4 *>(smem + L.obs);
  float2 *wt_s = reinterpret_cast<float2 *>(smem + L.w);   // (w_k, t_k - t0)

  const int tid = threadIdx.x;
  const int64_t sys0 = (int64_t)blockIdx.x * ST;
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const Split3 tr3 = split3(t_ref), te3 = split3(a.t0);
  const float dref_f = (tr3.x0 - te3.x0) + (tr3.x1 - te3.x1);     // t_ref - t0, float
  const float jit2 = d2f(a.jitter2);

  for (int i = tid; i < ST * J; i += block) {
    const int sl = i / J, j = i - sl * J;
    const int64_t s = sys0 + sl;
    GradPlanetF q = {};
    if (s < a.n_sys && dbg_ok(a.invalid, s * NP + 5 * j + 4 < a.n_sys * NP, kDbgParam, s * NP))
      q = grad_setup_mixed(a.params + s * NP + 5 * j, t_ref, a.t0);
    pl_s[i] = q;
  }
  for (int i = tid; i < ST; i += block) {
    const int64_t s = sys0 + i;
    gam_s[i] = s < a.n_sys ? d2f(system_gamma_g(a.params + s * NP, J)) : 0.0f;
    if (NLL) sj_s[i] = s < a.n_sys ? d2f(system_jitter_g(a.params + s * NP, J)) : 0.0f;
  }

  const int sl = tid / G, c = tid - sl * G;
  const int64_t s = sys0 + sl;
  Kahan acc = {0.0f, 0.0f};
  // d/dP terms carry (t - t0)/P^2 and cancel heavily across observations, so
  // they are summed with compensation (plain FP32 sums lost up to ~3e-3)
  Kahan gP[J];
  float g[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = 0.0f;
#pragma unroll
  for (int j = 0; j < J; ++j) gP[j] = Kahan{0.0f, 0.0f};

  for (int k0 = 0; k0 < a.n_obs; k0 += obs_tile) {
    const int nk = min(obs_tile, a.n_obs - k0);
    __syncthreads();
    for (int k = tid; k < nk; k += block) {
      if (!dbg_ok(a.invalid, k0 + k < a.n_obs, kDbgObs, k0 + k)) continue;
      float th, tl, vh, vl;
      sub_ds(split3(a.t[k0 + k]), tr3, th, tl);
      split_d(a.v[k0 + k], vh, vl);
      obs_s[k] = make_float4(th, tl, vh, vl);
      const float sg = d2f(a.sigma[k0 + k]);
      const float var = __fmaf_rn(sg, sg, jit2);
      wt_s[k] = make_float2(NLL ? sg * sg : (var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000)),
                            th + dref_f);
    }
    __syncthreads();
    const float gam = gam_s[sl];
    const float sj = NLL ? sj_s[sl] : 0.0f;
    const GradPlanetF *q = pl_s + sl * J;
    for (int k = c; k < nk; k += G) {
      const float4 o = obs_s[k];
      const float2 wt = wt_s[k];
      float sEj[J], cEj[J];
      Kahan V = {0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const PlanetF p = q[j].base;
        const float M = mean_anomaly_mixed(o.x, o.y, p);
        kepler_f32_h(M, p.e, q[j].m, sEj[j], cEj[j]);
        kahan_add(V, velocity_mixed(p, sEj[j], cEj[j]));
      }
      const float r = __fadd_rn(__fsub_rn(V.big, o.z), __fsub_rn(gam, __fadd_rn(V.small, o.w)));
      float wk = wt.x, a2;
      if (NLL) {
        const float var = __fmaf_rn(sj, sj, wt.x);           // sigma_k^2 + sigma_j^2
        wk = var > 0.0f ? rcp_fast(var) : __int_as_float(0x7fc00000);
        const float wr = wk * r;
        kahan_add(acc, __fmaf_rn(wr, r, lg2_fast(var) * 0.693147180559945309f));
        a2 = wr;
        g[NP - 1] = __fmaf_rn(sj * wk, __fmaf_rn(-wr, r, 1.0f), g[NP - 1]);
      } else {
        const float wr = wk * r;
        kahan_add(acc, wr * r);
        a2 = 2.0f * wr;
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const GradPlanetF qj = q[j];
        Partials<float> d;
        const float invD = rcp_fast(__fmaf_rn(-qj.base.e, cEj[j], 1.0f));
        velocity_partials(qj.base.e, qj.K, qj.cw, qj.sw, qj.beta, qj.ibeta, sEj[j], cEj[j], invD,
                            d);
        d.dP = d.dM * (-kTwoPiF * wt.y * qj.n2);
        kahan_add(gP[j], a2 * d.dP);
        g[5 * j + 1] = fmaf(a2, d.dK, g[5 * j + 1]);
        g[5 * j + 2] = fmaf(a2, d.de, g[5 * j + 2]);
        g[5 * j + 3] = fmaf(a2, d.dw, g[5 * j + 3]);
        g[5 * j + 4] = fmaf(a2, d.dM, g[5 * j + 4]);
      }
      g[5 * J] += a2;
    }
  }

  for (int m = G >> 1; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      Kahan op = {shfl_xor(gP[j].big, m), shfl_xor(gP[j].small, m)};
      kahan_merge(gP[j], op);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) g[i] += shfl_xor(g[i], m);
  }
#pragma unroll
  for (int j = 0; j < J; ++j) g[5 * j] = kahan_value(gP[j]);
  if (c == 0 && s < a.n_sys) {
    // NaN for an invalid system
    const float poison = 0.0f * gam_s[sl] + (NLL ? 0.0f * sj_s[sl] : 0.0f);
    const float value = NLL ? 0.5f * (kahan_value(acc) + (float)a.n_obs * (float)kLn2PiG) + poison
                            : kahan_value(acc) + poison;
    if (chi2_out) chi2_out[s] = value;
    note_invalid(a.invalid, value);
#pragma unroll
    for (int i = 0; i < NP; ++i) grad_out[s * NP + i] = g[i] + poison;
  }
}

// ------------------------------------------------------------ FP64

template <int J, bool NLL = false>
__global__ void __launch_bounds__(256)
grad_f64_kernel(UniformArgs a, int G, int obs_tile, double *__restrict__ chi2_out,
                double *__restrict__ grad_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NP = 5 * J + 1 + (NLL ? 1 : 0);
  const int block = blockDim.x;
  const int ST = block / G;
  const F64GradLayout L(ST, J, obs_tile);
  double2 *tab_s = reinterpret_cast<double2 *>(smem + L.tab);
  GradPlanetD *pl_s = reinterpret_cast<GradPlanetD *>(smem + L.pl);
  double *gam_s = reinterpret_cast<double *>(smem + L.gam);
  double *sj_s = reinterpret_cast<double *>(smem + L.sj);
  ObsGD *obs_s = reinterpret_cast<ObsGD *>(smem + L.obs);

  const int tid = threadIdx.x;
  const int64_t sys0 = (int64_t)blockIdx.x * ST;
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const double dref = t_ref - a.t0;
  sincos_table_build(tab_s, tid, block);      // read after the tile loop's first barrier

  for (int i = (tid & 31) * (block >> 5) + (tid >> 5); i < ST * J; i += block) {
    const int sl = i / J, j = i - sl * J;
    const int64_t s = sys0 + sl;
    GradPlanetD q = {};
    if (s < a.n_sys && dbg_ok(a.invalid, s * NP + 5 * j + 4 < a.n_sys * NP, kDbgParam, s * NP))
      q = grad_setup_f64(a.params + s * NP + 5 * j, dref);
    pl_s[i] = q;
  }
  for (int i = tid; i < ST; i += block) {
    const int64_t s = sys0 + i;
    gam_s[i] = s < a.n_sys ? system_gamma_g(a.params + s * NP, J) : 0.0;
    if (NLL) sj_s[i] = s < a.n_sys ? system_jitter_g(a.params + s * NP, J) : 0.0;
  }

  const int sl = tid / G, c = tid - sl * G;
  const int64_t s = sys0 + sl;
  double acc = 0.0;
  double g[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = 0.0;

  for (int k0 = 0; k0 < a.n_obs; k0 += obs_tile) {
    const int nk = min(obs_tile, a.n_obs - k0);
    __syncthreads();
    for (int k = tid; k < nk; k += block) {
      if (!dbg_ok(a.invalid, k0 + k < a.n_obs, kDbgObs, k0 + k)) continue;
      ObsGD o;
      const double tk = a.t[k0 + k];
      o.tau = tk - t_ref;
      o.v = a.v[k0 + k];
      o.w = NLL ? a.sigma[k0 + k] * a.sigma[k0 + k] : inv_variance_g(a.sigma[k0 + k], a.jitter2);
      o.dt = tk - a.t0;
      obs_s[k] = o;
    }
    __syncthreads();
    const double gam = gam_s[sl];
    const GradPlanetD *q = pl_s + sl * J;
    bool hi = false;
#pragma unroll
    for (int j = 0; j < J; ++j) hi = hi || q[j].base.e > (double)kEccFast;
    with_high_e(any_high_e(hi), [&](auto tag) {
      constexpr bool HI = decltype(tag)::value;
      for (int k = c; k < nk; k += G) {
        const ObsGD o = obs_s[k];
        double sEj[J], cEj[J];
        double V = gam;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const PlanetD p = q[j].base;
          const double M = mean_anomaly_f64(o.tau, p);
          kepler_f64<HI>(M, p.e, sEj[j], cEj[j], tab_s);
          V = velocity_add_f64(p, sEj[j], cEj[j], V);
        }
        const double r = V - o.v;
        double a2;
        if (NLL) {
          const double sj = sj_s[sl];
          const double var = fma(sj, sj, o.w);
          const double wk = var > 0.0 ? 1.0 / var : nan_d();
          acc += fma(wk * r, r, log(var));
          a2 = wk * r;
          g[NP - 1] = fma(sj * wk, fma(-wk * r, r, 1.0), g[NP - 1]);
        } else {
          acc = fma(o.w * r, r, acc);
          a2 = 2.0 * o.w * r;
        }
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const GradPlanetD qj = q[j];
          Partials<double> d;
          const double invD = 1.0 / fma(-qj.base.e, cEj[j], 1.0);
          velocity_partials(qj.base.e, qj.K, qj.cw, qj.sw, qj.base.beta, qj.ibeta, sEj[j], cEj[j],
                            invD, d);
          d.dP = d.dM * (-kTwoPi * o.dt * qj.n2);
          g[5 * j + 0] = fma(a2, d.dP, g[5 * j + 0]);
          g[5 * j + 1] = fma(a2, d.dK, g[5 * j + 1]);
          g[5 * j + 2] = fma(a2, d.de, g[5 * j + 2]);
          g[5 * j + 3] = fma(a2, d.dw, g[5 * j + 3]);
          g[5 * j + 4] = fma(a2, d.dM, g[5 * j + 4]);
        }
        g[5 * J] += a2;
      }
    });
  }

  for (int m = G >> 1; m >= 1; m >>= 1) {
    acc += shfl_xor(acc, m);
#pragma unroll
    for (int i = 0; i < NP; ++i) g[i] += shfl_xor(g[i], m);
  }
  if (c == 0 && s < a.n_sys) {
    const double poison = 0.0 * gam_s[sl] + (NLL ? 0.0 * sj_s[sl] : 0.0);
    const double value = NLL ? 0.5 * (acc + a.n_obs * kLn2PiG) + poison : acc + poison;
    if (chi2_out) chi2_out[s] = value;
    note_invalid(a.invalid, value);
#pragma unroll
    for (int i = 0; i < NP; ++i) grad_out[s * NP + i] = g[i] + poison;
  }
}

// ------------------------------------------------------------ Gauss-Newton
//
// H = sum_k w_k J_k J_k^T per system (J_k = dV_k/dtheta), with chi2 and its
// gradient from the same pass: the matrix and the right-hand side of a
// Levenberg-Marquardt step (Sec. 6 lists derivatives for least-squares
// refinement as future work).  One warp per system; each lane evaluates one
// observation of a batch of 32 and writes u_k = sqrt(w_k) J_k as a row of a
// 32 x n matrix U in shared memory; the warp then adds U^T U to its
// accumulators.  Mixed path: that update is a rank-32 dense contraction per
// batch on the tensor cores (mma.sync m16n8k8 here; the tcgen05 form
// follows), TF32 inputs in the three-
// product split hi*hi + hi*lo + lo*hi, FP32 accumulation), only the tiles
// on or above the diagonal.  Each element of U is split into its (hi, lo)
// pair once, when its row is written; since B = U and A = U^T cover the
// same elements, the B fragments are halves of the A fragments.  FP64 path:
// FMAs on the FP64 pipe, the packed upper-triangle entries spread over the
// lanes.

constexpr int kGnWarps = 4;      // mixed: systems (warps) per CTA
constexpr int kGnWarpsD = 2;     // FP64
constexpr int kGnObsTile = 256;

__host__ __device__ constexpr int gn_np(int J) { return 5 * J + 1; }
__host__ __device__ constexpr int gn_mt(int J) { return (gn_np(J) + 15) / 16; }
__host__ __device__ constexpr int gn_nt(int J) { return (gn_np(J) + 7) / 8; }
// Row stride of U in (hi, lo) pairs: the tiled width 16 MT (>= 8 NT) plus 4,
// which is 4 mod 16 pairs, so that with the column swizzle below the 64-bit
// row writes and fragment loads of each half-warp hit 32 different banks.
__host__ __device__ constexpr int gn_row2(int J) { return gn_mt(J) * 16 + 4; }

struct GnMixedLayout {
  size_t pl, gam, obs, w, u, total;
  __host__ __device__ GnMixedLayout(int J, int obs_tile) {
    pl = 0;
    gam = pl + sizeof(GradPlanetF) * kGnWarps * J;
    obs = align_up(gam + sizeof(float) * kGnWarps, 16);
    w = obs + sizeof(float4) * obs_tile;
    u = align_up(w + sizeof(float4) * obs_tile, 16);
    total = align_up(u + sizeof(float2) * kGnWarps * 32 * gn_row2(J), 16);
  }
};

struct GnF64Layout {
  size_t pl, gam, obs, pq, u, total;
  __host__ __device__ GnF64Layout(int J, int obs_tile) {
    const int np = gn_np(J), ntri = np * (np + 1) / 2;
    pl = 0;
    gam = pl + sizeof(GradPlanetD) * kGnWarpsD * J;
    obs = align_up(gam + sizeof(double) * kGnWarpsD, 16);
    pq = obs + sizeof(ObsGD) * obs_tile;
    u = align_up(pq + sizeof(short2) * ntri, 16);
    total = align_up(u + sizeof(double) * kGnWarpsD * 32 * (np | 1), 16);
  }
};

// Index of H[p][q], q >= p, in the packed upper triangle (row by row).
__device__ __forceinline__ int tri_index(int np, int p, int q) {
  return p * np - (p * (p - 1)) / 2 + (q - p);
}

// x = hi + lo + err with hi, lo TF32 numbers (FP32 with the 13 low
// significand bits zero): hi keeps the leading 11 significant bits of x, so
// |x - hi| < 2^-10 |x| and x - hi is exact in FP32; lo keeps the leading 11
// bits of x - hi, so |err| < 2^-20 |x|.  A product from the three terms
// hi*hi + hi*lo + lo*hi is then within about 3 * 2^-20 of the FP32 one.
__device__ __forceinline__ float2 tf32_pair(float x) {
  constexpr unsigned kTf32Mask = 0xffffe000u;
  const float hi = __uint_as_float(__float_as_uint(x) & kTf32Mask);
  const float lo = __uint_as_float(__float_as_uint(__fsub_rn(x, hi)) & kTf32Mask);
  return make_float2(hi, lo);
}

// One observation of the Gauss-Newton pass for the lane: its chi2 and
// gradient terms are added to acc, gP, g, and its row u = sqrt(w) J written
// to urow.  A lane past the batch's end evaluates a valid observation with
// weight 0, so all lanes run the same instructions.
template <int J>
__device__ __forceinline__ void gn_obs(const float4 &o, const float4 &wt, bool live, float gam,
                                       const GradPlanetF (&qr)[J], Kahan &acc, Kahan (&gP)[J],
                                       float (&g)[5 * J + 1], float (&urow)[5 * J + 1]) {
  float sEj[J], cEj[J];
  Kahan V = {0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const PlanetF &p = qr[j].base;
    const float M = mean_anomaly_mixed(o.x, o.y, p);
    kepler_f32_h(M, p.e, qr[j].m, sEj[j], cEj[j]);
    kahan_add(V, velocity_mixed(p, sEj[j], cEj[j]));
  }
  const float r = __fadd_rn(__fsub_rn(V.big, o.z), __fsub_rn(gam, __fadd_rn(V.small, o.w)));
  const float wk = live ? wt.x : 0.0f, wr = wk * r, a2 = 2.0f * wr;
  kahan_add(acc, wr * r);
  const float sw = live ? wt.z : 0.0f;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const GradPlanetF &qj = qr[j];
    Partials<float> d;
    const float invD = rcp_fast(__fmaf_rn(-qj.base.e, cEj[j], 1.0f));
    velocity_partials(qj.base.e, qj.K, qj.cw, qj.sw, qj.beta, qj.ibeta, sEj[j], cEj[j], invD, d);
    d.dP = d.dM * (-kTwoPiF * wt.y * qj.n2);
    kahan_add(gP[j], a2 * d.dP);
    g[5 * j + 1] = fmaf(a2, d.dK, g[5 * j + 1]);
    g[5 * j + 2] = fmaf(a2, d.de, g[5 * j + 2]);
    g[5 * j + 3] = fmaf(a2, d.dw, g[5 * j + 3]);
    g[5 * j + 4] = fmaf(a2, d.dM, g[5 * j + 4]);
    urow[5 * j + 0] = sw * d.dP;
    urow[5 * j + 1] = sw * d.dK;
    urow[5 * j + 2] = sw * d.de;
    urow[5 * j + 3] = sw * d.dw;
    urow[5 * j + 4] = sw * d.dM;
  }
  g[5 * J] += a2;
  urow[5 * J] = sw;
}

// D = A B + D for one 16 x 8 tile, A 16 x 8 (row), B 8 x 8 (col), TF32.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int J>
__global__ void __launch_bounds__(kGnWarps * 32)
gn_mixed_kernel(UniformArgs a, float *__restrict__ chi2_out, float *__restrict__ grad_out,
                float *__restrict__ jtj_out) {
  constexpr int NP = gn_np(J), MT = gn_mt(J), NT = gn_nt(J), ROW2 = gn_row2(J);
  constexpr int NTRI = NP * (NP + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const GnMixedLayout L(J, kGnObsTile);
  GradPlanetF *pl_s = reinterpret_cast<GradPlanetF *>(smem + L.pl);
  float *gam_s = reinterpret_cast<float *>(smem + L.gam);
  float4 *obs_s = reinterpret_cast<float4 *>(smem + L.obs);
  float4 *wt_s = reinterpret_cast<float4 *>(smem + L.w);
  float2 *u_all = reinterpret_cast<float2 *>(smem + L.u);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int block = kGnWarps * 32;
  const int64_t sys0 = (int64_t)blockIdx.x * kGnWarps;
  const int64_t s = sys0 + warp;
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const Split3 tr3 = split3(t_ref), te3 = split3(a.t0);
  const float dref_f = (tr3.x0 - te3.x0) + (tr3.x1 - te3.x1);     // t_ref - t0
  const float jit2 = d2f(a.jitter2);

  for (int i = tid; i < kGnWarps * J; i += block) {
    const int64_t si = sys0 + i / J;
    GradPlanetF q = {};
    if (si < a.n_sys &&
        dbg_ok(a.invalid, si * NP + 5 * (i % J) + 4 < a.n_sys * NP, kDbgParam, si * NP))
      q = grad_setup_mixed(a.params + si * NP + 5 * (i % J), t_ref, a.t0);
    pl_s[i] = q;
  }
  for (int i = tid; i < kGnWarps; i += block)
    gam_s[i] = sys0 + i < a.n_sys ? d2f(system_gamma_g(a.params + (sys0 + i) * NP, J)) : 0.0f;
  for (int i = tid; i < kGnWarps * 32 * ROW2; i += block)
    u_all[i] = make_float2(0.0f, 0.0f);                           // incl. padding

  // The (hi, lo) pair of element (row r, column c) of U sits at
  // r * ROW2 + (c ^ ((r >> 2) & 3)): with ROW2 = 4 mod 16 both the row writes
  // (one row per lane) and the fragment loads touch 32 different banks in
  // each half-warp.
  float2 *u = u_all + warp * 32 * ROW2;
  const int gid = lane >> 2, tig = lane & 3;
  const int sw_row = (lane >> 2) & 3;
  Kahan acc = {0.0f, 0.0f};
  Kahan gP[J];
  float g[NP];
  float C[MT][NT][4];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = 0.0f;
#pragma unroll
  for (int j = 0; j < J; ++j) gP[j] = Kahan{0.0f, 0.0f};
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) C[mt][nt][i] = 0.0f;

  for (int k0 = 0; k0 < a.n_obs; k0 += kGnObsTile) {
    const int nk = min(kGnObsTile, a.n_obs - k0);
    __syncthreads();
    for (int k = tid; k < nk; k += block) {
      if (!dbg_ok(a.invalid, k0 + k < a.n_obs, kDbgObs, k0 + k)) continue;
      float th, tl, vh, vl;
      sub_ds(split3(a.t[k0 + k]), tr3, th, tl);
      split_d(a.v[k0 + k], vh, vl);
      obs_s[k] = make_float4(th, tl, vh, vl);
      const float sg = d2f(a.sigma[k0 + k]);
      const float var = __fmaf_rn(sg, sg, jit2);
      const float wk = var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000);
      wt_s[k] = make_float4(wk, th + dref_f, sqrtf(wk), 0.0f);
    }
    __syncthreads();
    const float gam = gam_s[warp];
    const GradPlanetF *q = pl_s + warp * J;
    for (int kb = 0; kb < nk; kb += 32) {
      const int k = kb + lane;
      float urow[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) urow[i] = 0.0f;
      if (k < nk) {
        const float4 o = obs_s[k];
        const float4 wt = wt_s[k];
        float sEj[J], cEj[J];
        Kahan V = {0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const PlanetF p = q[j].base;
          const float M = mean_anomaly_mixed(o.x, o.y, p);
          kepler_f32_h(M, p.e, q[j].m, sEj[j], cEj[j]);
          kahan_add(V, velocity_mixed(p, sEj[j], cEj[j]));
        }
        const float r = __fadd_rn(__fsub_rn(V.big, o.z), __fsub_rn(gam, __fadd_rn(V.small, o.w)));
        const float wk = wt.x, wr = wk * r, a2 = 2.0f * wr;
        kahan_add(acc, wr * r);
        const float sw = wt.z;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const GradPlanetF qj = q[j];
          Partials<float> d;
          const float invD = rcp_fast(__fmaf_rn(-qj.base.e, cEj[j], 1.0f));
          velocity_partials(qj.base.e, qj.K, qj.cw, qj.sw, qj.beta, qj.ibeta, sEj[j], cEj[j], invD,
                            d);
          d.dP = d.dM * (-kTwoPiF * wt.y * qj.n2);
          kahan_add(gP[j], a2 * d.dP);
          g[5 * j + 1] = fmaf(a2, d.dK, g[5 * j + 1]);
          g[5 * j + 2] = fmaf(a2, d.de, g[5 * j + 2]);
          g[5 * j + 3] = fmaf(a2, d.dw, g[5 * j + 3]);
          g[5 * j + 4] = fmaf(a2, d.dM, g[5 * j + 4]);
          urow[5 * j + 0] = sw * d.dP;
          urow[5 * j + 1] = sw * d.dK;
          urow[5 * j + 2] = sw * d.de;
          urow[5 * j + 3] = sw * d.dw;
          urow[5 * j + 4] = sw * d.dM;
        }
        g[5 * J] += a2;
        urow[5 * J] = sw;
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) u[lane * ROW2 + (i ^ sw_row)] = tf32_pair(urow[i]);
      __syncwarp();
      // H += U^T U: k-steps of 8 rows; A = U^T (16 x 8 per m-tile), B = U (8 x 8 per n-tile)
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const float2 *r0 = u + (ks * 8 + tig) * ROW2;
        const float2 *r1 = r0 + 4 * ROW2;
        const int g0 = gid ^ ((2 * ks) & 3), g1 = gid ^ ((2 * ks + 1) & 3);   // row swizzles
        unsigned ah[MT][4], al[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const float2 x[4] = {r0[16 * mt + g0], r0[16 * mt + g0 + 8], r1[16 * mt + g1],
                               r1[16 * mt + g1 + 8]};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            ah[mt][i] = __float_as_uint(x[i].x);
            al[mt][i] = __float_as_uint(x[i].y);
          }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          // columns 8 nt .. 8 nt + 7 of U: half h of m-tile nt / 2
          const int m = nt >> 1, h = nt & 1;
          const unsigned bh[2] = {ah[m][h], ah[m][2 + h]}, bl[2] = {al[m][h], al[m][2 + h]};
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            if (8 * nt + 7 >= 16 * mt) {        // a tile on or above the diagonal
              mma_tf32(C[mt][nt], al[mt], bh);
              mma_tf32(C[mt][nt], ah[mt], bl);
              mma_tf32(C[mt][nt], ah[mt], bh);
            }
          }
        }
      }
      __syncwarp();
    }
  }

  for (int m = 16; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      Kahan op = {shfl_xor(gP[j].big, m), shfl_xor(gP[j].small, m)};
      kahan_merge(gP[j], op);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) g[i] += shfl_xor(g[i], m);
  }
#pragma unroll
  for (int j = 0; j < J; ++j) g[5 * j] = kahan_value(gP[j]);
  if (s >= a.n_sys) return;
  const float poison = 0.0f * gam_s[warp];             // NaN for an invalid system
  if (lane == 0) {
    const float value = kahan_value(acc) + poison;
    if (chi2_out) chi2_out[s] = value;
    note_invalid(a.invalid, value);
  }
  if (grad_out) {
#pragma unroll
    for (int i = 0; i < NP; ++i)
      if (lane == (i & 31)) grad_out[s * NP + i] = g[i] + poison;
  }
  float *H = jtj_out + s * NTRI;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      if (8 * nt + 7 < 16 * mt) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = 16 * mt + gid + (i >= 2 ? 8 : 0);
        const int col = 8 * nt + 2 * tig + (i & 1);
        if (row < NP && col < NP && col >= row) H[tri_index(NP, row, col)] = C[mt][nt][i] + poison;
      }
    }
}

// ---------------------------------------------- Gauss-Newton on tcgen05
//
// The same pass with the U^T U update on the fifth-generation tensor cores:
// the operands come from shared memory through matrix descriptors, the
// accumulator stays in tensor memory (TMEM) for the whole launch, and one
// thread issues each batch's MMAs, so the warps evaluating observations
// spend no issue slots or shared-memory loads on the contraction.  The
// smallest tcgen05 tile is M = 64 rows, four times one system's 16 (n_pl
// <= 3: 5 n_pl + 1 <= 16 parameters; rows beyond them never reach a kept
// entry), so the CTA's four warps write their systems' U^T rows into one
// 64-row tile (rows 16 w .. 16 w + 15 for warp w; TF32 (hi, lo) pairs as in
// gn_mixed_kernel, in two tiles, K-major, 128-byte swizzle), and thread 0
// issues the batch's MMAs (M = 64, N = 64, K = 8 per step).  H = U^T U is
// symmetric, so of the three products of the split, hi hi^T + lo hi^T +
// hi lo^T, the last is the transpose of the second: two accumulators in
// TMEM, D1 += hi hi^T and D2 += lo hi^T (two MMAs per K step, not three),
// give H = D1 + D2 + D2^T in the epilogue.  The four diagonal 16 x 16
// blocks are kept; 3/4 of the products are cross-system terms that are
// thrown away.  A batch is 64 observations, two per lane, evaluated side by
// side (two independent chains per planet for the scheduler); its tile is
// two 64 x 32 halves.  The order of the observations along K is free (the
// sum runs over all of them), so lane l puts its pair at K = 2l and 2l + 1
// and writes both words of an element with one 8-byte store.
// One tile suffices: a warp rewrites it only after evaluating the next 64
// observations, by which time the MMAs that read it have long completed
// (its lane 0 still waits on the mbarrier their commit arrives on).  A CTA
// barrier per batch hands the written tile to the issuing thread (on a
// GB300 this ran 822 us on 65536 x 3 x 512 against 891 us with a "full"
// mbarrier that let the other warps run a batch ahead of warp 0).  With
// M = 64 the accumulator's row r sits in TMEM lane 32 (r / 16) + r % 16, so
// warp w reads its system's blocks from its own lanes 32 w .. 32 w + 15,
// columns 16 w .. 16 w + 15 (D1) and 64 + 16 w .. 64 + 16 w + 15 (D2), and
// transposes D2's block through shared memory.  Every wait is bounded; a
// wait that gives up makes the CTA's results NaN (counted by the
// invalid-system counter) and the TMEM is still freed.

constexpr int kTcHalfBytes = 64 * 32 * 4;       // 64 rows x 32 observations, TF32
constexpr int kTcBatch = 64;                    // observations per batch
constexpr int kTcObsTile = 512;                 // observations staged at a time
constexpr int kTcCols = 128;                    // TMEM columns per CTA: D1, D2
constexpr uint64_t kTcWaitLimit = 20000000;     // ns an mbarrier wait may take (20 ms)

struct GnTcLayout {
  size_t u, pl, gam, obs, w, bar, slot, total;
  __host__ __device__ GnTcLayout(int J) {
    u = 0;                                       // hi halves, then lo halves: 1024-aligned
    pl = u + 4 * kTcHalfBytes;
    gam = pl + sizeof(GradPlanetF) * kGnWarps * J;
    obs = align_up(gam + sizeof(float) * kGnWarps, 16);
    w = obs + sizeof(float4) * kTcObsTile;
    bar = align_up(w + sizeof(float4) * kTcObsTile, 8);
    slot = bar + sizeof(uint64_t);
    total = align_up(slot + 16, 16) + 1024;     // 1024 bytes to align the base
  }
};

// Lane 0 waits; the warp learns the outcome (and is ordered after it).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, uint64_t limit, int lane) {
  bool ok = true;
  if (lane == 0) ok = tc::mbar_wait(bar, parity, limit);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// Writes the lane's two observations, columns 2 l and 2 l + 1 of U^T for
// lane l, into the tile: element (row 16 warp + p, column c) of a half
// (columns 0-31 and 32-63 of the batch) sits in 8-row group 2 warp + p / 8
// (1024 bytes each), row p % 8 (128 bytes), 16-byte chunk (c / 4) ^ (p % 8),
// word c % 4, so the pair is one aligned 8-byte word.  `rows` points at the
// lane's half, 8-row group and word; `lane_q` is its chunk before the
// swizzle.  The hi parts are TF32 (low 13 bits cleared), so that hi + lo is
// exact; the lo parts are stored whole: the tensor core takes their upper
// 19 bits, as clearing the rest here would (were it to round them instead,
// an element would move by less than 2^-20 of itself).
template <int NP>
__device__ __forceinline__ void gn_tc_store(unsigned char *rows, uint32_t lane_q,
                                            const float (&ua)[NP], const float (&ub)[NP]) {
  constexpr unsigned kTf32Mask = 0xffffe000u;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float ha = __uint_as_float(__float_as_uint(ua[p]) & kTf32Mask);
    const float hb = __uint_as_float(__float_as_uint(ub[p]) & kTf32Mask);
    const uint32_t off = (p >> 3) * 1024 + (p & 7) * 128 + ((lane_q ^ (p & 7)) << 4);
    *reinterpret_cast<float2 *>(rows + off) = make_float2(ha, hb);
    *reinterpret_cast<float2 *>(rows + 2 * kTcHalfBytes + off) =
        make_float2(__fsub_rn(ua[p], ha), __fsub_rn(ub[p], hb));
  }
}

template <int J>
__global__ void __launch_bounds__(kGnWarps * 32, 4)
gn_mixed_tc_kernel(UniformArgs a, float *__restrict__ chi2_out, float *__restrict__ grad_out,
                   float *__restrict__ jtj_out) {
  constexpr int NP = gn_np(J);
  constexpr int NTRI = NP * (NP + 1) / 2;
  static_assert(NP <= 16, "one system's U^T fits 16 rows of the M = 64 tile");
  static_assert(kGnWarps == 4, "four systems per M = 64 tile");
  constexpr uint32_t IDESC = tc::idesc_tf32(64, 64);
  constexpr int kThreads = kGnWarps * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  const GnTcLayout L(J);
  GradPlanetF *pl_s = reinterpret_cast<GradPlanetF *>(smem + L.pl);
  float *gam_s = reinterpret_cast<float *>(smem + L.gam);
  float4 *obs_s = reinterpret_cast<float4 *>(smem + L.obs);
  float4 *wt_s = reinterpret_cast<float4 *>(smem + L.w);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);   // commits of the MMAs
  uint32_t *slot = reinterpret_cast<uint32_t *>(smem + L.slot);
  unsigned char *tiles = smem + L.u;
  const uint32_t tiles_a = tc::smem_u32(tiles), bar_a = tc::smem_u32(bar);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t sys0 = (int64_t)blockIdx.x * kGnWarps;
  const int64_t s = sys0 + warp;

  if (warp == 0) tc::tmem_alloc(tc::smem_u32(slot), kTcCols);
  if (tid == 0) {
    tc::mbar_init(bar_a, 1);                   // one commit per batch
    tc::mbar_init_fence();
  }
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const Split3 tr3 = split3(t_ref), te3 = split3(a.t0);
  const float dref_f = (tr3.x0 - te3.x0) + (tr3.x1 - te3.x1);     // t_ref - t0
  const float jit2 = d2f(a.jitter2);
  for (int i = tid; i < kGnWarps * J; i += kThreads) {
    const int64_t si = sys0 + i / J;
    GradPlanetF q = {};
    if (si < a.n_sys &&
        dbg_ok(a.invalid, si * NP + 5 * (i % J) + 4 < a.n_sys * NP, kDbgParam, si * NP))
      q = grad_setup_mixed(a.params + si * NP + 5 * (i % J), t_ref, a.t0);
    pl_s[i] = q;
  }
  for (int i = tid; i < kGnWarps; i += kThreads)
    gam_s[i] = sys0 + i < a.n_sys ? d2f(system_gamma_g(a.params + (sys0 + i) * NP, J)) : 0.0f;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *slot;

  GradPlanetF qr[J];
#pragma unroll
  for (int j = 0; j < J; ++j) qr[j] = pl_s[warp * J + j];
  const float gam = gam_s[warp];
  // lane l: columns 2 l, 2 l + 1 of the batch, in half l / 16
  const uint32_t lane_q = (uint32_t)(lane & 15) >> 1;
  unsigned char *my_rows = tiles + (lane >> 4) * kTcHalfBytes + 2048 * warp + 8 * (lane & 1);
  // The descriptors of the batch's K steps differ from the tile's in the
  // start address alone (bits 0-13: the address / 16; the tiles end below
  // 2^18 bytes, so an offset adds without a carry out of the field).
  const uint64_t dtile = tc::desc_kmajor_sw128(tiles_a);
  Kahan acc = {0.0f, 0.0f};
  Kahan gP[J];
  float g[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = 0.0f;
#pragma unroll
  for (int j = 0; j < J; ++j) gP[j] = Kahan{0.0f, 0.0f};
  uint32_t nb = 0;                                   // batches (commits) so far
  bool ok = true;

  for (int k0 = 0; k0 < a.n_obs; k0 += kTcObsTile) {
    const int nk = min(kTcObsTile, a.n_obs - k0);
    __syncthreads();
    for (int k = tid; k < nk; k += kThreads) {
      if (!dbg_ok(a.invalid, k0 + k < a.n_obs, kDbgObs, k0 + k)) continue;
      float th, tl, vh, vl;
      sub_ds(split3(a.t[k0 + k]), tr3, th, tl);
      split_d(a.v[k0 + k], vh, vl);
      obs_s[k] = make_float4(th, tl, vh, vl);
      const float sg = d2f(a.sigma[k0 + k]);
      const float var = __fmaf_rn(sg, sg, jit2);
      const float wk = var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000);
      wt_s[k] = make_float4(wk, th + dref_f, sqrtf(wk), 0.0f);
    }
    __syncthreads();
    for (int kb = 0; kb < nk; kb += kTcBatch) {
      const int ka = kb + lane, kbb = kb + 32 + lane;
      const int ia = min(ka, nk - 1), ib = min(kbb, nk - 1);
      float ua[NP], ub[NP];
      gn_obs<J>(obs_s[ia], wt_s[ia], ka < nk, gam, qr, acc, gP, g, ua);
      gn_obs<J>(obs_s[ib], wt_s[ib], kbb < nk, gam, qr, acc, gP, g, ub);
      if (nb > 0 && ok)                  // the MMAs that read the tile before
        ok = warp_wait(bar_a, (nb - 1) & 1u, kTcWaitLimit, lane);
      gn_tc_store<NP>(my_rows, lane_q, ua, ub);
      tc::fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
          // K step ks: columns 8 ks .. 8 ks + 7 of the batch, in half ks / 4
          const uint32_t off = ((ks >> 2) * kTcHalfBytes + 32 * (ks & 3)) >> 4;
          const uint64_t hi = dtile + off, lo = dtile + off + (2 * kTcHalfBytes >> 4);
          const uint32_t accumulate = (nb | ks) != 0;
          tc::mma_tf32(taddr, hi, hi, IDESC, accumulate);                 // D1 += hi hi^T
          tc::mma_tf32(taddr + kTcCols / 2, lo, hi, IDESC, accumulate);   // D2 += lo hi^T
        }
        tc::commit(bar_a);
      }
      ++nb;
    }
  }

  // Every MMA is complete once the last commit's phase is; a longer wait if
  // a wait gave up before.
  float h[16];
  if (nb > 0) {
    const bool last_ok = warp_wait(bar_a, (nb - 1) & 1u, ok ? kTcWaitLimit : 4 * kTcWaitLimit,
                                   lane);
    ok = ok && last_ok;
    tc::fence_after_sync();
    const uint32_t blk = taddr + ((uint32_t)(32 * warp) << 16) + 16u * warp;
    float h2[16];
    tc::tmem_ld16(blk, h);
    tc::tmem_ld16(blk + kTcCols / 2, h2);
    // H = D1 + D2 + D2^T: lane r < 16 holds row r of both blocks; D2's is
    // transposed through 16 x 17 floats of the warp's own in the staged
    // observations' shared memory (read by no warp after the last batch's
    // barrier).
    float *tr = reinterpret_cast<float *>(obs_s) + warp * 16 * 17;
    if (lane < 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) tr[lane * 17 + i] = h2[i];
    }
    __syncwarp();
    if (lane < 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) h[i] += h2[i] + tr[i * 17 + lane];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) h[i] = 0.0f;
  }

  for (int m = 16; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      Kahan op = {shfl_xor(gP[j].big, m), shfl_xor(gP[j].small, m)};
      kahan_merge(gP[j], op);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) g[i] += shfl_xor(g[i], m);
  }
#pragma unroll
  for (int j = 0; j < J; ++j) g[5 * j] = kahan_value(gP[j]);
  if (s < a.n_sys) {
    // NaN for an invalid system, or where a wait on the tensor cores gave up
    const float poison = ok ? 0.0f * gam : __int_as_float(0x7fc00000);
    if (lane == 0) {
      const float value = kahan_value(acc) + poison;
      if (chi2_out) chi2_out[s] = value;
      note_invalid(a.invalid, value);
    }
    if (grad_out) {
#pragma unroll
      for (int i = 0; i < NP; ++i)
        if (lane == (i & 31)) grad_out[s * NP + i] = g[i] + poison;
    }
    float *H = jtj_out + s * NTRI;
    if (lane < NP) {
#pragma unroll
      for (int c = 0; c < NP; ++c)
        if (c >= lane) H[tri_index(NP, lane, c)] = h[c] + poison;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(taddr, kTcCols);
  }
}

template <int J>
__global__ void __launch_bounds__(kGnWarpsD * 32)
gn_f64_kernel(UniformArgs a, double *__restrict__ chi2_out, double *__restrict__ grad_out,
              double *__restrict__ jtj_out) {
  constexpr int NP = gn_np(J), ROWD = NP | 1;
  constexpr int NTRI = NP * (NP + 1) / 2, E = (NTRI + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const GnF64Layout L(J, kGnObsTile);
  GradPlanetD *pl_s = reinterpret_cast<GradPlanetD *>(smem + L.pl);
  double *gam_s = reinterpret_cast<double *>(smem + L.gam);
  ObsGD *obs_s = reinterpret_cast<ObsGD *>(smem + L.obs);
  short2 *pq_s = reinterpret_cast<short2 *>(smem + L.pq);
  double *u_all = reinterpret_cast<double *>(smem + L.u);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int block = kGnWarpsD * 32;
  const int64_t sys0 = (int64_t)blockIdx.x * kGnWarpsD;
  const int64_t s = sys0 + warp;
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const double dref = t_ref - a.t0;

  for (int i = tid; i < kGnWarpsD * J; i += block) {
    const int64_t si = sys0 + i / J;
    GradPlanetD q = {};
    if (si < a.n_sys &&
        dbg_ok(a.invalid, si * NP + 5 * (i % J) + 4 < a.n_sys * NP, kDbgParam, si * NP))
      q = grad_setup_f64(a.params + si * NP + 5 * (i % J), dref);
    pl_s[i] = q;
  }
  for (int i = tid; i < kGnWarpsD; i += block)
    gam_s[i] = sys0 + i < a.n_sys ? system_gamma_g(a.params + (sys0 + i) * NP, J) : 0.0;
  for (int p = tid; p < NP; p += block) {               // packed (p, q) table
    const int base = p * NP - (p * (p - 1)) / 2;
    for (int q = p; q < NP; ++q) pq_s[base + q - p] = make_short2((short)p, (short)q);
  }

  double *u = u_all + warp * 32 * ROWD;
  double acc = 0.0, g[NP], h[E];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = 0.0;
#pragma unroll
  for (int i = 0; i < E; ++i) h[i] = 0.0;

  for (int k0 = 0; k0 < a.n_obs; k0 += kGnObsTile) {
    const int nk = min(kGnObsTile, a.n_obs - k0);
    __syncthreads();
    for (int k = tid; k < nk; k += block) {
      if (!dbg_ok(a.invalid, k0 + k < a.n_obs, kDbgObs, k0 + k)) continue;
      ObsGD o;
      const double tk = a.t[k0 + k];
      o.tau = tk - t_ref;
      o.v = a.v[k0 + k];
      o.w = inv_variance_g(a.sigma[k0 + k], a.jitter2);
      o.dt = tk - a.t0;
      obs_s[k] = o;
    }
    __syncthreads();
    const double gam = gam_s[warp];
    const GradPlanetD *q = pl_s + warp * J;
    bool hi = false;                        // uniform: the warp holds one system
#pragma unroll
    for (int j = 0; j < J; ++j) hi = hi || q[j].base.e > (double)kEccFast;
    for (int kb = 0; kb < nk; kb += 32) {
      const int k = kb + lane;
      double urow[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) urow[i] = 0.0;
      if (k < nk) {
        const ObsGD o = obs_s[k];
        double sEj[J], cEj[J];
        double V = gam;
        with_high_e(hi, [&](auto tag) {
          constexpr bool HI = decltype(tag)::value;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const PlanetD p = q[j].base;
            const double M = mean_anomaly_f64(o.tau, p);
            kepler_f64<HI>(M, p.e, sEj[j], cEj[j]);
            V = velocity_add_f64(p, sEj[j], cEj[j], V);
          }
        });
        const double r = V - o.v;
        const double a2 = 2.0 * o.w * r;
        acc = fma(o.w * r, r, acc);
        const double sw = sqrt(o.w);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const GradPlanetD qj = q[j];
          Partials<double> d;
          const double invD = 1.0 / fma(-qj.base.e, cEj[j], 1.0);
          velocity_partials(qj.base.e, qj.K, qj.cw, qj.sw, qj.base.beta, qj.ibeta, sEj[j], cEj[j],
                            invD, d);
          d.dP = d.dM * (-kTwoPi * o.dt * qj.n2);
          g[5 * j + 0] = fma(a2, d.dP, g[5 * j + 0]);
          g[5 * j + 1] = fma(a2, d.dK, g[5 * j + 1]);
          g[5 * j + 2] = fma(a2, d.de, g[5 * j + 2]);
          g[5 * j + 3] = fma(a2, d.dw, g[5 * j + 3]);
          g[5 * j + 4] = fma(a2, d.dM, g[5 * j + 4]);
          urow[5 * j + 0] = sw * d.dP;
          urow[5 * j + 1] = sw * d.dK;
          urow[5 * j + 2] = sw * d.de;
          urow[5 * j + 3] = sw * d.dw;
          urow[5 * j + 4] = sw * d.dM;
        }
        g[5 * J] += a2;
        urow[5 * J] = sw;
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) u[lane * ROWD + i] = urow[i];
      __syncwarp();
      const int rows = min(32, nk - kb);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int e = lane + 32 * i;
        if (e < NTRI) {
          const short2 pq = pq_s[e];
          double sum = 0.0;
          for (int rr = 0; rr < rows; ++rr) sum = fma(u[rr * ROWD + pq.x], u[rr * ROWD + pq.y], sum);
          h[i] += sum;
        }
      }
      __syncwarp();
    }
  }

  for (int m = 16; m >= 1; m >>= 1) {
    acc += shfl_xor(acc, m);
#pragma unroll
    for (int i = 0; i < NP; ++i) g[i] += shfl_xor(g[i], m);
  }
  if (s >= a.n_sys) return;
  const double poison = 0.0 * gam_s[warp];
  if (lane == 0) {
    const double value = acc + poison;
    if (chi2_out) chi2_out[s] = value;
    note_invalid(a.invalid, value);
  }
  if (grad_out) {
#pragma unroll
    for (int i = 0; i < NP; ++i)
      if (lane == (i & 31)) grad_out[s * NP + i] = g[i] + poison;
  }
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int e = lane + 32 * i;
    if (e < NTRI) jtj_out[s * NTRI + e] = h[i] + poison;
  }
}

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t smem_grad(int n_pl, const Tile &t, bool f64) {
  const int ST = t.block / t.G;
  return f64 ? F64GradLayout(ST, n_pl, t.obs_tile).total
             : MixedGradLayout(ST, n_pl, t.obs_tile).total;
}

#define KC_DISPATCH_J(J, MACRO) \
  switch (J) {                  \
    case 1: MACRO(1); break;    \
    case 2: MACRO(2); break;    \
    case 3: MACRO(3); break;    \
    case 4: MACRO(4); break;    \
    case 5: MACRO(5); break;    \
    case 6: MACRO(6); break;    \
    case 7: MACRO(7); break;    \
    case 8: MACRO(8); break;    \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_grad_mixed(const UniformArgs &a, const Tile &tile, float *chi2, float *grad,
                              cudaStream_t st, bool nll) {
  if (tile.G > 32) return cudaErrorInvalidValue;
  const size_t smem = smem_grad(a.n_pl, tile, false);
  const int ST = tile.block / tile.G;
  const int grid = (int)((a.n_sys + ST - 1) / ST);
  cudaError_t err = cudaSuccess;
#define KC_LAUNCH_NLL(JJ, NN)                                                                   \
  err = set_smem(grad_mixed_kernel<JJ, NN>, smem);                                              \
  if (err == cudaSuccess)                                                                       \
    grad_mixed_kernel<JJ, NN><<<grid, tile.block, smem, st>>>(a, tile.G, tile.obs_tile, chi2,     \
                                                              grad);
#define KC_LAUNCH(JJ)                      \
  if (nll) {                               \
    KC_LAUNCH_NLL(JJ, true)                \
  } else {                                 \
    KC_LAUNCH_NLL(JJ, false)               \
  }
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
#undef KC_LAUNCH_NLL
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t launch_grad_f64(const UniformArgs &a, const Tile &tile, double *chi2, double *grad,
                            cudaStream_t st, bool nll) {
  if (tile.G > 32) return cudaErrorInvalidValue;
  const size_t smem = smem_grad(a.n_pl, tile, true);
  const int ST = tile.block / tile.G;
  const int grid = (int)((a.n_sys + ST - 1) / ST);
  cudaError_t err = cudaSuccess;
#define KC_LAUNCH_NLL(JJ, NN)                                                                 \
  err = set_smem(grad_f64_kernel<JJ, NN>, smem);                                              \
  if (err == cudaSuccess)                                                                     \
    grad_f64_kernel<JJ, NN><<<grid, tile.block, smem, st>>>(a, tile.G, tile.obs_tile, chi2,     \
                                                            grad);
#define KC_LAUNCH(JJ)                      \
  if (nll) {                               \
    KC_LAUNCH_NLL(JJ, true)                \
  } else {                                 \
    KC_LAUNCH_NLL(JJ, false)               \
  }
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
#undef KC_LAUNCH_NLL
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

// The tcgen05 variant (split 4): n_pl <= 3.  Every resident CTA holds
// kTcCols TMEM columns, so the launch is refused unless the SM's 512
// columns cover all CTAs that can be resident at once (an allocation would
// otherwise wait for another CTA to finish).
template <int J>
cudaError_t launch_gn_tc(const UniformArgs &a, void *chi2, void *grad, void *jtj,
                         cudaStream_t st) {
  const size_t smem = GnTcLayout(J).total;
  cudaError_t err = set_smem(gn_mixed_tc_kernel<J>, smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gn_mixed_tc_kernel<J>,
                                                      kGnWarps * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1 || per_sm * kTcCols > 512) return cudaErrorInvalidConfiguration;
  const int grid = (int)((a.n_sys + kGnWarps - 1) / kGnWarps);
  gn_mixed_tc_kernel<J><<<grid, kGnWarps * 32, smem, st>>>(a, (float *)chi2, (float *)grad,
                                                           (float *)jtj);
  return cudaGetLastError();
}

// Without a tuned entry the mixed Gauss-Newton kernel updates U^T U on
// tcgen05 where it can (n_pl <= 3): on a GB300, 65536 systems x 3 planets x
// 512 observations took 822 us against 869 us with mma.sync (whose
// registers do not leave room for two observations per lane: 958 us).
int gn_default_variant(int n_pl) { return n_pl <= 3 ? 4 : 0; }

bool gn_variant_ok(int variant, int n_pl) {
  return variant == 0 || (variant == 4 && n_pl >= 1 && n_pl <= 3);
}

cudaError_t launch_gauss_newton(const UniformArgs &a, bool f64, void *chi2, void *grad,
                                void *jtj, cudaStream_t st, int variant) {
  cudaError_t err = cudaSuccess;
  if (!f64 && variant != 0) {
    if (!gn_variant_ok(variant, a.n_pl)) return cudaErrorInvalidValue;
    switch (a.n_pl) {
      case 1: return launch_gn_tc<1>(a, chi2, grad, jtj, st);
      case 2: return launch_gn_tc<2>(a, chi2, grad, jtj, st);
      default: return launch_gn_tc<3>(a, chi2, grad, jtj, st);
    }
  }
  if (f64) {
    const int grid = (int)((a.n_sys + kGnWarpsD - 1) / kGnWarpsD);
#define KC_LAUNCH(JJ)                                                                        \
  {                                                                                          \
    const size_t smem = GnF64Layout(JJ, kGnObsTile).total;                                   \
    err = set_smem(gn_f64_kernel<JJ>, smem);                                                 \
    if (err == cudaSuccess)                                                                  \
      gn_f64_kernel<JJ><<<grid, kGnWarpsD * 32, smem, st>>>(a, (double *)chi2, (double *)grad, \
                                                            (double *)jtj);                  \
  }
    KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  } else {
    const int grid = (int)((a.n_sys + kGnWarps - 1) / kGnWarps);
#define KC_LAUNCH(JJ)                                                                        \
  {                                                                                          \
    const size_t smem = GnMixedLayout(JJ, kGnObsTile).total;                                 \
    err = set_smem(gn_mixed_kernel<JJ>, smem);                                               \
    if (err == cudaSuccess)                                                                  \
      gn_mixed_kernel<JJ><<<grid, kGnWarps * 32, smem, st>>>(a, (float *)chi2, (float *)grad, \
                                                             (float *)jtj);                  \
  }
    KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  }
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

}  // namespace kc
