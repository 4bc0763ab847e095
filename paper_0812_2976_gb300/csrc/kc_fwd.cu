// kc_fwd.cu -- fused chi-square kernels (mean anomaly -> Kepler -> velocity
// -> residual -> reduction in one pass), model prediction and the
// elementwise Kepler solver.
//
// The paper evaluates chi2 either with four kernels that write M, E and the
// planet velocities to device memory, or with M and E kernels followed by a
// fused velocity+chi2 kernel (Sec. 4.4, Table 1).  Here the whole chain runs
// in registers: only the parameters are read from HBM and one value per
// system is written back.
//
// Work layout: each system is handled by G consecutive threads of a CTA; the
// thread with index c in its group takes observations k = c, c+G, c+2G, ...
// The observations (shared by every system, Sec. 4.1) are staged once per
// CTA in shared memory (Sec. 5, "Device Memory Caching": cooperative load)
// and the per-planet constants are computed once per (system, planet) in
// FP64 and kept in shared memory.  Partial chi2 of the G threads are
// combined with warp shuffles (and shared memory when G > 32).
#include <algorithm>
#include <cmath>

#include "kc_demc.cuh"
#include "kc_device.cuh"
#include "kc_internal.h"

namespace kc {

namespace {

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct MixedLayout {
  size_t pl, gam, s2, red, obs, w, total;
  __host__ __device__ MixedLayout(int ST, int J, int nwarps, int obs_tile) {
    pl = 0;
    gam = pl + sizeof(PlanetF) * ST * J;
    s2 = gam + sizeof(float) * ST;
    red = align_up(s2 + sizeof(float) * ST, 16);
    obs = align_up(red + sizeof(float) * 3 * 32 * nwarps, 16);   // 3 per thread
    w = obs + sizeof(float4) * obs_tile;
    total = align_up(w + sizeof(float) * obs_tile, 16);
  }
};

struct ObsD {
  double tau, v, w, pad;
};

struct F64Layout {
  size_t tab, pl, gam, s2, red, obs, total;
  __host__ __device__ F64Layout(int ST, int J, int nwarps, int obs_tile) {
    tab = 0;                                          // sin/cos table, 4 KB
    pl = tab + sizeof(double2) * kSinTabN;
    gam = pl + sizeof(PlanetD) * ST * J;
    s2 = gam + sizeof(double) * ST;
    red = align_up(s2 + sizeof(double) * ST, 16);
    obs = align_up(red + sizeof(double) * 2 * nwarps, 16);
    total = align_up(obs + sizeof(ObsD) * obs_tile, 16);
  }
};

// gamma of system s, or NaN when any parameter of the system is invalid.
__device__ inline double system_gamma(const double *p, int J) {
  bool ok = finite_bits(p[5 * J]);
  for (int j = 0; j < J; ++j)
    ok = ok && planet_valid(p[5 * j], p[5 * j + 1], p[5 * j + 2], p[5 * j + 3], p[5 * j + 4]);
  return ok ? p[5 * J] : __longlong_as_double(0x7ff8000000000000ll);
}

// Free jitter (the likelihood variant): sigma_j^2 of a system whose
// parameters end with (gamma, sigma_j); NaN if sigma_j is not finite.
__device__ inline double system_jitter2(const double *p, int J) {
  const double sj = p[5 * J + 1];
  return isfinite(sj) ? sj * sj : __longlong_as_double(0x7ff8000000000000ll);
}

// The same as a float for the mixed path (no FP64 instruction).
__device__ inline float system_jitter2_f(const double *p, int J) {
  const float sj = d2f(p[5 * J + 1]);
  return finite_bits(p[5 * J + 1]) ? sj * sj : __int_as_float(0x7fc00000);
}

constexpr float kLn2F = 0.693147180559945309f;
constexpr double kLn2Pi = 1.8378770664093454836;      // ln(2 pi)

// Inverse variance 1/(sigma_k^2 + sigma_jit^2) (Eq. 5); NaN if not positive.
__device__ inline double inv_variance(double sigma, double jitter2) {
  const double var = fma(sigma, sigma, jitter2);
  return (var > 0.0) ? 1.0 / var : __longlong_as_double(0x7ff8000000000000ll);
}

// ------------------------------------------------------------ mixed

// Thread that handles setup item i: items are dealt round-robin over the
// warps so that the double-precision setup runs on every SM sub-partition.
__device__ inline int setup_slot(int tid, int nwarps) { return (tid & 31) * nwarps + (tid >> 5); }

// Prepared inputs of the split variant: per-(system, planet) constants,
// per-system gamma (NaN if invalid) and converted observations, written by
// prep_mixed_kernel into stream-ordered scratch.
struct MixedPrep {
  const PlanetF *pl;     // [n_sys * n_pl]
  const float *gam;      // [n_sys]
  const float4 *obs;     // [n_obs] (tau_hi, tau_lo, v_hi, v_lo)
  const float *w;        // [n_obs]
};

// PRE = false: each CTA computes its planets' constants (FP64) and converts
// the observations itself.  PRE = true (split variant): both come from
// prep_mixed_kernel, launched just before with programmatic dependent
// launch; the CTA waits for it, then only copies.
// NLL = true (with PRE = false): every system carries its own jitter after
// gamma and the kernel returns the negative log-likelihood
//   1/2 sum_k [r_k^2/(sigma_k^2 + sigma_j^2) + ln(2 pi (sigma_k^2 + sigma_j^2))].
// SINGLE = true (with PRE = false): the pure single-precision variant of
// Sec. 5 (precision comparisons only): times, epoch and periods rounded to
// float and the phase formed in float.
// DEMC = true: the launch carries a DE-MC step (a.demc): proposals formed in
// the prologue when a.demc.z is set, the Metropolis decision in the
// epilogue.  Plain evaluations use DEMC = false and contain neither.
// At most 104 registers up to four planets, 128 above (blocks of at most
// 256 threads): left alone the compiler keeps Mikkola's per-planet constants
// of all J planets live across the observation loop (124 registers at
// J = 4, four CTAs of 128 per SM); capped, it recomputes part of them and
// the kernel runs 2 % faster on both the paper batch and the 2^20-system
// sweep.
template <int J, bool PRE, bool NLL = false, bool SINGLE = false, bool DEMC = false>
__global__ void __maxnreg__(J <= 4 ? 104 : 128)
chi2_mixed_kernel(UniformArgs a, MixedPrep prep, int G, int obs_tile, float *__restrict__ out,
                  float *__restrict__ resid_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int block = blockDim.x;
  const int nwarps = block >> 5;
  const int ST = block / G;
  const MixedLayout L(ST, J, nwarps, obs_tile);
  PlanetF *pl_s = reinterpret_cast<PlanetF *>(smem + L.pl);
  float *gam_s = reinterpret_cast<float *>(smem + L.gam);
  float *s2_s = reinterpret_cast<float *>(smem + L.s2);
  float *red_s = reinterpret_cast<float *>(smem + L.red);
  float4 *obs_s = reinterpret_cast<float4 *>(smem + L.obs);
  float *w_s = reinterpret_cast<float *>(smem + L.w);

  const int tid = threadIdx.x;
  const int64_t sys0 = (int64_t)blockIdx.x * ST;
  const int npar = 5 * J + 1 + (NLL ? 1 : 0);
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const float jit2 = d2f(a.jitter2);
  const Split3 tr3 = split3(t_ref);
  const int nk0 = min(obs_tile, a.n_obs);

  // tau = t - t_ref and v as float pairs, w = 1/(sigma^2 + jit^2) (NLL keeps
  // sigma_k^2: its weight depends on each system's own jitter)
  auto stage = [&](int slot, double t, double v, double sigma) {
    float th, tl, vh, vl;
    if (SINGLE) {
      th = __fsub_rn(d2f(t), d2f(a.t0));
      tl = 0.0f;
    } else {
      sub_ds(split3(t), tr3, th, tl);
    }
    split_d(v, vh, vl);
    obs_s[slot] = make_float4(th, tl, vh, vl);
    const float sg = d2f(sigma);
    const float var = __fmaf_rn(sg, sg, jit2);
    w_s[slot] = NLL ? sg * sg : (var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000));
  };

  if (PRE) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int i = tid; i < ST * J; i += block) {
      const int64_t s = sys0 + i / J;
      PlanetF q = {0, 0, 0, 0, 0, 0, 0, 0};
      if (s < a.n_sys) q = prep.pl[sys0 * J + i];
      pl_s[i] = q;
    }
    for (int i = tid; i < ST; i += block) {
      const int64_t s = sys0 + i;
      gam_s[i] = s < a.n_sys ? prep.gam[s] : 0.0f;
    }
    for (int k = tid; k < nk0; k += block) {
      obs_s[k] = prep.obs[k];
      w_s[k] = prep.w[k];
    }
  } else {
    // Prologue, all latency: the loads of the first observation tile go out
    // before the planet setup so that the two overlap.
    const bool has0 = tid < nk0, has1 = tid + block < nk0;
    double t0v = 0.0, v0v = 0.0, s0v = 0.0, t1v = 0.0, v1v = 0.0, s1v = 0.0;
    if (has0) { t0v = a.t[tid]; v0v = a.v[tid]; s0v = a.sigma[tid]; }
    if (has1) { t1v = a.t[tid + block]; v1v = a.v[tid + block]; s1v = a.sigma[tid + block]; }
    // per-(system, planet) constants, once (Eqs. 4/6 phase offset); an
    // invalid planet carries e = NaN, which poisons its system's chi2
    for (int i = tid; i < ST * J; i += block) {
      const int sl = i / J, j = i - sl * J;
      const int64_t s = sys0 + sl;
      PlanetF q = {0, 0, 0, 0, 0, 0, 0, 0};
      if (s < a.n_sys) {
        double p[5];
        if (DEMC && a.demc.z) {
          demc_form(a, s, 5 * j, npar, p);        // DE-MC: this planet's proposal
        } else if (dbg_ok(a.invalid, s * npar + 5 * j + 4 < a.n_sys * npar, kDbgParam,
                          s * npar + 5 * j)) {
#pragma unroll
          for (int k = 0; k < 5; ++k) p[k] = a.params[s * npar + 5 * j + k];
        } else {
#pragma unroll
          for (int k = 0; k < 5; ++k) p[k] = 0.0;
        }
        q = planet_setup_mixed(p, t_ref, a.t0);
        if (SINGLE) {     // 1/P and M0/(2 pi) in float, the phase taken from t - t0
          q.n_hi = 1.0f / d2f(p[0]);
          q.n_lo2pi = 0.0f;
          q.c_hi = d2f(p[4]) * (1.0f / kTwoPiF);
          q.c_lo2pi = 0.0f;
        }
        if (!planet_valid(p[0], p[1], p[2], p[3], p[4])) q.e = __int_as_float(0x7fc00000);
      }
      pl_s[i] = q;
    }
    for (int i = tid; i < ST; i += block) {
      const int64_t s = sys0 + i;
      float g = 0.0f;
      if (s < a.n_sys) {
        double gd[1];
        if (DEMC && a.demc.z)
          demc_form(a, s, 5 * J, npar, gd);
        else
          gd[0] = a.params[s * npar + 5 * J];
        g = finite_bits(gd[0]) ? d2f(gd[0]) : __int_as_float(0x7fc00000);
      }
      gam_s[i] = g;
      if (NLL) s2_s[i] = s < a.n_sys ? system_jitter2_f(a.params + s * npar, J) : 0.0f;
    }
    if (has0) stage(tid, t0v, v0v, s0v);
    if (has1) stage(tid + block, t1v, v1v, s1v);
    for (int k = tid + 2 * block; k < nk0; k += block) stage(k, a.t[k], a.v[k], a.sigma[k]);
  }
  __syncthreads();

  const int sl = tid / G, c = tid - sl * G;
  const int64_t s = sys0 + sl;
  const bool want_resid = resid_out != nullptr;
  Kahan acc = {0.0f, 0.0f};
  float rmax = 0.0f;
  const float gam = gam_s[sl];
  const float s2 = NLL ? s2_s[sl] : 0.0f;
  PlanetF q[J];
  float poison = 0.0f * gam + (NLL ? 0.0f * s2 : 0.0f);   // NaN for an invalid system
#pragma unroll
  for (int j = 0; j < J; ++j) {
    q[j] = pl_s[sl * J + j];
    poison += 0.0f * q[j].e;
  }

  for (int k0 = 0; k0 < a.n_obs; k0 += obs_tile) {
    const int nk = min(obs_tile, a.n_obs - k0);
    if (k0 > 0) {
      __syncthreads();
      for (int k = tid; k < nk; k += block) {
        if (!dbg_ok(a.invalid, k0 + k < a.n_obs && k < obs_tile, kDbgObs, k0 + k)) continue;
        if (PRE) {
          obs_s[k] = prep.obs[k0 + k];
          w_s[k] = prep.w[k0 + k];
        } else {
          stage(k, a.t[k0 + k], a.v[k0 + k], a.sigma[k0 + k]);
        }
      }
      __syncthreads();
    }
    for (int k = c; k < nk; k += G) {
      const float4 o = obs_s[k];
      Kahan V = {0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const float M =
            SINGLE ? mean_anomaly_single(o.x, q[j]) : mean_anomaly_mixed(o.x, o.y, q[j]);
        float sE, cE;
        const float E = kepler_f32(M, q[j].e, sE, cE);
        if (want_resid) rmax = fmaxf(rmax, fabsf((E - M) - q[j].e * sE));
        kahan_add(V, velocity_mixed(q[j], sE, cE));
      }
      // residual V - v_obs with the model and the observation as float pairs
      const float r = __fadd_rn(__fsub_rn(V.big, o.z), __fsub_rn(gam, __fadd_rn(V.small, o.w)));
      if (NLL) {
        const float var = w_s[k] + s2;              // sigma_k^2 + sigma_j^2
        const float wk = var > 0.0f ? rcp_fast(var) : __int_as_float(0x7fc00000);
        kahan_add(acc, __fmaf_rn(wk * r, r, lg2_fast(var) * kLn2F));
      } else {
        kahan_add(acc, w_s[k] * r * r);
      }
    }
  }

  // combine the G partial sums of each system
  if (G & (G - 1)) {
    // G not a power of two (a system's threads may straddle two warps): the
    // first thread of each system merges the others' sums in thread order
    __syncthreads();
    red_s[3 * tid] = acc.big;
    red_s[3 * tid + 1] = acc.small;
    red_s[3 * tid + 2] = rmax;
    __syncthreads();
    if (c == 0) {
      for (int i = tid + 1; i < tid + G; ++i) {
        Kahan o = {red_s[3 * i], red_s[3 * i + 1]};
        kahan_merge(acc, o);
        rmax = fmaxf(rmax, red_s[3 * i + 2]);
      }
    }
  }
  const int gw = (G & (G - 1)) ? 1 : (G < 32 ? G : 32);
  for (int m = gw >> 1; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
    rmax = fmaxf(rmax, shfl_xor(rmax, m));
  }
  if (G > 32 && !(G & (G - 1))) {
    const int warp = tid >> 5, lane = tid & 31;
    __syncthreads();
    if (lane == 0) {
      red_s[3 * warp] = acc.big;
      red_s[3 * warp + 1] = acc.small;
      red_s[3 * warp + 2] = rmax;
    }
    __syncthreads();
    if (c == 0) {
      for (int w = warp + 1; w < warp + G / 32; ++w) {
        Kahan o = {red_s[3 * w], red_s[3 * w + 1]};
        kahan_merge(acc, o);
        rmax = fmaxf(rmax, red_s[3 * w + 2]);
      }
    }
  }
  if (c == 0 && s < a.n_sys) {
    // the poison turns an invalid system into NaN even when n_obs == 0
    const float value = NLL ? 0.5f * (kahan_value(acc) + (float)a.n_obs * (float)kLn2Pi) + poison
                            : kahan_value(acc) + poison;
    out[s] = value;
    note_invalid(a.invalid, value);
    if (resid_out) resid_out[s] = rmax;
    if (DEMC) demc_accept<5 * J + 1 + (NLL ? 1 : 0)>(a, s, value);
  }
}

// Split variant, first pass: every per-(system, planet) setup, gamma and
// observation conversion of the batch, spread over the whole grid (once per
// batch instead of once per CTA).
__global__ void __launch_bounds__(64)
prep_mixed_kernel(UniformArgs a, PlanetF *__restrict__ pl, float *__restrict__ gam,
                  float4 *__restrict__ obs, float *__restrict__ w,
                  unsigned *__restrict__ counters) {
  // let the dependent main kernel be scheduled as this grid drains; its
  // griddepcontrol.wait still waits for this grid's completion
  asm volatile("griddepcontrol.launch_dependents;");
  const int J = a.n_pl, npar = 5 * J + 1;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const float jit2 = d2f(a.jitter2);
  for (int64_t i = tid; i < a.n_sys * J; i += nth) {
    const int64_t s = i / J;
    pl[i] = planet_setup_mixed(a.params + s * npar + 5 * (i - s * J), t_ref, a.t0);
  }
  const Split3 tr3 = split3(t_ref);
  for (int64_t s = tid; s < a.n_sys; s += nth) {
    gam[s] = d2f(system_gamma(a.params + s * npar, J));
    if (counters) counters[s] = 0u;
  }
  for (int64_t k = tid; k < a.n_obs; k += nth) {
    float th, tl, vh, vl;
    sub_ds(split3(a.t[k]), tr3, th, tl);
    split_d(a.v[k], vh, vl);
    obs[k] = make_float4(th, tl, vh, vl);
    const float sg = d2f(a.sigma[k]);
    const float var = __fmaf_rn(sg, sg, jit2);
    w[k] = var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000);
  }
}

// Split variant 2: one warp per (system, chunk of observations).  A system's
// G threads form G/32 warps, each taking a contiguous chunk of the
// observations, so the batch becomes many small independent units (no CTA
// barrier, no per-CTA staging) and the grid's tail is short.  Each warp
// writes its partial chi2 (a Kahan pair) and max residual; the last warp of
// a system to finish (per-system counter, zeroed by the preparation pass)
// merges the partials in chunk order, so the result does not depend on the
// order in which warps finish.
struct ChunkScratch {
  float2 *part;          // [n_sys * chunks] (big, small)
  float *part_resid;     // [n_sys * chunks]
  unsigned *count;       // [n_sys]
};

template <int J>
__global__ void __launch_bounds__(256)
chi2_mixed_chunk_kernel(UniformArgs a, MixedPrep prep, ChunkScratch cs, int chunks,
                        float *__restrict__ out, float *__restrict__ resid_out) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int64_t unit = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (unit >= a.n_sys * chunks) return;               // whole warps only
  const int64_t s = unit / chunks;
  const int c = (int)(unit - s * chunks);
  const int len = (a.n_obs + chunks - 1) / chunks;
  const int k0 = c * len, k1 = min(a.n_obs, k0 + len);
  PlanetF q[J];
#pragma unroll
  for (int j = 0; j < J; ++j) q[j] = prep.pl[s * J + j];
  const float gam = prep.gam[s];
  const bool want_resid = resid_out != nullptr;
  Kahan acc = {0.0f, 0.0f};
  float rmax = 0.0f;
  for (int k = k0 + lane; k < k1; k += 32) {
    const float4 o = prep.obs[k];
    const float wk = prep.w[k];
    Kahan V = {0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const float M = mean_anomaly_mixed(o.x, o.y, q[j]);
      float sE, cE;
      const float E = kepler_f32(M, q[j].e, sE, cE);
      if (want_resid) rmax = fmaxf(rmax, fabsf((E - M) - q[j].e * sE));
      kahan_add(V, velocity_mixed(q[j], sE, cE));
    }
    const float r = __fadd_rn(__fsub_rn(V.big, o.z), __fsub_rn(gam, __fadd_rn(V.small, o.w)));
    kahan_add(acc, wk * r * r);
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
    rmax = fmaxf(rmax, shfl_xor(rmax, m));
  }
  unsigned done = 0;
  if (lane == 0) {
    cs.part[unit] = make_float2(acc.big, acc.small);
    cs.part_resid[unit] = rmax;
    __threadfence();                                    // partial visible before the count
    done = atomicAdd(cs.count + s, 1u);
  }
  done = __shfl_sync(0xffffffffu, done, 0);
  if (done != (unsigned)(chunks - 1)) return;           // not the last chunk of s
  __threadfence();
  // merge the chunks' partials in chunk order (lane c holds chunk c)
  Kahan m = {0.0f, 0.0f};
  float rm = 0.0f;
  if (lane < chunks) {
    const float2 p = __ldcg(cs.part + s * chunks + lane);
    m.big = p.x;
    m.small = p.y;
    rm = __ldcg(cs.part_resid + s * chunks + lane);
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Kahan o = {__shfl_down_sync(0xffffffffu, m.big, d), __shfl_down_sync(0xffffffffu, m.small, d)};
    const float ro = __shfl_down_sync(0xffffffffu, rm, d);
    if ((lane & (2 * d - 1)) == 0 && lane + d < 32) {
      kahan_merge(m, o);
      rm = fmaxf(rm, ro);
    }
  }
  if (lane == 0) {
    out[s] = kahan_value(m) + 0.0f * gam;
    note_invalid(a.invalid, out[s]);
    if (resid_out) resid_out[s] = rm;
  }
}

// ------------------------------------------------------------ FP64

template <int J, bool NLL = false, bool DEMC = false>
__global__ void __launch_bounds__(256, 2)
chi2_f64_kernel(UniformArgs a, int G, int obs_tile, double *__restrict__ out,
                float *__restrict__ resid_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int block = blockDim.x;
  const int ST = block / G;
  const F64Layout L(ST, J, block / 32, obs_tile);
  double2 *tab_s = reinterpret_cast<double2 *>(smem + L.tab);
  PlanetD *pl_s = reinterpret_cast<PlanetD *>(smem + L.pl);
  double *gam_s = reinterpret_cast<double *>(smem + L.gam);
  double *s2_s = reinterpret_cast<double *>(smem + L.s2);
  double *red_s = reinterpret_cast<double *>(smem + L.red);
  ObsD *obs_s = reinterpret_cast<ObsD *>(smem + L.obs);

  const int tid = threadIdx.x;
  const int64_t sys0 = (int64_t)blockIdx.x * ST;
  const int npar = 5 * J + 1 + (NLL ? 1 : 0);
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  const double dref = t_ref - a.t0;
  const bool want_resid = resid_out != nullptr;
  sincos_table_build(tab_s, tid, block);      // read after the tile loop's first barrier

  for (int i = setup_slot(tid, block >> 5); i < ST * J; i += block) {
    const int sl = i / J, j = i - sl * J;
    const int64_t s = sys0 + sl;
    PlanetD q = {};
    if (s < a.n_sys && dbg_ok(a.invalid, s * npar + 5 * j + 4 < a.n_sys * npar, kDbgParam,
                              s * npar + 5 * j))
      q = planet_setup_f64(a.params + s * npar + 5 * j, dref);
    pl_s[i] = q;
  }
  for (int i = tid; i < ST; i += block) {
    const int64_t s = sys0 + i;
    gam_s[i] = s < a.n_sys ? system_gamma(a.params + s * npar, J) : 0.0;
    if (NLL) s2_s[i] = s < a.n_sys ? system_jitter2(a.params + s * npar, J) : 0.0;
  }

  const int sl = tid / G, c = tid - sl * G;
  const int64_t s = sys0 + sl;
  double acc = 0.0, rmax = 0.0;

  for (int k0 = 0; k0 < a.n_obs; k0 += obs_tile) {
    const int nk = min(obs_tile, a.n_obs - k0);
    __syncthreads();
    for (int k = tid; k < nk; k += block) {
      if (!dbg_ok(a.invalid, k0 + k < a.n_obs && k < obs_tile, kDbgObs, k0 + k)) continue;
      ObsD o;
      o.tau = a.t[k0 + k] - t_ref;
      o.v = a.v[k0 + k];
      o.w = NLL ? a.sigma[k0 + k] * a.sigma[k0 + k] : inv_variance(a.sigma[k0 + k], a.jitter2);
      o.pad = 0.0;
      obs_s[k] = o;
    }
    __syncthreads();
    const double gam = gam_s[sl];
    const PlanetD *q = pl_s + sl * J;
    bool hi = false;
#pragma unroll
    for (int j = 0; j < J; ++j) hi = hi || q[j].e > (double)kEccFast;
    with_high_e(any_high_e(hi), [&](auto tag) {
      constexpr bool HI = decltype(tag)::value;
      for (int k = c; k < nk; k += G) {
        const ObsD o = obs_s[k];
        double V = gam;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const PlanetD p = q[j];
          const double M = mean_anomaly_f64(o.tau, p);
          double sE, cE;
          const double E = kepler_f64<HI>(M, p.e, sE, cE, tab_s);
          if (want_resid) rmax = fmax(rmax, fabs((E - M) - p.e * sE));
          V = velocity_add_f64(p, sE, cE, V);
        }
        const double r = V - o.v;
        if (NLL) {
          const double var = o.w + s2_s[sl];
          const double wk = var > 0.0 ? 1.0 / var : __longlong_as_double(0x7ff8000000000000ll);
          acc += fma(wk * r, r, log(var));
        } else {
          acc = fma(o.w * r, r, acc);
        }
      }
    });
  }

  const int gw = G < 32 ? G : 32;
  for (int m = gw >> 1; m >= 1; m >>= 1) {
    acc += shfl_xor(acc, m);
    rmax = fmax(rmax, shfl_xor(rmax, m));
  }
  if (G > 32) {
    const int warp = tid >> 5, lane = tid & 31;
    __syncthreads();
    if (lane == 0) {
      red_s[2 * warp] = acc;
      red_s[2 * warp + 1] = rmax;
    }
    __syncthreads();
    if (c == 0) {
      for (int w = warp + 1; w < warp + G / 32; ++w) {
        acc += red_s[2 * w];
        rmax = fmax(rmax, red_s[2 * w + 1]);
      }
    }
  }
  if (c == 0 && s < a.n_sys) {
    const double poison = 0.0 * gam_s[sl] + (NLL ? 0.0 * s2_s[sl] : 0.0);
    const double value = NLL ? 0.5 * (acc + a.n_obs * kLn2Pi) + poison : acc + poison;
    out[s] = value;
    note_invalid(a.invalid, value);
    if (resid_out) resid_out[s] = (float)rmax;
    if (DEMC) demc_accept<5 * J + 1 + (NLL ? 1 : 0)>(a, s, value);
  }
}

// ------------------------------------------------------------ prediction

// V(t_k) = gamma + sum_j v_j(t_k) in FP64, one thread per (system, obs).
__global__ void rv_predict_kernel(const double *__restrict__ params, const double *__restrict__ t,
                                  int64_t n_sys, int J, int n_obs, double t0,
                                  double *__restrict__ v_out) {
  const int64_t total = n_sys * (int64_t)n_obs;
  const int npar = 5 * J + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / n_obs;
    const int k = (int)(i - s * n_obs);
    const double *p = params + s * npar;
    const double t_ref = t[0];
    double V = system_gamma(p, J);
    for (int j = 0; j < J; ++j) {
      const PlanetD q = planet_setup_f64(p + 5 * j, t_ref - t0);
      const double M = mean_anomaly_f64(t[k] - t_ref, q);
      double sE, cE;
      kepler_f64(M, q.e, sE, cE);
      V = velocity_add_f64(q, sE, cE, V);
    }
    v_out[i] = V;
  }
}

// ------------------------------------------------------------ Kepler only

template <typename T>
__device__ inline T reduce_pi(T M);
template <>
__device__ inline double reduce_pi<double>(double M) {
  return M - kTwoPi * rint(M * kInvTwoPi);
}
template <>
__device__ inline float reduce_pi<float>(float M) {
  // Cody-Waite with 2 pi split into two floats (|M| < 2^22 on the fast path)
  if (fabsf(M) <= 3.14159265f) return M;
  if (!(fabsf(M) < 4194304.0f)) {                      // rare: reduce in double
    const double m = (double)M;
    return (float)(m - kTwoPi * rint(m * kInvTwoPi));
  }
  const float q = round_small(M * 0.159154943091895336f);
  return __fmaf_rn(-q, -1.74845553e-7f, __fmaf_rn(-q, 6.28318548202514648f, M));
}

// One (M, e) per thread; the lanes of a warp vote for the high-eccentricity
// variant (the lanes still in the grid-stride loop).
__global__ void kepler_f64_kernel(const double *__restrict__ M, const double *__restrict__ e,
                                  int64_t n, double *__restrict__ E) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    const double ei = e[i], Mi = reduce_pi(M[i]);
    if (any_high_e(ei > (double)kEccFast, __activemask()))
      E[i] = kepler_f64<true>(Mi, ei, s, c);
    else
      E[i] = kepler_f64<false>(Mi, ei, s, c);
  }
}

// Four (M, e) per thread and iteration when the three arrays are 16-byte
// aligned: float4 streaming loads and stores (the data are touched once) and
// four independent solves in flight per thread, which keeps more loads
// outstanding than one element per thread does.  The rest (or everything,
// unaligned) one element per thread.
__device__ __forceinline__ float4 kepler_f32_x4(float4 m, float4 ee) {
  float s, c;
  float4 r;
  r.x = kepler_f32(reduce_pi(m.x), ee.x, s, c);
  r.y = kepler_f32(reduce_pi(m.y), ee.y, s, c);
  r.z = kepler_f32(reduce_pi(m.z), ee.z, s, c);
  r.w = kepler_f32(reduce_pi(m.w), ee.w, s, c);
  return r;
}

__global__ void kepler_f32_kernel(const float *__restrict__ M, const float *__restrict__ e,
                                  int64_t n, float *__restrict__ E) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool aligned = ((reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(e) |
                         reinterpret_cast<uintptr_t>(E)) & 15u) == 0;
  const int64_t n4 = aligned ? n / 4 : 0;
  const float4 *M4 = reinterpret_cast<const float4 *>(M);
  const float4 *e4 = reinterpret_cast<const float4 *>(e);
  float4 *E4 = reinterpret_cast<float4 *>(E);
  for (int64_t i = tid; i < n4; i += stride) {
    __stcs(E4 + i, kepler_f32_x4(__ldcs(M4 + i), __ldcs(e4 + i)));
  }
  for (int64_t i = 4 * n4 + tid; i < n; i += stride) {
    float s, c;
    E[i] = kepler_f32(reduce_pi(M[i]), e[i], s, c);
  }
}

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int grid_for(int64_t n_sys, int ST) { return (int)((n_sys + ST - 1) / ST); }

int elementwise_grid(int64_t n) {
  const int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 32;
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

size_t smem_chi2_mixed(int n_pl, const Tile &t) {
  return MixedLayout(t.block / t.G, n_pl, t.block / 32, t.obs_tile).total;
}

size_t smem_chi2_f64(int n_pl, const Tile &t) {
  return F64Layout(t.block / t.G, n_pl, t.block / 32, t.obs_tile).total;
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

size_t mixed_prep_bytes(int64_t n_sys, int n_pl, int n_obs) {
  return align_up(sizeof(PlanetF) * n_sys * n_pl, 256) + align_up(sizeof(float) * n_sys, 256) +
         align_up(sizeof(float4) * n_obs, 256) + align_up(sizeof(float) * n_obs, 256);
}

size_t mixed_chunk_bytes(int64_t n_sys, int chunks) {
  return align_up(sizeof(float2) * n_sys * chunks, 256) +
         align_up(sizeof(float) * n_sys * chunks, 256) + align_up(sizeof(unsigned) * n_sys, 256);
}

size_t mixed_scratch_bytes(int64_t n_sys, int n_pl, int n_obs, const Tile &tile) {
  size_t b = mixed_prep_bytes(n_sys, n_pl, n_obs);
  if (tile.split == 2) b += mixed_chunk_bytes(n_sys, tile.G / 32);
  return b;
}

cudaError_t launch_chi2_mixed_prepared(const UniformArgs &a, const Tile &tile, void *scratch,
                                       float *out, float *resid, cudaStream_t st) {
  unsigned char *base = static_cast<unsigned char *>(scratch);
  PlanetF *pl = reinterpret_cast<PlanetF *>(base);
  base += align_up(sizeof(PlanetF) * a.n_sys * a.n_pl, 256);
  float *gam = reinterpret_cast<float *>(base);
  base += align_up(sizeof(float) * a.n_sys, 256);
  float4 *obs = reinterpret_cast<float4 *>(base);
  base += align_up(sizeof(float4) * a.n_obs, 256);
  float *w = reinterpret_cast<float *>(base);
  base += align_up(sizeof(float) * a.n_obs, 256);
  const int chunks = tile.split == 2 ? tile.G / 32 : 0;
  ChunkScratch cs{nullptr, nullptr, nullptr};
  if (chunks > 0) {
    cs.part = reinterpret_cast<float2 *>(base);
    base += align_up(sizeof(float2) * a.n_sys * chunks, 256);
    cs.part_resid = reinterpret_cast<float *>(base);
    base += align_up(sizeof(float) * a.n_sys * chunks, 256);
    cs.count = reinterpret_cast<unsigned *>(base);
  }
  // Each setup item is a long dependent chain (float expansions, ~2k cycles),
  // so the items are spread thinly over every SM (64-thread CTAs, one item
  // per thread) rather than packed into a few full CTAs.
  const int64_t items = std::max<int64_t>(a.n_sys * a.n_pl, std::max<int64_t>(a.n_obs, 1));
  const int prep_grid = (int)std::min<int64_t>((items + 63) / 64, (int64_t)sm_count() * 16);
  prep_mixed_kernel<<<prep_grid, 64, 0, st>>>(a, pl, gam, obs, w, cs.count);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  MixedPrep prep{pl, gam, obs, w};
  const size_t smem = chunks > 0 ? 0 : smem_chi2_mixed(a.n_pl, tile);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_for(a.n_sys, tile.block / tile.G));
  cfg.blockDim = dim3(tile.block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (chunks > 0) {
    const int64_t threads = a.n_sys * chunks * 32;
    cfg.gridDim = dim3((unsigned)((threads + tile.block - 1) / tile.block));
#define KC_LAUNCH(JJ) \
  err = cudaLaunchKernelEx(&cfg, chi2_mixed_chunk_kernel<JJ>, a, prep, cs, chunks, out, resid);
    KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
  }
#define KC_LAUNCH(JJ)                                                                         \
  if (a.demc.states) {                                                                        \
    err = set_smem(chi2_mixed_kernel<JJ, true, false, false, true>, smem);                    \
    if (err == cudaSuccess)                                                                   \
      err = cudaLaunchKernelEx(&cfg, chi2_mixed_kernel<JJ, true, false, false, true>, a, prep, \
                               tile.G, tile.obs_tile, out, resid);                            \
  } else {                                                                                    \
    err = set_smem(chi2_mixed_kernel<JJ, true>, smem);                                        \
    if (err == cudaSuccess)                                                                   \
      err = cudaLaunchKernelEx(&cfg, chi2_mixed_kernel<JJ, true>, a, prep, tile.G,            \
                               tile.obs_tile, out, resid);                                    \
  }
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

// DE-MC proposals still to be formed (a.demc.z != NULL), for launch paths
// whose kernels do not form them: the proposal kernel runs first and a
// marks them as formed.
static cudaError_t form_proposals(UniformArgs &a, cudaStream_t st) {
  if (!a.demc.states || !a.demc.z) return cudaSuccess;
  const DemcAccept &d = a.demc;
  cudaError_t err = launch_demcmc_propose(d.states, 5 * a.n_pl + 1, d.first, a.n_sys,
                                          d.partner_first, d.partner_count, d.gamma,
                                          d.eps_scale, d.z, d.u,
                                          const_cast<double *>(a.params), st);
  a.demc.z = nullptr;
  return err;
}

cudaError_t launch_chi2_mixed(const UniformArgs &a_in, const Tile &tile_in, float *out,
                              float *resid, cudaStream_t st) {
  UniformArgs a = a_in;
  Tile tile = tile_in;
  if (tile.split == 3) return launch_chi2_mixed_warp(a, tile, out, resid, st);
  if (tile.split) {
    // No stream-ordered allocation inside a graph being captured: the fused
    // kernel (no scratch) stands in for the split variants there.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(st, &cs);
    if (err != cudaSuccess) return err;
    if (cs != cudaStreamCaptureStatusNone) {
      if (tile.G > tile.block) tile = default_tile(Kind::Chi2Mixed, a.n_sys, a.n_pl, a.n_obs);
      tile.split = 0;
    }
  }
  if (tile.split) {
    cudaError_t err = form_proposals(a, st);
    if (err != cudaSuccess) return err;
    // stream-ordered scratch from the library's pool (kept cached between calls)
    void *scratch = nullptr;
    err = scratch_alloc(&scratch, mixed_scratch_bytes(a.n_sys, a.n_pl, a.n_obs, tile), st);
    if (err != cudaSuccess) return err;
    err = launch_chi2_mixed_prepared(a, tile, scratch, out, resid, st);
    // the chunked two-pass variant has no per-system epilogue: a DE-MC
    // Metropolis step runs as its own kernel after it
    if (err == cudaSuccess && tile.split == 2 && a.demc.states)
      err = launch_demcmc_accept(a.demc.states, a.demc.chi2, a.params, out, a.demc.first,
                                 a.n_sys, 5 * a.n_pl + 1, a.demc.u, false, a.demc.accepted, st);
    cudaError_t err2 = cudaFreeAsync(scratch, st);
    return err != cudaSuccess ? err : err2;
  }
  const size_t smem = smem_chi2_mixed(a.n_pl, tile);
  const int grid = grid_for(a.n_sys, tile.block / tile.G);
  const MixedPrep none{nullptr, nullptr, nullptr, nullptr};
  cudaError_t err = cudaSuccess;
#define KC_LAUNCH(JJ)                                                                       \
  if (a.demc.states) {                                                                      \
    err = set_smem(chi2_mixed_kernel<JJ, false, false, false, true>, smem);                 \
    if (err == cudaSuccess)                                                                 \
      chi2_mixed_kernel<JJ, false, false, false, true><<<grid, tile.block, smem, st>>>(      \
          a, none, tile.G, tile.obs_tile, out, resid);                                      \
  } else {                                                                                  \
    err = set_smem(chi2_mixed_kernel<JJ, false>, smem);                                     \
    if (err == cudaSuccess)                                                                 \
      chi2_mixed_kernel<JJ, false><<<grid, tile.block, smem, st>>>(a, none, tile.G,           \
                                                                   tile.obs_tile, out, resid); \
  }
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t launch_chi2_f64(const UniformArgs &a_in, const Tile &tile, double *out,
                            float *resid, cudaStream_t st) {
  // the FP64 kernel checks gamma against the whole parameter row, so its
  // proposals are formed before it
  UniformArgs a = a_in;
  cudaError_t err = form_proposals(a, st);
  if (err != cudaSuccess) return err;
  const size_t smem = smem_chi2_f64(a.n_pl, tile);
  const int grid = grid_for(a.n_sys, tile.block / tile.G);
#define KC_LAUNCH(JJ)                                                                      \
  if (a.demc.states) {                                                                     \
    err = set_smem(chi2_f64_kernel<JJ, false, true>, smem);                                \
    if (err == cudaSuccess)                                                                \
      chi2_f64_kernel<JJ, false, true><<<grid, tile.block, smem, st>>>(a, tile.G,            \
                                                                      tile.obs_tile, out, resid); \
  } else {                                                                                 \
    err = set_smem(chi2_f64_kernel<JJ>, smem);                                             \
    if (err == cudaSuccess)                                                                \
      chi2_f64_kernel<JJ><<<grid, tile.block, smem, st>>>(a, tile.G, tile.obs_tile, out,     \
                                                          resid);                          \
  }
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t launch_chi2_single(const UniformArgs &a, const Tile &tile, float *out, float *resid,
                               cudaStream_t st) {
  const size_t smem = smem_chi2_mixed(a.n_pl, tile);
  const int grid = grid_for(a.n_sys, tile.block / tile.G);
  const MixedPrep none{nullptr, nullptr, nullptr, nullptr};
  cudaError_t err = cudaSuccess;
#define KC_LAUNCH(JJ)                                                                         \
  err = set_smem(chi2_mixed_kernel<JJ, false, false, true>, smem);                            \
  if (err == cudaSuccess)                                                                     \
    chi2_mixed_kernel<JJ, false, false, true><<<grid, tile.block, smem, st>>>(a, none, tile.G,  \
                                                                              tile.obs_tile,  \
                                                                              out, resid);
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t launch_nll_mixed(const UniformArgs &a, const Tile &tile, float *out, cudaStream_t st) {
  const size_t smem = smem_chi2_mixed(a.n_pl, tile);
  const int grid = grid_for(a.n_sys, tile.block / tile.G);
  const MixedPrep none{nullptr, nullptr, nullptr, nullptr};
  cudaError_t err = cudaSuccess;
#define KC_LAUNCH(JJ)                                                                       \
  err = set_smem(chi2_mixed_kernel<JJ, false, true>, smem);                                 \
  if (err == cudaSuccess)                                                                   \
    chi2_mixed_kernel<JJ, false, true><<<grid, tile.block, smem, st>>>(a, none, tile.G,       \
                                                                       tile.obs_tile, out,   \
                                                                       nullptr);
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t launch_nll_f64(const UniformArgs &a, const Tile &tile, double *out, cudaStream_t st) {
  const size_t smem = smem_chi2_f64(a.n_pl, tile);
  const int grid = grid_for(a.n_sys, tile.block / tile.G);
  cudaError_t err = cudaSuccess;
#define KC_LAUNCH(JJ)                                                                      \
  err = set_smem(chi2_f64_kernel<JJ, true>, smem);                                         \
  if (err == cudaSuccess)                                                                  \
    chi2_f64_kernel<JJ, true><<<grid, tile.block, smem, st>>>(a, tile.G, tile.obs_tile, out, \
                                                              nullptr);
  KC_DISPATCH_J(a.n_pl, KC_LAUNCH)
#undef KC_LAUNCH
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t launch_rv_predict(const double *params, const double *t, int64_t n_sys, int n_pl,
                              int n_obs, double t0, double *v_out, cudaStream_t st) {
  const int64_t total = n_sys * (int64_t)n_obs;
  rv_predict_kernel<<<elementwise_grid(total), 256, 0, st>>>(params, t, n_sys, n_pl, n_obs, t0,
                                                             v_out);
  return cudaGetLastError();
}

cudaError_t launch_kepler_f64(const double *M, const double *e, int64_t n, double *E,
                              cudaStream_t st) {
  kepler_f64_kernel<<<elementwise_grid(n), 256, 0, st>>>(M, e, n, E);
  return cudaGetLastError();
}

cudaError_t launch_kepler_f32(const float *M, const float *e, int64_t n, float *E,
                              cudaStream_t st) {
  kepler_f32_kernel<<<elementwise_grid((n + 3) / 4), 256, 0, st>>>(M, e, n, E);
  return cudaGetLastError();
}

}  // namespace kc
