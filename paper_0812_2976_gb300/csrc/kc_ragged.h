// kc_ragged.h -- device descriptors and launchers of the ragged path
// (kc_ragged.cu), used by the plan runtime (kc_plan.cu).  Not installed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kc {

// Converted observation of the FP64 ragged path: t - t_ref, v, weight
// 1/(sigma^2 + jitter^2), t - t0.
struct __align__(32) ObsR64 {
  double tau, v, w, dt;
};

// Device view of a ragged batch.  System s: n_pl[s] planets whose
// parameters start at params[par_off[s]]; observations [obs_off[s],
// obs_off[s+1]) of the plan's converted arrays; t_ref[s] is its first
// observation time.  order lists the systems in decreasing work.
struct RaggedDev {
  const int64_t *obs_off;
  const int64_t *par_off;
  const int32_t *n_pl;
  const int64_t *order;
  const double *t_ref;
  int64_t n_sys;
  double t0;
  unsigned long long *invalid;   // NaN-result counter (kc_last_device_error) or NULL
  int64_t n_obs_total;           // observations of the plan (obs_off[n_sys])
  int64_t n_par_total;           // packed parameters of the plan (par_off[n_sys])
};

// Converts t, v, sigma (device, [obs_off[n_sys]]) to the kernel's form:
// mixed: obs_a float4 (tau_hi, tau_lo, v_hi, v_lo), obs_b float2 (w, t - t0);
// fp64: obs_a ObsR64, obs_b unused.  Fills t_ref.
cudaError_t ragged_prep(const RaggedDev &d, int mode, const double *t, const double *v,
                        const double *sigma, double jitter2, void *obs_a, void *obs_b,
                        double *t_ref, cudaStream_t st);

// The persistent kernel; *queue must be zero when it starts.
cudaError_t ragged_launch(const RaggedDev &d, int mode, bool grad, const void *obs_a,
                          const void *obs_b, const double *params, void *chi2, void *grad_out,
                          unsigned long long *queue, int grid, int block, cudaStream_t st);

const void *ragged_kernel_fn(int mode, bool grad);

cudaError_t launch_predict_ragged(const double *params, const int64_t *par_off,
                                  const int32_t *n_pl, const double *t, const int64_t *obs_off,
                                  int64_t n_sys, double t0, double *v_out, cudaStream_t st);
int ragged_max_blocks_per_sm(int mode, bool grad, int block);

}  // namespace kc
