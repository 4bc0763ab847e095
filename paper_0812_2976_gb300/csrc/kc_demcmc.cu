// kc_demcmc.cu -- one generation step of differential-evolution Markov chain
// Monte Carlo (DE-MC, ter Braak 2006) on the GPU, with chi2 from the fused
// kernels as the likelihood: the population-MCMC use the paper proposes for
// its evaluator (Sec. 6).
//
// Chain i of a population proposes x* = x_i + gamma (x_r1 - x_r2) + eps_i
// with r1 != r2 two other chains, and accepts with probability
// min(1, exp(-(chi2(x*) - chi2(x_i))/2)) (flat prior; invalid parameters give
// NaN chi2 and are rejected).  To update many chains at once and keep
// detailed balance, the population is split in two halves: a step updates
// one half, drawing r1, r2 from the other half, whose states stay fixed
// during the step (the ensemble parallelisation of Goodman & Weare as used by
// Foreman-Mackey et al. 2013).  The random numbers are inputs (standard
// normal and uniform draws), so the step is a deterministic function of
// them; the kernels turn them into the perturbation and the partner pair.
// In a mixed-precision step the fused chi2 kernel forms the proposals in its
// prologue and takes the Metropolis decision in its epilogue (kc_fwd.cu);
// the two kernels here serve the other launch paths.
#include <cmath>

#include "kc_device.cuh"
#include "kc_internal.h"

namespace kc {

namespace {

// One thread per (proposal, parameter): the partner pair (demc_partners)
// and the proposal (demc_proposal, kc_device.cuh).
__global__ void demcmc_propose_kernel(const double *__restrict__ states, int n_par, int64_t first,
                                      int64_t count, int64_t pfirst, int64_t pcount,
                                      double gamma, const double *__restrict__ eps_scale,
                                      const double *__restrict__ z, const double *__restrict__ u,
                                      double *__restrict__ prop) {
  const int64_t total = count * n_par;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / n_par;
    const int p = (int)(idx - c * n_par);
    const int64_t i = first + c;
    int64_t r1, r2;
    demc_partners(u[3 * c + 1], u[3 * c + 2], pfirst, pcount, r1, r2);
    prop[idx] = demc_proposal(states, n_par, i, r1, r2, p, gamma, eps_scale[p], z[idx]);
  }
}

// Metropolis decision in double precision: accept iff ln u < -(chi2* - chi2)/2.
template <typename T>
__global__ void demcmc_accept_kernel(double *__restrict__ states, T *__restrict__ chi2,
                                     const double *__restrict__ prop,
                                     const T *__restrict__ chi2_prop, int64_t first,
                                     int64_t count, int n_par, const double *__restrict__ u,
                                     int32_t *__restrict__ accepted) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = first + c;
    const double delta = (double)chi2_prop[c] - (double)chi2[i];
    const bool acc = log(u[3 * c]) < -0.5 * delta;      // false when delta is NaN
    if (acc) {
      for (int p = 0; p < n_par; ++p) states[i * n_par + p] = prop[c * n_par + p];
      chi2[i] = chi2_prop[c];
    }
    if (accepted) accepted[c] = acc ? 1 : 0;
  }
}

int grid_elems(int64_t n) {
  const int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 32;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_demcmc_propose(const double *states, int n_par, int64_t first, int64_t count,
                                  int64_t pfirst, int64_t pcount, double gamma,
                                  const double *eps_scale, const double *z, const double *u,
                                  double *prop, cudaStream_t st) {
  demcmc_propose_kernel<<<grid_elems(count * n_par), 256, 0, st>>>(
      states, n_par, first, count, pfirst, pcount, gamma, eps_scale, z, u, prop);
  return cudaGetLastError();
}

cudaError_t launch_demcmc_accept(double *states, void *chi2, const double *prop,
                                 const void *chi2_prop, int64_t first, int64_t count, int n_par,
                                 const double *u, bool f64, int32_t *accepted, cudaStream_t st) {
  if (f64)
    demcmc_accept_kernel<double><<<grid_elems(count), 256, 0, st>>>(
        states, (double *)chi2, prop, (const double *)chi2_prop, first, count, n_par, u,
        accepted);
  else
    demcmc_accept_kernel<float><<<grid_elems(count), 256, 0, st>>>(
        states, (float *)chi2, prop, (const float *)chi2_prop, first, count, n_par, u,
        accepted);
  return cudaGetLastError();
}

}  // namespace kc
