// kc_demc.cuh -- the DE-MC step's pieces that run inside the chi2 kernels:
// the proposal formed in a kernel's prologue and the Metropolis decision in
// its epilogue (differential-evolution MCMC, ter Braak 2006: the population
// MCMC the paper proposes as the evaluator's consumer, Sec. 6).  Shared by
// the fused kernels of kc_fwd.cu and the warp-per-system kernel of
// kc_chi2_warp.cu.
#pragma once

#include "kc_device.cuh"
#include "kc_internal.h"

namespace kc {

// The Metropolis decision of DE-MC in the epilogue of the chi2 kernel that
// has just evaluated proposal s (demcmc_accept_kernel's rule and
// arithmetic, applied to the value the kernel stores).  NPAR parameters per
// chain.  An accepted proposal is copied in chunks whose loads are all
// issued before their stores: the states and the proposals may alias as far
// as the compiler knows, so a plain loop would hold every load back until
// the one before it had returned (NPAR dependent memory round trips at the
// end of the CTA's work).
template <int NPAR, typename T>
__device__ __forceinline__ void demc_accept(const UniformArgs &a, int64_t s, T value) {
  constexpr int kCopy = 8;
  const DemcAccept &d = a.demc;
  const int64_t i = d.first + s;
  T *chi2 = static_cast<T *>(d.chi2);
  const double delta = (double)value - (double)chi2[i];
  const bool acc = log(d.u[3 * s]) < -0.5 * delta;      // false when delta is NaN
  if (acc) {
#pragma unroll
    for (int p0 = 0; p0 < NPAR; p0 += kCopy) {
      double x[kCopy];
#pragma unroll
      for (int k = 0; k < kCopy; ++k)
        if (p0 + k < NPAR) x[k] = a.params[s * NPAR + p0 + k];
#pragma unroll
      for (int k = 0; k < kCopy; ++k)
        if (p0 + k < NPAR) d.states[i * NPAR + p0 + k] = x[k];
    }
    chi2[i] = value;
  }
  if (d.accepted) d.accepted[s] = acc ? 1 : 0;
}

// Parameters p0 .. p0 + N - 1 of proposal s, formed in the fused kernel's
// prologue (the proposal kernel's arithmetic, demc_proposal) and stored to
// the proposals, which params points at (the caller's writable buffer).
template <int N>
__device__ __forceinline__ void demc_form(const UniformArgs &a, int64_t s, int p0, int npar,
                                          double (&out)[N]) {
  const DemcAccept &d = a.demc;
  int64_t r1, r2;
  demc_partners(d.u[3 * s + 1], d.u[3 * s + 2], d.partner_first, d.partner_count, r1, r2);
  double *prop = const_cast<double *>(a.params) + s * npar;
#pragma unroll
  for (int k = 0; k < N; ++k)
    out[k] = demc_proposal(d.states, npar, d.first + s, r1, r2, p0 + k, d.gamma,
                           d.eps_scale[p0 + k], d.z[s * npar + p0 + k]);
  // stored after every load (a store between them would hold the next
  // parameter's loads back until the previous ones had returned: the
  // proposals may alias the states as far as the compiler knows)
#pragma unroll
  for (int k = 0; k < N; ++k) prop[p0 + k] = out[k];
}

}  // namespace kc
