// kc_noalloc.cu -- kc_chi2_eval_mixed_noalloc: the two-pass mixed chi-square
// (preparation kernel + main kernel, see kc_fwd.cu) with its scratch in a
// fixed array that lives in the library's device image, so the call itself
// never allocates device memory.
//
// Who needs this: callers that may not allocate at the moment they evaluate,
// e.g. code running under a strict memory budget where every device byte is
// reserved up front, a host process whose allocator must not be re-entered
// (inside another library's callback), or a scheduler that forbids
// cudaMalloc / pool growth on its critical path.  They pass inputs and
// outputs as usual; the intermediate per-planet constants and converted
// observations go to the array below instead of to a memory pool.
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>

#include "kc_internal.h"

namespace {

// The scratch array.  Every GPU that loads libkc.so holds it until the
// process exits.  Host code must not take its address directly (the host
// symbol is only a stand-in); it asks the runtime for the device address.
static __device__ __align__(256) unsigned char kc_noalloc_scratch[KC_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
std::map<int, void *> g_addr;   // device ordinal -> device address of the array

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
cudaError_t scratch_address(void **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_addr.find(dev);
  if (it != g_addr.end()) {
    *ptr = it->second;
    return cudaSuccess;
  }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, kc_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_addr[dev] = p;
  *ptr = p;
  return cudaSuccess;
}

}  // namespace

extern "C" kc_status kc_chi2_eval_mixed_noalloc(const double *params, const double *t,
                                                const double *v_obs, const double *sigma,
                                                int64_t n_sys, int32_t n_pl, int32_t n_obs,
                                                double t0, double jitter, float *out,
                                                float *max_kepler_resid, kc_stream stream) {
  const char *fn = "kc_chi2_eval_mixed_noalloc";
  if (n_sys < 0) return kc::fail(KC_ERR_ARG, "%s: n_sys < 0", fn);
  // the same upper bound as every other uniform call: it keeps the scratch
  // size below (the products of n_sys in size_t) from wrapping around
  if (n_sys > (int64_t(1) << 40)) return kc::fail(KC_ERR_ARG, "%s: n_sys too large", fn);
  if (n_pl < 1 || n_pl > KC_MAX_PLANETS)
    return kc::fail(KC_ERR_ARG, "%s: n_pl = %d outside 1..%d", fn, n_pl, KC_MAX_PLANETS);
  if (n_obs < 0 || n_obs > KC_MAX_OBS)
    return kc::fail(KC_ERR_ARG, "%s: n_obs = %d outside 0..%d", fn, n_obs, KC_MAX_OBS);
  if (!std::isfinite(t0) || !std::isfinite(jitter))
    return kc::fail(KC_ERR_ARG, "%s: t0 and jitter must be finite", fn);
  if (n_sys == 0) return kc::ok();
  if (!params || !out || (n_obs > 0 && (!t || !v_obs || !sigma)))
    return kc::fail(KC_ERR_ARG, "%s: NULL input or output", fn);
  if (((uintptr_t)params | (uintptr_t)t | (uintptr_t)v_obs | (uintptr_t)sigma) & 7)
    return kc::fail(KC_ERR_ARG, "%s: input not 8-byte aligned", fn);
  const size_t need = kc::mixed_prep_bytes(n_sys, n_pl, n_obs);
  if (need > (size_t)KC_NOALLOC_SCRATCH_BYTES)
    return kc::fail(KC_ERR_ARG,
                    "%s: needs %zu bytes of scratch for n_sys=%lld, n_pl=%d, n_obs=%d; the "
                    "fixed array holds %zu (32 B per planet + 4 B per system + 20 B per "
                    "observation, each part rounded up to 256 B)",
                    fn, need, (long long)n_sys, n_pl, n_obs, (size_t)KC_NOALLOC_SCRATCH_BYTES);
  void *scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return kc::cuda_status(e, "kc_chi2_eval_mixed_noalloc: scratch address");
  // Nothing in the array has to start at zero: the preparation kernel of this
  // call writes every byte the main kernel then reads.
  const kc::UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, t0, jitter * jitter,
                          kc::invalid_counter()};
  kc::Tile tile = kc::choose_tile(kc::Kind::Chi2Mixed, n_sys, n_pl, n_obs);
  if (tile.G > tile.block || tile.split >= 2)
    tile = kc::default_tile(kc::Kind::Chi2Mixed, n_sys, n_pl, n_obs);
  tile.split = 1;
  return kc::cuda_status(kc::launch_chi2_mixed_prepared(a, tile, scratch, out, max_kepler_resid,
                                                        reinterpret_cast<cudaStream_t>(stream)),
                         fn);
}
