// kc_api.cu -- the library's C ABI (include/kc.h): argument checks, launch
// shapes and error reporting around the kernels of kc_fwd.cu / kc_grad.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kc_internal.h"
#include "kc_ragged.h"

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace kc {

kc_status fail(kc_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

kc_status ok() {
  g_last_error.clear();
  return KC_OK;
}

kc_status cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return ok();
  cudaGetLastError();   // a failed API call leaves its error as the "last" one: clear it
  return fail(KC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;
}  // namespace

// One memory pool per device for the library's stream-ordered scratch; it
// keeps up to 256 MiB cached between calls so repeated calls do not go back
// to the driver.
cudaError_t scratch_alloc(void **ptr, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = 256ull << 20;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      g_pools[dev] = pool;
    } else {
      pool = it->second;
    }
  }
  return cudaMallocFromPoolAsync(ptr, bytes > 0 ? bytes : 256, pool, st);
}

namespace {
// [0]: systems whose result came out NaN (invalid parameters or
// observations), summed over every launch on the device since the last
// read; [1]: the first failed index check of a KC_DEBUG build (zero if none).
__device__ unsigned long long g_invalid_systems[2] = {0ull, 0ull};
std::mutex g_inv_mu;
std::map<int, unsigned long long *> g_inv_addr;
}  // namespace

namespace {
std::mutex g_sm_mu;
std::map<int, int> g_sm_count;
}  // namespace

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> lk(g_sm_mu);
  auto it = g_sm_count.find(dev);
  if (it != g_sm_count.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  g_sm_count[dev] = n;
  return n;
}

unsigned long long *invalid_counter() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_inv_mu);
  auto it = g_inv_addr.find(dev);
  if (it != g_inv_addr.end()) return it->second;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_invalid_systems) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  g_inv_addr[dev] = static_cast<unsigned long long *>(p);
  return static_cast<unsigned long long *>(p);
}

}  // namespace kc

using kc::cuda_status;
using kc::fail;
using kc::ok;

namespace {

kc_status check_uniform(const double *params, const double *t, const double *v,
                        const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                        const void *out, const char *fn) {
  if (n_sys < 0) return fail(KC_ERR_ARG, "%s: n_sys < 0", fn);
  if (n_pl < 1 || n_pl > KC_MAX_PLANETS)
    return fail(KC_ERR_ARG, "%s: n_pl = %d outside 1..%d", fn, n_pl, KC_MAX_PLANETS);
  if (n_obs < 0 || n_obs > KC_MAX_OBS)
    return fail(KC_ERR_ARG, "%s: n_obs = %d outside 0..%d", fn, n_obs, KC_MAX_OBS);
  if (n_sys > (int64_t(1) << 40)) return fail(KC_ERR_ARG, "%s: n_sys too large", fn);
  if (n_sys > 0) {
    if (!params) return fail(KC_ERR_ARG, "%s: params is NULL", fn);
    if (!out) return fail(KC_ERR_ARG, "%s: output is NULL", fn);
    if (n_obs > 0 && (!t || !v || !sigma))
      return fail(KC_ERR_ARG, "%s: t, v_obs or sigma is NULL", fn);
  }
  const uintptr_t mis = (uintptr_t)params | (uintptr_t)t | (uintptr_t)v | (uintptr_t)sigma;
  if (mis & 7) return fail(KC_ERR_ARG, "%s: input not 8-byte aligned", fn);
  return KC_OK;
}

}  // namespace

namespace kc {

int obs_tile_for(Kind kind, int n_obs) {
  const bool f64 = kind == Kind::Chi2F64 || kind == Kind::GradF64;
  const int cap = f64 ? 2048 : 4096;
  return n_obs < cap ? (n_obs > 0 ? n_obs : 1) : cap;
}

// Built-in launch shape.  G threads share one system; enough threads to fill
// the device's SMs a few times over, but each thread keeps at least four
// observations so the per-system combine stays cheap.
Tile default_tile(Kind kind, int64_t n_sys, int n_pl, int n_obs) {
  const bool grad = kind == Kind::GradF64 || kind == Kind::GradMixed;
  Tile t;
  t.block = 256;
  const int64_t want_threads = int64_t(sm_count()) * 2048 * 2;
  int G = 1;
  while (G < 256 && n_sys * G < want_threads) G <<= 1;
  const int max_g_obs = n_obs >= 4 ? n_obs / 4 : 1;
  while (G > 1 && G > max_g_obs) G >>= 1;
  if (grad && G > 32) G = 32;
  if (G < 4) G = 4;
  t.G = G;
  t.obs_tile = obs_tile_for(kind, n_obs);
  (void)n_pl;
  return t;
}

namespace {

int bucket(int64_t x) {
  int b = 0;
  while (x > 1) {
    x >>= 1;
    ++b;
  }
  return b;
}

// A table entry holds for one kernel, planet count, power-of-two size class
// of n_sys and n_obs, and SM count (a shape tuned on one part is not taken
// for another with a different number of SMs).
struct TileKey {
  int kind, n_pl, sys_b, obs_b, sms;
  bool operator<(const TileKey &o) const {
    return std::tie(kind, n_pl, sys_b, obs_b, sms) <
           std::tie(o.kind, o.n_pl, o.sys_b, o.obs_b, o.sms);
  }
};

std::mutex g_tile_mu;
std::map<TileKey, Tile> g_tiles;

TileKey key_of(Kind kind, int64_t n_sys, int n_pl, int n_obs) {
  return TileKey{(int)kind, n_pl, bucket(n_sys), bucket(n_obs), sm_count()};
}

}  // namespace

// The tile used without a table entry.
Tile builtin_tile(Kind kind, int64_t n_sys, int n_pl, int n_obs) {
  if (kind == Kind::Chi2Mixed) return warp_tile(n_sys, n_pl, n_obs);
  if (kind == Kind::GnMixed) return Tile{32, 128, 0, gn_default_variant(n_pl)};
  return default_tile(kind, n_sys, n_pl, n_obs);
}

bool has_tile_entry(Kind kind, int64_t n_sys, int n_pl, int n_obs) {
  std::lock_guard<std::mutex> lk(g_tile_mu);
  return g_tiles.count(key_of(kind, n_sys, n_pl, n_obs)) != 0;
}

Tile choose_tile(Kind kind, int64_t n_sys, int n_pl, int n_obs) {
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tiles.find(key_of(kind, n_sys, n_pl, n_obs));
    if (it != g_tiles.end()) {
      Tile t = it->second;
      t.obs_tile = obs_tile_for(kind, n_obs);
      return t;
    }
  }
  return builtin_tile(kind, n_sys, n_pl, n_obs);
}

}  // namespace kc

using kc::Kind;
using kc::Tile;
using kc::UniformArgs;

extern "C" {

const char *kc_status_string(kc_status s) {
  switch (s) {
    case KC_OK: return "ok";
    case KC_ERR_ARG: return "invalid argument";
    case KC_ERR_CUDA: return "CUDA error";
    case KC_ERR_NOMEM: return "out of device memory";
    case KC_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *kc_last_error(void) { return g_last_error.c_str(); }

kc_status kc_measure_pipe_rate(int32_t pipe, double *ops_per_sm_clock, kc_stream stream) {
  const char *fn = "kc_measure_pipe_rate";
  if (!ops_per_sm_clock) return fail(KC_ERR_ARG, "%s: NULL pointer", fn);
  if (pipe != 0 && pipe != 1) return fail(KC_ERR_ARG, "%s: pipe must be 0 (FP32) or 1 (FP64)", fn);
  *ops_per_sm_clock = 0.0;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e, fn);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool f64 = pipe == 1;
  const int iters = f64 ? 256 : 16384;     // a few ms either way
  void *sink = nullptr;
  long long *cyc_d = nullptr;
  e = cudaMallocAsync(&sink, (size_t)n_sm * 1024 * (f64 ? 8 : 4), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&cyc_d, sizeof(long long) * n_sm, s);
  std::vector<long long> cyc(n_sm, 0);
  if (e == cudaSuccess) e = kc::probe_fma_rate(f64, n_sm, iters / 4, sink, cyc_d, s);  // warm-up
  if (e == cudaSuccess) e = kc::probe_fma_rate(f64, n_sm, iters, sink, cyc_d, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cyc.data(), cyc_d, sizeof(long long) * n_sm, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (sink) cudaFreeAsync(sink, s);
  if (cyc_d) cudaFreeAsync(cyc_d, s);
  if (e != cudaSuccess) return cuda_status(e, fn);
  // the slowest CTA sets the rate an SM sustains
  long long worst = 1;
  for (long long c : cyc) worst = c > worst ? c : worst;
  *ops_per_sm_clock = 1024.0 * 8.0 * iters / (double)worst;
  return ok();
}

kc_status kc_last_device_error(int64_t *n_invalid) {
  if (!n_invalid) return fail(KC_ERR_ARG, "kc_last_device_error: NULL pointer");
  *n_invalid = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "kc_last_device_error: device");
  unsigned long long n = 0, zero = 0;
  e = cudaMemcpyFromSymbol(&n, kc::g_invalid_systems, sizeof(n));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kc::g_invalid_systems, &zero, sizeof(zero));
  if (e != cudaSuccess) return cuda_status(e, "kc_last_device_error: counter");
  *n_invalid = (int64_t)n;
  return ok();
}

kc_status kc_debug_word(uint64_t *word) {
  if (!word) return fail(KC_ERR_ARG, "kc_debug_word: NULL pointer");
  *word = 0;
#ifndef KC_DEBUG
  return fail(KC_ERR_UNSUPPORTED, "kc_debug_word: library built without KC_DEBUG");
#else
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "kc_debug_word: device");
  unsigned long long w = 0, zero = 0;
  e = cudaMemcpyFromSymbol(&w, kc::g_invalid_systems, sizeof(w), sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbol(kc::g_invalid_systems, &zero, sizeof(zero), sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_status(e, "kc_debug_word: word");
  *word = w;
  return ok();
#endif
}

int32_t kc_version(void) { return 100; }

kc_status kc_chi2_eval_ex(const double *params, const double *t, const double *v_obs,
                          const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                          double t0, double jitter, kc_mode mode, void *out,
                          float *max_kepler_resid, kc_stream stream) {
  kc_status st = check_uniform(params, t, v_obs, sigma, n_sys, n_pl, n_obs, out,
                               "kc_chi2_eval_ex");
  if (st != KC_OK) return st;
  if (mode != KC_FP64 && mode != KC_MIXED && mode != KC_FP32)
    return fail(KC_ERR_ARG, "kc_chi2_eval_ex: bad mode");
  if (!std::isfinite(t0) || !std::isfinite(jitter))
    return fail(KC_ERR_ARG, "kc_chi2_eval_ex: t0 and jitter must be finite");
  if (n_sys == 0) return ok();
  UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, t0, jitter * jitter, kc::invalid_counter()};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == KC_FP64) {
    const Tile tile = kc::choose_tile(Kind::Chi2F64, n_sys, n_pl, n_obs);
    return cuda_status(kc::launch_chi2_f64(a, tile, static_cast<double *>(out),
                                           max_kepler_resid, s),
                       "kc_chi2_eval_ex (fp64)");
  }
  if (mode == KC_FP32)
    return cuda_status(kc::launch_chi2_single(a, kc::default_tile(Kind::Chi2Mixed, n_sys, n_pl,
                                                                  n_obs),
                                              static_cast<float *>(out), max_kepler_resid, s),
                       "kc_chi2_eval_ex (fp32)");
  const Tile tile = kc::choose_tile(Kind::Chi2Mixed, n_sys, n_pl, n_obs);
  return cuda_status(kc::launch_chi2_mixed(a, tile, static_cast<float *>(out),
                                           max_kepler_resid, s),
                     "kc_chi2_eval_ex (mixed)");
}

kc_status kc_chi2_eval(const double *params, const double *t, const double *v_obs,
                       const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                       double *out, kc_stream stream) {
  return kc_chi2_eval_ex(params, t, v_obs, sigma, n_sys, n_pl, n_obs, 0.0, 0.0, KC_FP64, out,
                         nullptr, stream);
}

kc_status kc_chi2_eval_mixed(const double *params, const double *t, const double *v_obs,
                             const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                             float *out, float *max_kepler_resid, kc_stream stream) {
  return kc_chi2_eval_ex(params, t, v_obs, sigma, n_sys, n_pl, n_obs, 0.0, 0.0, KC_MIXED, out,
                         max_kepler_resid, stream);
}

kc_status kc_chi2_grad(const double *params, const double *t, const double *v_obs,
                       const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                       double t0, double jitter, kc_mode mode, void *chi2_out, void *grad_out,
                       kc_stream stream) {
  kc_status st = check_uniform(params, t, v_obs, sigma, n_sys, n_pl, n_obs, grad_out,
                               "kc_chi2_grad");
  if (st != KC_OK) return st;
  if (mode != KC_FP64 && mode != KC_MIXED) return fail(KC_ERR_ARG, "kc_chi2_grad: bad mode");
  if (!std::isfinite(t0) || !std::isfinite(jitter))
    return fail(KC_ERR_ARG, "kc_chi2_grad: t0 and jitter must be finite");
  if (n_sys == 0) return ok();
  UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, t0, jitter * jitter, kc::invalid_counter()};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == KC_FP64) {
    const Tile tile = kc::choose_tile(Kind::GradF64, n_sys, n_pl, n_obs);
    return cuda_status(kc::launch_grad_f64(a, tile, static_cast<double *>(chi2_out),
                                           static_cast<double *>(grad_out), s),
                       "kc_chi2_grad (fp64)");
  }
  const Tile tile = kc::choose_tile(Kind::GradMixed, n_sys, n_pl, n_obs);
  return cuda_status(kc::launch_grad_mixed(a, tile, static_cast<float *>(chi2_out),
                                           static_cast<float *>(grad_out), s),
                     "kc_chi2_grad (mixed)");
}

// Tile for the free-jitter kernels: the tuned or default shape of the
// fused kernel of that kind (they have no two-pass variant).
static Tile nll_tile(Kind kind, int64_t n_sys, int32_t n_pl, int32_t n_obs) {
  Tile tile = kc::choose_tile(kind, n_sys, n_pl, n_obs);
  if (tile.split != 0 || tile.G > tile.block) tile = kc::default_tile(kind, n_sys, n_pl, n_obs);
  tile.split = 0;
  return tile;
}

kc_status kc_chi2_gauss_newton(const double *params, const double *t, const double *v_obs,
                               const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                               double t0, double jitter, kc_mode mode, void *chi2_out,
                               void *grad_out, void *jtj_out, kc_stream stream) {
  const char *fn = "kc_chi2_gauss_newton";
  kc_status st = check_uniform(params, t, v_obs, sigma, n_sys, n_pl, n_obs, jtj_out, fn);
  if (st != KC_OK) return st;
  if (mode != KC_FP64 && mode != KC_MIXED) return fail(KC_ERR_ARG, "%s: bad mode", fn);
  if (!std::isfinite(t0) || !std::isfinite(jitter))
    return fail(KC_ERR_ARG, "%s: t0 and jitter must be finite", fn);
  const uintptr_t al = mode == KC_FP64 ? 7 : 3;
  if (((uintptr_t)chi2_out | (uintptr_t)grad_out | (uintptr_t)jtj_out) & al)
    return fail(KC_ERR_ARG, "%s: output not aligned for its type", fn);
  if (n_sys == 0) return ok();
  UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, t0, jitter * jitter,
                kc::invalid_counter()};
  int variant = 0;
  if (mode == KC_MIXED) {
    variant = kc::choose_tile(Kind::GnMixed, n_sys, n_pl, n_obs).split;
    if (!kc::gn_variant_ok(variant, n_pl)) variant = 0;
  }
  return cuda_status(kc::launch_gauss_newton(a, mode == KC_FP64, chi2_out, grad_out, jtj_out,
                                             reinterpret_cast<cudaStream_t>(stream), variant),
                     fn);
}

kc_status kc_nll_eval(const double *params, const double *t, const double *v_obs,
                      const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs, double t0,
                      kc_mode mode, void *out, kc_stream stream) {
  kc_status st = check_uniform(params, t, v_obs, sigma, n_sys, n_pl, n_obs, out, "kc_nll_eval");
  if (st != KC_OK) return st;
  if (mode != KC_FP64 && mode != KC_MIXED) return fail(KC_ERR_ARG, "kc_nll_eval: bad mode");
  if (!std::isfinite(t0)) return fail(KC_ERR_ARG, "kc_nll_eval: t0 must be finite");
  if (n_sys == 0) return ok();
  UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, t0, 0.0, kc::invalid_counter()};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == KC_FP64)
    return cuda_status(kc::launch_nll_f64(a, nll_tile(Kind::Chi2F64, n_sys, n_pl, n_obs),
                                          static_cast<double *>(out), s),
                       "kc_nll_eval (fp64)");
  return cuda_status(kc::launch_nll_mixed(a, nll_tile(Kind::Chi2Mixed, n_sys, n_pl, n_obs),
                                          static_cast<float *>(out), s),
                     "kc_nll_eval (mixed)");
}

kc_status kc_nll_grad(const double *params, const double *t, const double *v_obs,
                      const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs, double t0,
                      kc_mode mode, void *nll_out, void *grad_out, kc_stream stream) {
  kc_status st = check_uniform(params, t, v_obs, sigma, n_sys, n_pl, n_obs, grad_out,
                               "kc_nll_grad");
  if (st != KC_OK) return st;
  if (mode != KC_FP64 && mode != KC_MIXED) return fail(KC_ERR_ARG, "kc_nll_grad: bad mode");
  if (!std::isfinite(t0)) return fail(KC_ERR_ARG, "kc_nll_grad: t0 must be finite");
  if (n_sys == 0) return ok();
  UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, t0, 0.0, kc::invalid_counter()};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == KC_FP64)
    return cuda_status(kc::launch_grad_f64(a, nll_tile(Kind::GradF64, n_sys, n_pl, n_obs),
                                           static_cast<double *>(nll_out),
                                           static_cast<double *>(grad_out), s, true),
                       "kc_nll_grad (fp64)");
  return cuda_status(kc::launch_grad_mixed(a, nll_tile(Kind::GradMixed, n_sys, n_pl, n_obs),
                                           static_cast<float *>(nll_out),
                                           static_cast<float *>(grad_out), s, true),
                     "kc_nll_grad (mixed)");
}

kc_status kc_demcmc_step(double *states, void *chi2, int64_t n_chains, int32_t n_pl,
                         const double *t, const double *v_obs, const double *sigma, int32_t n_obs,
                         double t0, double jitter, kc_mode mode, int64_t first, int64_t count,
                         int64_t partner_first, int64_t partner_count, double gamma,
                         const double *eps_scale, const double *z, const double *u,
                         double *proposals, void *chi2_prop, int32_t *accepted,
                         kc_stream stream) {
  const char *fn = "kc_demcmc_step";
  if (n_chains < 0 || first < 0 || count < 0 || first + count > n_chains)
    return fail(KC_ERR_ARG, "%s: need 0 <= first <= first + count <= n_chains", fn);
  if (partner_first < 0 || partner_count < 2 || partner_first + partner_count > n_chains)
    return fail(KC_ERR_ARG,
                "%s: need 0 <= partner_first, partner_count >= 2, partner_first + "
                "partner_count <= n_chains", fn);
  if (count > 0 && partner_first < first + count && first < partner_first + partner_count)
    return fail(KC_ERR_ARG, "%s: the partner range overlaps the updated range", fn);
  if (mode != KC_FP64 && mode != KC_MIXED) return fail(KC_ERR_ARG, "%s: bad mode", fn);
  if (!std::isfinite(gamma)) return fail(KC_ERR_ARG, "%s: gamma must be finite", fn);
  if (count == 0) return ok();
  if (!states || !chi2 || !eps_scale || !z || !u || !proposals || !chi2_prop)
    return fail(KC_ERR_ARG, "%s: NULL pointer", fn);
  if (((uintptr_t)states | (uintptr_t)eps_scale | (uintptr_t)z | (uintptr_t)u |
       (uintptr_t)proposals) & 7)
    return fail(KC_ERR_ARG, "%s: pointer not 8-byte aligned", fn);
  kc_status st = check_uniform(states, t, v_obs, sigma, count, n_pl, n_obs, chi2_prop, fn);
  if (st != KC_OK) return st;
  if (!std::isfinite(t0) || !std::isfinite(jitter))
    return fail(KC_ERR_ARG, "%s: t0 and jitter must be finite", fn);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the proposals formed in the mixed kernel's prologue (by the proposal
  // kernel before the other launch paths), their chi2, and the Metropolis
  // step in the kernel's epilogue
  UniformArgs a{proposals, t,   v_obs, sigma, count, n_pl, n_obs, t0, jitter * jitter,
                kc::invalid_counter(),
                kc::DemcAccept{states, chi2, u, accepted, first, z, eps_scale, partner_first,
                               partner_count, gamma}};
  cudaError_t e;
  if (mode == KC_FP64) {
    const Tile tile = kc::choose_tile(Kind::Chi2F64, count, n_pl, n_obs);
    e = kc::launch_chi2_f64(a, tile, static_cast<double *>(chi2_prop), nullptr, s);
  } else {
    // a tuned or pinned tile if there is one, else the built-in warp tile
    // with one warp (or less) per system
    Tile tile = kc::choose_tile(Kind::Chi2Mixed, count, n_pl, n_obs);
    if (!kc::has_tile_entry(Kind::Chi2Mixed, count, n_pl, n_obs))
      tile = kc::warp_tile(count, n_pl, n_obs, false);
    e = kc::launch_chi2_mixed(a, tile, static_cast<float *>(chi2_prop), nullptr, s);
  }
  return cuda_status(e, "kc_demcmc_step");
}

kc_status kc_rv_predict(const double *params, const double *t, int64_t n_sys, int32_t n_pl,
                        int32_t n_obs, double t0, double *v_out, kc_stream stream) {
  if (n_sys < 0 || n_obs < 0 || n_obs > KC_MAX_OBS)
    return fail(KC_ERR_ARG, "kc_rv_predict: bad sizes");
  if (n_pl < 1 || n_pl > KC_MAX_PLANETS) return fail(KC_ERR_ARG, "kc_rv_predict: bad n_pl");
  if (n_sys == 0 || n_obs == 0) return ok();
  if (!params || !t || !v_out) return fail(KC_ERR_ARG, "kc_rv_predict: NULL pointer");
  if (((uintptr_t)params | (uintptr_t)t | (uintptr_t)v_out) & 7)
    return fail(KC_ERR_ARG, "kc_rv_predict: pointer not 8-byte aligned");
  if (!std::isfinite(t0)) return fail(KC_ERR_ARG, "kc_rv_predict: t0 must be finite");
  return cuda_status(kc::launch_rv_predict(params, t, n_sys, n_pl, n_obs, t0, v_out,
                                           reinterpret_cast<cudaStream_t>(stream)),
                     "kc_rv_predict");
}

kc_status kc_rv_predict_ragged(const double *params, const int64_t *par_off,
                               const int32_t *n_pl, const double *t, const int64_t *obs_off,
                               int64_t n_sys, double t0, double *v_out, kc_stream stream) {
  if (n_sys < 0) return fail(KC_ERR_ARG, "kc_rv_predict_ragged: n_sys < 0");
  if (n_sys == 0) return ok();
  if (!params || !par_off || !n_pl || !t || !obs_off || !v_out)
    return fail(KC_ERR_ARG, "kc_rv_predict_ragged: NULL pointer");
  if (((uintptr_t)params | (uintptr_t)t | (uintptr_t)v_out | (uintptr_t)par_off |
       (uintptr_t)obs_off) & 7)
    return fail(KC_ERR_ARG, "kc_rv_predict_ragged: pointer not 8-byte aligned");
  if (!std::isfinite(t0)) return fail(KC_ERR_ARG, "kc_rv_predict_ragged: t0 must be finite");
  return cuda_status(kc::launch_predict_ragged(params, par_off, n_pl, t, obs_off, n_sys, t0,
                                               v_out, reinterpret_cast<cudaStream_t>(stream)),
                     "kc_rv_predict_ragged");
}

kc_status kc_kepler_solve(const void *M, const void *e, int64_t n, kc_mode mode, void *E_out,
                          kc_stream stream) {
  if (n < 0) return fail(KC_ERR_ARG, "kc_kepler_solve: n < 0");
  if (mode != KC_FP64 && mode != KC_MIXED) return fail(KC_ERR_ARG, "kc_kepler_solve: bad mode");
  if (n == 0) return ok();
  if (!M || !e || !E_out) return fail(KC_ERR_ARG, "kc_kepler_solve: NULL pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (mode == KC_FP64)
    return cuda_status(kc::launch_kepler_f64(static_cast<const double *>(M),
                                             static_cast<const double *>(e), n,
                                             static_cast<double *>(E_out), s),
                       "kc_kepler_solve (fp64)");
  return cuda_status(kc::launch_kepler_f32(static_cast<const float *>(M),
                                           static_cast<const float *>(e), n,
                                           static_cast<float *>(E_out), s),
                     "kc_kepler_solve (mixed)");
}

namespace {

kc::Kind kind_of(kc_kernel kernel, kc_mode mode) {
  if (kernel == KC_KERNEL_CHI2) return mode == KC_FP64 ? kc::Kind::Chi2F64 : kc::Kind::Chi2Mixed;
  if (kernel == KC_KERNEL_GN) return kc::Kind::GnMixed;
  return mode == KC_FP64 ? kc::Kind::GradF64 : kc::Kind::GradMixed;
}

// Tiled kernels: chi2 and gradient in both modes, Gauss-Newton mixed only.
bool kernel_ok(kc_kernel kernel, kc_mode mode) {
  if (mode != KC_FP64 && mode != KC_MIXED) return false;
  if (kernel == KC_KERNEL_GN) return mode == KC_MIXED;
  return kernel == KC_KERNEL_CHI2 || kernel == KC_KERNEL_GRAD;
}

bool tile_ok(kc_kernel kernel, kc_mode mode, const kc_tile &t) {
  const int G = t.threads_per_system, B = t.block;
  if (kernel == KC_KERNEL_GN)     // one warp per system, four per CTA; the variant in split
    return mode == KC_MIXED && G == 32 && B == 128 && (t.split == 0 || t.split == 4);
  if (t.split == 3) return kernel == KC_KERNEL_CHI2 && mode == KC_MIXED && kc::warp_tile_ok(G, B);
  if (B < 32 || B > 256 || (B & 31)) return false;
  if (t.split < 0 || t.split > 2) return false;
  if (t.split != 0 && (kernel != KC_KERNEL_CHI2 || mode != KC_MIXED)) return false;
  if (t.split == 2)     // one warp per chunk: G = 32 x chunks, chunks <= 32
    return G >= 32 && G <= 1024 && !(G & (G - 1));
  if (G < 1 || G > B || (B % G)) return false;
  // any G for the mixed chi2 kernel (a G that is not a power of two merges
  // its systems' partial sums through shared memory); powers of two elsewhere
  if ((G & (G - 1)) && (kernel != KC_KERNEL_CHI2 || mode != KC_MIXED)) return false;
  if (kernel == KC_KERNEL_GRAD && G > 32) return false;
  return true;
}

}  // namespace

kc_status kc_set_tile(kc_kernel kernel, kc_mode mode, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                      const kc_tile *tile) {
  if (!kernel_ok(kernel, mode) || n_sys < 0 || n_obs < 0 || n_pl < 1 || n_pl > KC_MAX_PLANETS)
    return fail(KC_ERR_ARG, "kc_set_tile: bad kernel, mode or sizes");
  const kc::TileKey key = kc::key_of(kind_of(kernel, mode), n_sys, n_pl, n_obs);
  std::lock_guard<std::mutex> lk(kc::g_tile_mu);
  if (!tile) {
    kc::g_tiles.erase(key);
    return ok();
  }
  if (!tile_ok(kernel, mode, *tile)) return fail(KC_ERR_ARG, "kc_set_tile: inadmissible tile");
  if (kernel == KC_KERNEL_GN && !kc::gn_variant_ok(tile->split, n_pl))
    return fail(KC_ERR_ARG, "kc_set_tile: the tcgen05 Gauss-Newton variant needs n_pl <= 3");
  kc::g_tiles[key] = Tile{tile->threads_per_system, tile->block, 0, tile->split};
  return ok();
}

kc_status kc_get_tile(kc_kernel kernel, kc_mode mode, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                      kc_tile *tile) {
  if (!tile || !kernel_ok(kernel, mode) || n_sys < 0 || n_obs < 0 || n_pl < 1 ||
      n_pl > KC_MAX_PLANETS)
    return fail(KC_ERR_ARG, "kc_get_tile: bad arguments");
  const Tile t = kc::choose_tile(kind_of(kernel, mode), n_sys, n_pl, n_obs);
  tile->threads_per_system = t.G;
  tile->block = t.block;
  tile->split = t.split;
  return ok();
}

kc_status kc_autotune(const double *params, const double *t, const double *v_obs,
                      const double *sigma, int64_t n_sys, int32_t n_pl, int32_t n_obs,
                      kc_kernel kernel, kc_mode mode, kc_tile *best, float *best_ms,
                      kc_stream stream) {
  kc_status st = check_uniform(params, t, v_obs, sigma, n_sys, n_pl, n_obs, params,
                               "kc_autotune");
  if (st != KC_OK) return st;
  if (!kernel_ok(kernel, mode)) return fail(KC_ERR_ARG, "kc_autotune: bad kernel or mode");
  if (n_sys == 0) return fail(KC_ERR_ARG, "kc_autotune: empty problem");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const kc::Kind kind = kind_of(kernel, mode);
  const size_t elem = mode == KC_FP64 ? sizeof(double) : sizeof(float);
  const size_t npar = 5 * (size_t)n_pl + 1;
  void *chi = nullptr, *grad = nullptr, *jtj = nullptr;
  cudaError_t e = cudaMallocAsync(&chi, elem * n_sys, s);
  if (e == cudaSuccess && kernel != KC_KERNEL_CHI2)
    e = cudaMallocAsync(&grad, elem * n_sys * npar, s);
  if (e == cudaSuccess && kernel == KC_KERNEL_GN)
    e = cudaMallocAsync(&jtj, elem * n_sys * (npar * (npar + 1) / 2), s);
  if (e != cudaSuccess) {
    if (chi) cudaFreeAsync(chi, s);
    if (grad) cudaFreeAsync(grad, s);
    return fail(KC_ERR_NOMEM, "kc_autotune: cannot allocate timing buffers: %s",
                cudaGetErrorString(e));
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  UniformArgs a{params, t, v_obs, sigma, n_sys, n_pl, n_obs, 0.0, 0.0, kc::invalid_counter()};
  auto launch = [&](const Tile &tile) -> cudaError_t {
    switch (kind) {
      case kc::Kind::Chi2F64: return kc::launch_chi2_f64(a, tile, (double *)chi, nullptr, s);
      case kc::Kind::Chi2Mixed: return kc::launch_chi2_mixed(a, tile, (float *)chi, nullptr, s);
      case kc::Kind::GradF64: return kc::launch_grad_f64(a, tile, (double *)chi, (double *)grad, s);
      case kc::Kind::GradMixed:
        return kc::launch_grad_mixed(a, tile, (float *)chi, (float *)grad, s);
      case kc::Kind::GnMixed:
        return kc::launch_gauss_newton(a, false, chi, grad, jtj, s, tile.split);
    }
    return cudaErrorInvalidValue;
  };
  float best_t = 1e30f;
  Tile best_tile = kc::builtin_tile(kind, n_sys, n_pl, n_obs);
  best_tile.obs_tile = kc::obs_tile_for(kind, n_obs);
  // the built-in tile is kept unless a candidate beats it by 1 % (shapes
  // within timing noise of each other would otherwise trade places from
  // one run to the next)
  float builtin_t = 1e30f;
  const Tile builtin = best_tile;
  const char *env = getenv("KC_AUTOTUNE_VERBOSE");     // candidate timings to stderr
  const bool verbose = env && env[0] == '1';
  cudaError_t err = cudaSuccess;
  // powers of two, plus G = 12, 24, 48 with 96- and 192-thread blocks, and
  // G = 8, 16, 32 with 160- and 224-thread blocks: the CTA count of a
  // batch that fills about one wave then spreads more evenly over the
  // SMs (on a GB300, 4096 systems at 16 threads: 293 CTAs of 224 threads,
  // two per SM on 141 of its SMs, where 256 CTAs of 256 threads leave 48
  // SMs with one)
  std::vector<kc_tile> cands;
  // Gauss-Newton: the U^T U update by mma.sync or by tcgen05
  if (kernel == KC_KERNEL_GN)
    for (int split : {0, 4})
      if (kc::gn_variant_ok(split, n_pl)) cands.push_back(kc_tile{32, 128, split});
  for (int split = 0; split <= 2 && kernel != KC_KERNEL_GN; ++split) {
    for (int B : {32, 64, 128, 256})
      for (int G = 1; G <= (split == 2 ? 1024 : B); G <<= 1) cands.push_back(kc_tile{G, B, split});
    if (split < 2) {
      for (int B : {96, 192})
        for (int G : {12, 24, 48}) cands.push_back(kc_tile{G, B, split});
      for (int B : {160, 224})
        for (int G : {8, 16, 32}) cands.push_back(kc_tile{G, B, split});
    }
  }
  // the warp-per-system kernel: 8 to 128 lanes per system (a system over
  // two or four warps at 64 and 128), 4..32 warps per CTA
  for (int G : {8, 16, 32, 64, 128})
    for (int W = 4; W <= 32 && kernel == KC_KERNEL_CHI2; ++W)
      if ((32 * W) % G == 0) cands.push_back(kc_tile{G, 32 * W, 3});
  for (const kc_tile &cand : cands) {
    const int G = cand.threads_per_system, B = cand.block, split = cand.split;
    if (!tile_ok(kernel, mode, cand)) continue;
    if (n_obs > 0 && G > n_obs && split != 3 && kernel != KC_KERNEL_GN) continue;
    if (split == 2 && G / 32 > (n_obs + 31) / 32) continue;   // chunks of >= 32 obs
    if (split == 3 && !kc::warp_lanes_fit(G, n_obs)) continue;  // >= 4 obs per lane
    Tile tile{G, B, kc::obs_tile_for(kind, n_obs), split};
    err = launch(tile);                       // warm-up (and smem attribute)
    if (err == cudaErrorInvalidConfiguration && split >= 3) {
      err = cudaSuccess;                      // does not fit on an SM: nothing launched
      continue;
    }
    if (err != cudaSuccess) break;
    // per launch: the mean of four launches back to back (as a caller
    // evaluating batch after batch runs them: launches that overlap their
    // neighbours' start and end are credited for it), the best of three
    constexpr int kBackToBack = 4;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      for (int i = 0; i < kBackToBack && err == cudaSuccess; ++i) err = launch(tile);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= kBackToBack;
      tmin = ms < tmin ? ms : tmin;
    }
    if (err != cudaSuccess) break;
    if (verbose)
      fprintf(stderr, "kc_autotune: kind %d n_sys %lld G %3d block %3d split %d: %9.2f us\n",
              (int)kind, (long long)n_sys, G, B, split, 1e3 * tmin);
    if (tile.G == builtin.G && tile.block == builtin.block && tile.split == builtin.split)
      builtin_t = tmin;
    if (tmin < best_t) {
      best_t = tmin;
      best_tile = tile;
    }
  }
  if (builtin_t < 1e30f && best_t > 0.99f * builtin_t) {
    best_t = builtin_t;
    best_tile = builtin;
  }
  cudaFreeAsync(chi, s);
  if (grad) cudaFreeAsync(grad, s);
  if (jtj) cudaFreeAsync(jtj, s);
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_status(err, "kc_autotune");
  {
    std::lock_guard<std::mutex> lk(kc::g_tile_mu);
    kc::g_tiles[kc::key_of(kind, n_sys, n_pl, n_obs)] = best_tile;
  }
  if (best) {
    best->threads_per_system = best_tile.G;
    best->block = best_tile.block;
    best->split = best_tile.split;
  }
  if (best_ms) *best_ms = best_t;
  return ok();
}

}  // extern "C"
