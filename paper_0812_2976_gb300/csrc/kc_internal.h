// kc_internal.h -- host-side declarations shared by the library's
// translation units (launchers and the tile table).  Not installed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/kc.h"

namespace kc {

// Launch shape of a uniform-batch kernel: each system is handled by G
// consecutive threads (a power of two, 1..block); a CTA of `block` threads
// covers block/G systems; observations are staged in shared memory
// `obs_tile` at a time.
struct Tile {
  int G;
  int block;
  int obs_tile;
  int split = 0;   // mixed chi2 only: 1, 2 = two-pass variants (see kc_fwd.cu),
                   // 3 = the warp-per-system kernel of kc_chi2_warp.cu
};

// DE-MC step carried by a chi2 launch: the batch's systems are proposals
// for chains first .. first + n_sys - 1 (params points at them), and each
// system's chi2 is compared with its chain's (accept iff ln u[3 c] <
// -(chi2* - chi2)/2), the accepted proposal copied over the chain's state.
// With z != NULL the proposals are still to be formed from the states, the
// partner range and the draws: the fused mixed kernel forms them in its
// prologue, every other launch path with the proposal kernel first.
// states == NULL: a plain evaluation.
struct DemcAccept {
  double *states;          // [n_chains][5 n_pl + 1]
  void *chi2;              // [n_chains], float (mixed) or double (FP64)
  const double *u;         // [n_sys][3]
  int32_t *accepted;       // [n_sys] or NULL
  int64_t first;
  const double *z = nullptr;          // [n_sys][5 n_pl + 1] standard normal draws
  const double *eps_scale = nullptr;  // [5 n_pl + 1]
  int64_t partner_first = 0, partner_count = 0;
  double gamma = 0.0;
};

struct UniformArgs {
  const double *params;
  const double *t;
  const double *v;
  const double *sigma;
  int64_t n_sys;
  int n_pl;
  int n_obs;
  double t0;
  double jitter2;
  // device counter of systems whose result is NaN (invalid inputs); may be
  // NULL (kc_last_device_error reads it)
  unsigned long long *invalid;
  DemcAccept demc = {};
};

// Number of SMs of the current device (cudaDevAttrMultiProcessorCount),
// queried once per device and cached (kc_api.cu).  Launch heuristics size
// their grids with it; 1 if no device can be queried (host-only use of the
// tile table), which still gives valid launch shapes.
int sm_count();

// The library's per-device words (kc_api.cu): [0] the invalid-system
// counter, [1] the first failed index check of a KC_DEBUG build.  Kernels
// receive the address of [0]; NULL if it cannot be obtained.
unsigned long long *invalid_counter();

// Counts a NaN result (one atomic per invalid system).
template <typename T>
__device__ __forceinline__ void note_invalid(unsigned long long *ctr, T value) {
  if (ctr != nullptr && value != value) atomicAdd(ctr, 1ull);
}

// Index checks of a KC_DEBUG build (the library compiled with -DKC_DEBUG).
// A failed check records its site and the offending index in the debug word
// (the first failure wins; kc_debug_word reads it) and returns false; the
// caller then carries on with a safe substitute (the access skipped, or an
// index known to be in range), so a failed check neither traps, faults nor
// leaves a barrier waiting.  In a normal build every check is true and
// compiles to nothing.  words: the address kernels receive as their
// invalid-system counter.
enum DebugSite : unsigned {
  kDbgParam = 1,       // parameter index of a uniform batch
  kDbgObs = 2,         // observation index of a uniform batch
  kDbgSmem = 3,        // shared-memory slot (setup item, staged observation, system)
  kDbgOrder = 4,       // ragged: queue entry outside 0 .. n_sys - 1
  kDbgPlanets = 5,     // ragged: planet count outside 1 .. KC_MAX_PLANETS
  kDbgObsOff = 6,      // ragged: observation range outside the plan's observations
  kDbgParOff = 7,      // ragged: parameter range outside the packed parameters
};

template <typename I>
__device__ __forceinline__ bool dbg_ok(unsigned long long *words, bool ok, DebugSite site,
                                       I index) {
#ifdef KC_DEBUG
  if (!ok && words != nullptr)
    atomicCAS(words + 1, 0ull,
              (1ull << 63) | ((unsigned long long)site << 48) |
                  ((unsigned long long)(long long)index & 0xffffffffffffull));
  return ok;
#else
  (void)words;
  (void)site;
  (void)index;
  return true;
#endif
}

// Stream-ordered scratch from the library's per-device memory pool
// (kc_api.cu); freed with cudaFreeAsync on the same stream.
cudaError_t scratch_alloc(void **ptr, size_t bytes, cudaStream_t st);

// Forward chi2 (kc_fwd.cu).  launch_chi2_mixed_prepared runs the split
// variant on caller-provided scratch of mixed_scratch_bytes() bytes (256-byte
// aligned).
size_t mixed_prep_bytes(int64_t n_sys, int n_pl, int n_obs);
size_t mixed_scratch_bytes(int64_t n_sys, int n_pl, int n_obs, const Tile &tile);
cudaError_t launch_chi2_mixed_prepared(const UniformArgs &a, const Tile &tile, void *scratch,
                                       float *out, float *resid, cudaStream_t st);
cudaError_t launch_chi2_f64(const UniformArgs &a, const Tile &tile, double *out,
                            float *resid, cudaStream_t st);
// Gauss-Newton matrix with chi2 and its gradient (kc_grad.cu): chi2 / grad
// may be NULL; jtj is [n_sys][n (n + 1)/2], n = 5 n_pl + 1; float (mixed) or
// double (f64).  variant (mixed only; the tile's split): 0 = U^T U by
// mma.sync, 4 = by tcgen05 MMAs for four systems stacked in an M = 64 tile
// (n_pl <= 3, gn_variant_ok).
cudaError_t launch_gauss_newton(const UniformArgs &a, bool f64, void *chi2, void *grad,
                                void *jtj, cudaStream_t st, int variant);
bool gn_variant_ok(int variant, int n_pl);
// Built-in choice of variant for the mixed Gauss-Newton kernel.
int gn_default_variant(int n_pl);

// FMA-pipe throughput probe (kc_probe.cu): one CTA of 1024 threads per SM
// (grid n_sm), eight FMA chains per thread, iters steps; writes each CTA's
// SM-clock cycles to cycles[n_sm]; sink is [n_sm * 1024] of the type.
cudaError_t probe_fma_rate(bool f64, int n_sm, int iters, void *sink, long long *cycles,
                           cudaStream_t st);

// Pure single-precision variant (KC_FP32, a precision comparison only):
// the fused mixed kernel with times and periods rounded to float.
cudaError_t launch_chi2_single(const UniformArgs &a, const Tile &tile, float *out, float *resid,
                               cudaStream_t st);
cudaError_t launch_chi2_mixed(const UniformArgs &a, const Tile &tile, float *out,
                              float *resid, cudaStream_t st);
// Warp-per-system mixed chi2 (kc_chi2_warp.cu): G = 8, 16 or 32 lanes per
// system, or 64 or 128 (a system over two or four warps), `block` threads (a
// multiple of 32 and of G, at most 1024) per CTA, one CTA per block / G
// systems; warp_tile picks the shape that spreads the work evenly over the
// SMs.  Carries a DE-MC step when a.demc.states is set.
bool warp_tile_ok(int G, int block);
int warp_lanes_for(int n_obs);
// G lanes per system give every lane at least 4 observations (G = 8: always)
bool warp_lanes_fit(int G, int n_obs);
// The built-in warp tile; multi_warp admits systems split over 2 or 4 warps
// (not for the DE-MC step, whose epilogue those shapes move behind a CTA
// barrier: 2.93e4 against 3.12e4 generations/s on halves of 2048 chains).
Tile warp_tile(int64_t n_sys, int n_pl, int n_obs, bool multi_warp = true);
cudaError_t launch_chi2_mixed_warp(const UniformArgs &a, const Tile &tile, float *out,
                                   float *resid, cudaStream_t st);
// Gradient (kc_grad.cu); nll = true: the free-jitter log-likelihood variant
// (parameters 5*n_pl + 2 per system).
cudaError_t launch_grad_f64(const UniformArgs &a, const Tile &tile, double *chi2,
                            double *grad, cudaStream_t st, bool nll = false);
cudaError_t launch_grad_mixed(const UniformArgs &a, const Tile &tile, float *chi2,
                              float *grad, cudaStream_t st, bool nll = false);
// Free-jitter negative log-likelihood, forward only (kc_fwd.cu).
cudaError_t launch_nll_mixed(const UniformArgs &a, const Tile &tile, float *out, cudaStream_t st);
cudaError_t launch_nll_f64(const UniformArgs &a, const Tile &tile, double *out, cudaStream_t st);
// Model velocities and elementwise Kepler (kc_fwd.cu).
cudaError_t launch_rv_predict(const double *params, const double *t, int64_t n_sys, int n_pl,
                              int n_obs, double t0, double *v_out, cudaStream_t st);
cudaError_t launch_kepler_f64(const double *M, const double *e, int64_t n, double *E,
                              cudaStream_t st);
cudaError_t launch_kepler_f32(const float *M, const float *e, int64_t n, float *E,
                              cudaStream_t st);

// Shared-memory bytes a uniform kernel needs for a tile.
size_t smem_chi2_f64(int n_pl, const Tile &tile);
size_t smem_chi2_mixed(int n_pl, const Tile &tile);
size_t smem_grad(int n_pl, const Tile &tile, bool f64);

// Launch shape for a problem (kc_api.cu): the tuned table, else a heuristic.
enum class Kind { Chi2F64 = 0, Chi2Mixed = 1, GradF64 = 2, GradMixed = 3, GnMixed = 4 };
Tile default_tile(Kind kind, int64_t n_sys, int n_pl, int n_obs);
Tile builtin_tile(Kind kind, int64_t n_sys, int n_pl, int n_obs);  // without a table entry
Tile choose_tile(Kind kind, int64_t n_sys, int n_pl, int n_obs);
bool has_tile_entry(Kind kind, int64_t n_sys, int n_pl, int n_obs);  // tuned or pinned
int obs_tile_for(Kind kind, int n_obs);

// DE-MC step pieces (kc_demcmc.cu).
cudaError_t launch_demcmc_propose(const double *states, int n_par, int64_t first, int64_t count,
                                  int64_t pfirst, int64_t pcount, double gamma,
                                  const double *eps_scale, const double *z, const double *u,
                                  double *prop, cudaStream_t st);
cudaError_t launch_demcmc_accept(double *states, void *chi2, const double *prop,
                                 const void *chi2_prop, int64_t first, int64_t count, int n_par,
                                 const double *u, bool f64, int32_t *accepted, cudaStream_t st);

// Thread-local error reporting of the C ABI (kc_api.cu).
kc_status fail(kc_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
kc_status ok();
kc_status cuda_status(cudaError_t e, const char *what);

}  // namespace kc
