// kc_chi2_warp.cu -- the mixed-precision chi-square of a uniform batch with
// G = 8, 16, 32, 64 or 128 lanes per system (one warp per system at G = 32,
// two or four at 64 and 128), sized by the host so that the CTAs spread
// evenly over the SMs.
//
// Same arithmetic as the fused kernel of kc_fwd.cu (double-single phase,
// Sec. 5; Kepler's equation in single precision, Sec. 4.3; Eq. 3 velocity;
// Kahan sums of the planet velocities and of chi2, Sec. 4.4), laid out for
// the SMs rather than for a tile:
//
//  - A CTA of W warps evaluates W * 32 / G systems (one round).  The host
//    picks G and W so that the CTAs of the first wave land evenly on the
//    SMs (for 4096 systems, 27 warps per CTA: one CTA and 27 systems on
//    every SM, where tiles of 16 systems leave some SMs with 32 and others
//    with 16).  Larger batches run many waves; the hardware then overlaps
//    one CTA's prologue with the work of the others on its SM.
//  - Prologue: every global load (the reference time, this thread's
//    observation and its planet's parameters) is issued before any of them
//    is used, so the CTA waits for memory once.
//  - The observations (shared by every system, Sec. 4.1) are converted to
//    float pairs and staged in shared memory, padded with zero-weight
//    entries to whole chunks, so the inner loops have no tail.
//  - Each lane holds a chunk of kChunk observations (their phases and their
//    compensated velocity sums) in registers and streams the planets over
//    it: a planet's constants (phase, velocity and the hoisted part of
//    Mikkola's start, computed once per (system, planet)) are read from
//    shared memory once per chunk, and the chunk's kChunk Kepler solves are
//    independent chains for the scheduler to interleave.
//  - The lanes of a system combine their compensated sums with TwoSum
//    shuffles, and the warps of a system (G > 32) through a few words of
//    shared memory; no atomics, no scratch memory.  Splitting a system over
//    several warps keeps the SMs' warp slots filled when the batch is small
//    (2048 systems: 28 warps per SM instead of 14).
//  - Programmatic dependent launch: the kernel waits for the grids before
//    it in the stream to complete (griddepcontrol.wait, ahead of its first
//    global access) and at once lets the next launch on the stream begin
//    (griddepcontrol.launch_dependents), so that a following batch's CTAs
//    are placed on the SMs as this grid's CTAs exit instead of after the
//    whole grid has completed (back-to-back 4096 x 4 x 256 batches: 14.0 us
//    each instead of 16.4 us).  The launch asks for it only outside stream
//    capture: as programmatic edges in the DE-MC driver's graph (4096
//    chains, halves of 2048) it cost a quarter of the generations per
//    second (2.36e4 against 3.12e4), where back-to-back launches of 1024 to
//    4096 systems gained 2.7-2.9 us each.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "kc_demc.cuh"
#include "kc_device.cuh"
#include "kc_internal.h"

namespace kc {

namespace {

constexpr int kChunk = 4;           // observations per lane in registers
constexpr int kObsTileMax = 1024;   // observations staged per CTA at a time

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }
__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
// x rounded up to a multiple of the power of two m (no division)
__device__ __forceinline__ int round_up_pow2(int x, int m) { return (x + m - 1) & -m; }

// Planet constants of the kernel: phase and velocity (PlanetF) and the
// hoisted part of Mikkola's start (StartF); 48 bytes, three 16-byte loads.
struct PlanetW {
  PlanetF f;
  StartF m;
};

struct WarpLayout {
  size_t pl, gam, obs, w, red, total;
  __host__ __device__ WarpLayout(int spr, int J, int tile, int nwarps) {
    pl = 0;
    gam = pl + sizeof(PlanetW) * spr * J;
    obs = align16(gam + sizeof(float) * spr);
    w = obs + sizeof(float4) * tile;
    red = align16(w + sizeof(float) * tile);      // G > 32: 3 words per warp
    total = align16(red + sizeof(float) * 3 * nwarps);
  }
};

// Observations held per CTA: all of them (padded to whole chunks of every
// lane of a system) when they fit, else tiles of kObsTileMax.
__host__ __device__ inline int warp_obs_tile(int n_obs, int G) {
  return n_obs <= kObsTileMax ? round_up(n_obs > 0 ? n_obs : 1, G * kChunk) : kObsTileMax;
}

// Setup of one item of the CTA's round: items 0 .. spr*J - 1 are the
// (system, planet) constants, items spr*J .. spr*(J+1) - 1 the systems'
// gamma.  p holds the item's parameters (five, or gamma in p[0]); an
// invalid planet carries e = NaN, which poisons its system.
template <int J>
__device__ __forceinline__ void setup_item(int i, int spr, int64_t sys0, int64_t n_sys,
                                           const double (&p)[5], double t_ref, double t0,
                                           PlanetW *pl_s, float *gam_s, unsigned long long *dbg) {
  if (!dbg_ok(dbg, i < spr * (J + 1), kDbgSmem, i)) return;
  if (i < spr * J) {
    const int64_t s = sys0 + i / J;
    PlanetW q = {};
    if (s < n_sys) {
      q.f = planet_setup_mixed(p, t_ref, t0);
      if (!planet_valid(p[0], p[1], p[2], p[3], p[4])) q.f.e = __int_as_float(0x7fc00000);
      q.m = kepler_start_setup(q.f.e);
    }
    pl_s[i] = q;
  } else {
    const int sl = i - spr * J;
    float g = 0.0f;
    if (sys0 + sl < n_sys) g = finite_bits(p[0]) ? d2f(p[0]) : __int_as_float(0x7fc00000);
    gam_s[sl] = g;
  }
}

// The item's parameters.  DEMC: the launch evaluates DE-MC proposals; with
// a.demc.z set they are formed here from the chains' states and the draws
// (and stored to the proposals, which a.params points at).
template <int J, bool DEMC>
__device__ __forceinline__ void load_item(int i, int spr, int64_t sys0, const UniformArgs &a,
                                          double (&p)[5]) {
  const int npar = 5 * J + 1;
  if (i < spr * J) {
    const int sl = i / J, j = i - sl * J;
    const int64_t s = sys0 + sl;
    const int64_t at = s * npar + 5 * j;
    if (s < a.n_sys && dbg_ok(a.invalid, at + 4 < a.n_sys * npar, kDbgParam, at)) {
      if (DEMC && a.demc.z) {
        demc_form(a, s, 5 * j, npar, p);
      } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) p[k] = a.params[at + k];
      }
    }
  } else {
    const int64_t s = sys0 + (i - spr * J);
    if (s < a.n_sys && dbg_ok(a.invalid, s * npar + 5 * J < a.n_sys * npar, kDbgParam,
                              s * npar + 5 * J)) {
      if (DEMC && a.demc.z) {
        double g[1];
        demc_form(a, s, 5 * J, npar, g);
        p[0] = g[0];
      } else {
        p[0] = a.params[s * npar + 5 * J];
      }
    }
  }
}

// RESID: also the per-system max Kepler residual.  DEMC: the batch is a
// DE-MC step's proposals (a.demc): formed in the prologue, Metropolis
// decision in the epilogue; plain evaluations contain neither.
template <int J, bool RESID, bool DEMC>
__global__ void __maxnreg__(64)
chi2_mixed_warp_kernel(UniformArgs a, int lg, int tile, int ntiles, float *__restrict__ out,
                       float *__restrict__ resid_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  // everything written by earlier grids in the stream is visible after the
  // wait; the next grid may then start placing its CTAs (it waits likewise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int block = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = 1 << lg;
  const int spr = block >> lg;                   // systems of this CTA
  const WarpLayout L(spr, J, tile, block >> 5);
  PlanetW *pl_s = reinterpret_cast<PlanetW *>(smem + L.pl);
  float *gam_s = reinterpret_cast<float *>(smem + L.gam);
  float4 *obs_s = reinterpret_cast<float4 *>(smem + L.obs);
  float *w_s = reinterpret_cast<float *>(smem + L.w);

  const int64_t sys0 = (int64_t)blockIdx.x * spr;
  const int nitems = spr * (J + 1);
  const int step = G * kChunk;                   // a power of two
  const int nk0 = min(tile, a.n_obs);
  const int npad0 = round_up_pow2(nk0, step);

  // ---- prologue: every global load first ----
  const double t_ref = a.n_obs > 0 ? a.t[0] : a.t0;
  double p[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (tid < nitems) load_item<J, DEMC>(tid, spr, sys0, a, p);
  const bool has0 = tid < nk0 && dbg_ok(a.invalid, tid < a.n_obs, kDbgObs, tid);
  const bool has1 = tid + block < nk0 && dbg_ok(a.invalid, tid + block < a.n_obs, kDbgObs,
                                                tid + block);
  double t0v = 0.0, v0v = 0.0, s0v = 1.0, t1v = 0.0, v1v = 0.0, s1v = 1.0;
  if (has0) { t0v = a.t[tid]; v0v = a.v[tid]; s0v = a.sigma[tid]; }
  if (has1) { t1v = a.t[tid + block]; v1v = a.v[tid + block]; s1v = a.sigma[tid + block]; }

  // the reference time's split, needed by the threads that stage
  Split3 tr3 = {0.0f, 0.0f, 0.0f};
  if (tid < npad0 || ntiles > 1) tr3 = split3(t_ref);
  const float jit2 = d2f(a.jitter2);
  // tau = t - t_ref and v as float pairs, w = 1/(sigma^2 + jitter^2); the
  // padding up to whole chunks has zero weight (and tau = v = 0)
  auto convert = [&](int k, bool real, double t, double v, double sigma) {
    if (!dbg_ok(a.invalid, k < tile, kDbgSmem, k)) return;
    float4 o = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float wk = 0.0f;
    if (real) {
      sub_ds(split3(t), tr3, o.x, o.y);
      split_d(v, o.z, o.w);
      const float sg = d2f(sigma);
      const float var = __fmaf_rn(sg, sg, jit2);
      wk = var > 0.0f ? 1.0f / var : __int_as_float(0x7fc00000);
    }
    obs_s[k] = o;
    w_s[k] = wk;
  };

  if (tid < nitems) setup_item<J>(tid, spr, sys0, a.n_sys, p, t_ref, a.t0, pl_s, gam_s, a.invalid);
  for (int i = tid + block; i < nitems; i += block) {       // more items than threads
    double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    load_item<J, DEMC>(i, spr, sys0, a, q);
    setup_item<J>(i, spr, sys0, a.n_sys, q, t_ref, a.t0, pl_s, gam_s, a.invalid);
  }
  if (tid < npad0) convert(tid, has0, t0v, v0v, s0v);
  if (tid + block < npad0) convert(tid + block, has1, t1v, v1v, s1v);
  for (int k = tid + 2 * block; k < npad0; k += block) {
    const bool real = k < nk0 && dbg_ok(a.invalid, k < a.n_obs, kDbgObs, k);
    convert(k, real, real ? a.t[k] : 0.0, real ? a.v[k] : 0.0, real ? a.sigma[k] : 1.0);
  }
  __syncthreads();

  // ---- the CTA's systems, one per G lanes ----
  int slot = tid >> lg;
  if (!dbg_ok(a.invalid, slot < spr, kDbgSmem, slot)) slot = 0;
  const int c = tid & (G - 1);                   // the thread's place in its system
  const int64_t s = sys0 + slot;
  const PlanetW *q = pl_s + slot * J;
  const float gam = gam_s[slot];
  float poison = 0.0f * gam;                     // NaN for an invalid system
#pragma unroll
  for (int j = 0; j < J; ++j) poison += 0.0f * q[j].f.e;
  Kahan acc = {0.0f, 0.0f};
  float rmax = 0.0f;

  for (int t = 0; t < ntiles; ++t) {
    const int k0 = t * tile;
    const int nk = min(tile, a.n_obs - k0);
    const int npad = round_up_pow2(nk, step);
    if (t > 0) {
      __syncthreads();
      for (int k = tid; k < npad; k += block) {
        const bool real = k < nk && dbg_ok(a.invalid, k0 + k < a.n_obs, kDbgObs, k0 + k);
        convert(k, real, real ? a.t[k0 + k] : 0.0, real ? a.v[k0 + k] : 0.0,
                real ? a.sigma[k0 + k] : 1.0);
      }
      __syncthreads();
    }
    for (int base = c; base < npad; base += step) {
      if (!dbg_ok(a.invalid, base + ((kChunk - 1) << lg) < tile, kDbgSmem, base)) break;
      float th[kChunk], tl[kChunk];
      Kahan V[kChunk];
#pragma unroll
      for (int i = 0; i < kChunk; ++i) {
        const float2 tt = *reinterpret_cast<const float2 *>(obs_s + base + (i << lg));
        th[i] = tt.x;
        tl[i] = tt.y;
        V[i].big = 0.0f;
        V[i].small = 0.0f;
      }
      // two planets per iteration: the second one's constants load while the
      // first one's chains run (full unrolling spills at 64 registers)
#pragma unroll 2
      for (int j = 0; j < J; ++j) {
        const PlanetW qj = q[j];
#pragma unroll
        for (int i = 0; i < kChunk; ++i) {
          const float M = mean_anomaly_mixed(th[i], tl[i], qj.f);
          float sE, cE;
          const float E = kepler_f32_h(M, qj.f.e, qj.m, sE, cE);
          if (RESID) {
            const float r = fabsf((E - M) - qj.f.e * sE);
            rmax = fmaxf(rmax, base + (i << lg) < nk ? r : 0.0f);
          }
          kahan_add(V[i], velocity_h(qj.f, sE, cE));
        }
      }
#pragma unroll
      for (int i = 0; i < kChunk; ++i) {
        const int k = base + (i << lg);
        const float2 vo = *reinterpret_cast<const float2 *>(&obs_s[k].z);
        // residual V - v_obs with the model and the observation as float pairs
        const float r = __fadd_rn(__fsub_rn(V[i].big, vo.x),
                                  __fsub_rn(gam, __fadd_rn(V[i].small, vo.y)));
        kahan_add(acc, w_s[k] * r * r);
      }
    }
  }

  // combine the system's lanes within each of its warps (G a power of two)
  for (int m = (G < 32 ? G : 32) >> 1; m >= 1; m >>= 1) {
    Kahan o = {shfl_xor(acc.big, m), shfl_xor(acc.small, m)};
    kahan_merge(acc, o);
    if (RESID) rmax = fmaxf(rmax, shfl_xor(rmax, m));
  }
  if (G > 32) {
    // then its G / 32 warps, in warp order, through shared memory (lg is
    // the same for the whole CTA, so every thread reaches the barrier)
    float *red_s = reinterpret_cast<float *>(smem + L.red);
    if (lane == 0) {
      red_s[3 * warp] = acc.big;
      red_s[3 * warp + 1] = acc.small;
      red_s[3 * warp + 2] = rmax;
    }
    __syncthreads();
    if (c == 0) {
      for (int w = warp + 1; w < warp + (G >> 5); ++w) {
        if (!dbg_ok(a.invalid, w < (block >> 5), kDbgSmem, w)) break;
        const Kahan o = {red_s[3 * w], red_s[3 * w + 1]};
        kahan_merge(acc, o);
        rmax = fmaxf(rmax, red_s[3 * w + 2]);
      }
    }
  }
  if (c == 0 && s < a.n_sys) {
    const float value = kahan_value(acc) + poison;   // NaN survives n_obs == 0
    out[s] = value;
    note_invalid(a.invalid, value);
    if (RESID) resid_out[s] = rmax;
    // the proposals this CTA formed are visible here after the barrier
    if (DEMC) demc_accept<5 * J + 1>(a, s, value);
  }
}

// Variants: 0 plain, 1 with the Kepler residual, 2 DE-MC step.
template <int J>
const void *warp_kernel_fn(int variant) {
  switch (variant) {
    case 0: return reinterpret_cast<const void *>(chi2_mixed_warp_kernel<J, false, false>);
    case 1: return reinterpret_cast<const void *>(chi2_mixed_warp_kernel<J, true, false>);
    case 2: return reinterpret_cast<const void *>(chi2_mixed_warp_kernel<J, false, true>);
  }
  return nullptr;
}

const void *warp_kernel_for(int J, int variant) {
  switch (J) {
    case 1: return warp_kernel_fn<1>(variant);
    case 2: return warp_kernel_fn<2>(variant);
    case 3: return warp_kernel_fn<3>(variant);
    case 4: return warp_kernel_fn<4>(variant);
    case 5: return warp_kernel_fn<5>(variant);
    case 6: return warp_kernel_fn<6>(variant);
    case 7: return warp_kernel_fn<7>(variant);
    case 8: return warp_kernel_fn<8>(variant);
  }
  return nullptr;
}

// CTAs of the kernel resident per SM (occupancy API), per device, planet
// count, block and shared-memory size; 0 when the shape does not fit.
std::mutex g_occ_mu;
std::map<std::tuple<int, int, int, size_t>, int> g_occ;

int blocks_per_sm(int J, int variant, int block, size_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;                                    // no device: shapes stay valid
  }
  const auto key = std::make_tuple(dev * 16 + J, block, variant, smem);
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
  }
  const void *fn = warp_kernel_for(J, variant);
  int n = 0;
  if (!fn) return 0;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ[key] = n;
  return n;
}

size_t warp_smem(int J, int G, int block, int n_obs) {
  return WarpLayout(block / G, J, warp_obs_tile(n_obs, G), block / 32).total;
}

int log2_lanes(int G) {
  int lg = 3;
  while ((8 << (lg - 3)) < G) ++lg;
  return lg;
}

}  // namespace

bool warp_tile_ok(int G, int block) {
  const bool lanes = G == 8 || G == 16 || G == 32 || G == 64 || G == 128;
  return lanes && block >= 32 && block <= 1024 && !(block & 31) && block % G == 0;
}

int warp_lanes_for(int n_obs) {
  if (n_obs >= 32 * kChunk) return 32;
  if (n_obs >= 16 * kChunk) return 16;
  return 8;
}

bool warp_lanes_fit(int G, int n_obs) { return G == 8 || n_obs >= G * kChunk; }

Tile warp_tile(int64_t n_sys, int n_pl, int n_obs, bool multi_warp) {
  // A grid of one CTA per block / G systems.  When it fits on the device
  // at once, an SM holds at most ceil(CTAs / n_sm) CTAs; otherwise the
  // hardware refills the SMs wave after wave and the load per SM is the
  // total over the SMs.  Pick the shape whose busiest SM carries the least
  // work (warps x 32 / G: systems' worth of lanes); among equals, the one
  // with more warps resident per SM (more latency hidden), then the larger
  // CTA (fewer CTAs share an SM: on the 4096-system batch one CTA of 27
  // warps per SM ran 18.4 us where three of nine ran 20.5 us, with the
  // same 27 systems per SM).  With multi_warp, 32 lanes per system and at
  // least 4 observations per lane at G = 64 or 128, a system split over 2
  // or 4 warps replaces that shape if its load is lower by more than 1 %,
  // or within 1 % in fewer waves, or in as many waves with at least as many
  // warps resident (then the larger CTA).  Back to back on n_obs = 256
  // (us per launch): 256 systems 6.51 -> 5.24, 512: 6.65 -> 5.41, 1024:
  // 7.44 -> 6.75, 2048: 9.52 -> 9.23; the 4096-system batch keeps its single
  // wave of 27-warp CTAs (13.9 against 17.4 for 64 lanes in 28-warp CTAs).
  const int G0 = warp_lanes_for(n_obs);
  const int64_t n_sm = sm_count();
  Tile best{G0, 8 * 32, 0, 3};
  double best_load = 1e300;
  int64_t best_warps = 0, best_waves = 0;
  for (int G : {G0, 64, 128}) {
    const bool multi = G > 32;
    if (multi && (!multi_warp || G0 != 32 || !warp_lanes_fit(G, n_obs))) continue;
    for (int W = 4; W <= 32; ++W) {
      const int block = 32 * W;
      if (block % G) continue;
      const int occ = blocks_per_sm(n_pl, 0, block, warp_smem(n_pl, G, block, n_obs));
      if (occ < 1) continue;
      const int64_t spc = block / G;                 // systems per CTA
      const int64_t ctas = (n_sys + spc - 1) / spc;
      const int64_t cap = n_sm * occ;
      const int64_t per_sm = (ctas + n_sm - 1) / n_sm;
      const int64_t resident = ctas <= cap ? per_sm : occ;
      const double load = (double)per_sm * W * 32.0 / G;
      const int64_t warps = resident * W;
      const int64_t waves = (ctas + cap - 1) / cap;
      bool take;
      if (!multi) {
        const bool tie = load <= best_load * (1.0 + 1e-9);
        take = load < best_load * (1.0 - 1e-9) || (tie && warps >= best_warps);
      } else {
        const bool near = load <= best_load * 1.01;
        take = load < best_load * 0.99 ||
               (near && (waves < best_waves || (waves == best_waves && warps >= best_warps)));
      }
      if (take) {
        best_load = load;
        best_warps = warps;
        best_waves = waves;
        best = Tile{G, block, 0, 3};
      }
    }
  }
  best.obs_tile = warp_obs_tile(n_obs, best.G);
  return best;
}

cudaError_t launch_chi2_mixed_warp(const UniformArgs &a, const Tile &tile, float *out,
                                   float *resid, cudaStream_t st) {
  const int G = tile.G, block = tile.block;
  if (!warp_tile_ok(G, block)) return cudaErrorInvalidValue;
  // a DE-MC step reports no residual (the DE-MC entry point has none)
  const int variant = a.demc.states ? 2 : (resid != nullptr ? 1 : 0);
  if (variant == 2) resid = nullptr;
  const void *fn = warp_kernel_for(a.n_pl, variant);
  if (!fn) return cudaErrorInvalidValue;
  const int spr = block / G;
  const int obs_tile = warp_obs_tile(a.n_obs, G);
  const size_t smem = WarpLayout(spr, a.n_pl, obs_tile, block / 32).total;
  if (blocks_per_sm(a.n_pl, variant, block, smem) < 1) return cudaErrorInvalidConfiguration;
  const int64_t ctas = (a.n_sys + spr - 1) / spr;
  if (ctas > 0x7fffffff) return cudaErrorInvalidConfiguration;
  UniformArgs args = a;
  int lg = log2_lanes(G), tl = obs_tile, nt = (a.n_obs + obs_tile - 1) / obs_tile;
  void *params[] = {&args, &lg, &tl, &nt, &out, &resid};
  // programmatic stream serialisation (the kernel's griddepcontrol.wait
  // keeps it ordered after the grids before it), not under stream capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return cudaGetLastError();
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelExC(&cfg, fn, params);
}

}  // namespace kc
