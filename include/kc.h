/*
 * kc.h -- C ABI of the GB300 batched Keplerian radial-velocity chi-square
 * library (libkc.so).
 *
 * The library evaluates, for huge batches of multi-planet Keplerian models,
 * the goodness of fit against one star's Doppler observations, as set out in
 * Ford (2008), "Parallel Algorithm for Solving Kepler's Equation on Graphics
 * Processing Units":
 *
 *   M_jk  = 2 pi frac((t_k - t0)/P_j) + M0_j              (Eqs. 4 and 6)
 *   E_jk  - e_j sin E_jk = M_jk                            (Eq. 1; the paper
 *                                                           iterates Danby's
 *                                                           step, Eqs. 7-10;
 *                                                           here a fixed-count
 *                                                           solve to the same
 *                                                           root, Sec. 4.3)
 *   v_jk  = K_j [cos(omega_j + f_jk) + e_j cos omega_j]    (Eq. 3)
 *   V_k   = gamma + sum_j v_jk                             (Eq. 2)
 *   chi2  = sum_k (V_k - v_k)^2 / (sigma_jit^2 + sigma_k^2) (Eq. 5)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Parameter layout.  One system is 5*n_pl + 1 doubles: (P, K, e, omega,
 *    M0) for each planet in turn (the five per-planet parameters of
 *    Sec. 4.1), then the systemic offset gamma.  Units: days, m/s, radians.
 *    A batch is row-major [n_sys][5*n_pl + 1].
 *  - Observations t, v_obs, sigma are [n_obs] doubles shared by every system
 *    (Sec. 4.1: "constants to be used for evaluating all models").
 *  - All array pointers are DEVICE pointers, owned by the caller, naturally
 *    aligned for their type.  The library never frees or retains them.
 *  - Every call is asynchronous on `stream` (NULL = the legacy default
 *    stream).  Host-detectable errors (NULL pointers, sizes out of range)
 *    return KC_ERR_ARG before anything is launched; a failed launch returns
 *    KC_ERR_CUDA.  kc_last_error() gives a message for the calling thread.
 *  - Physically invalid parameters (P <= 0, e outside [0, 1), non-finite
 *    values) give NaN for that system; a non-positive or NaN variance gives
 *    NaN for every system, an infinite one a zero weight.  Nothing traps:
 *    every device loop has a fixed trip count.  Each system whose result
 *    comes out NaN also adds one to a per-device counter read (and reset)
 *    by kc_last_device_error.
 *  - n_sys == 0 is a no-op.  n_obs == 0 gives chi2 = 0 (NaN if invalid).
 *  - Calls are thread-safe; concurrent calls on different streams do not
 *    share device memory, with one exception: every call of
 *    kc_chi2_eval_mixed_noalloc uses the same fixed array (see its
 *    declaration), so its calls must not overlap on the device.
 */
#ifndef KC_H
#define KC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *kc_stream;

typedef enum kc_status {
    KC_OK = 0,
    KC_ERR_ARG = 1,          /* bad pointer, size or mode                    */
    KC_ERR_CUDA = 2,         /* a CUDA call or kernel launch failed          */
    KC_ERR_NOMEM = 3,        /* a plan could not allocate its device memory  */
    KC_ERR_UNSUPPORTED = 4   /* no sm_103a device / feature not available    */
} kc_status;

/* Arithmetic of the path (Sec. 5, "Mixed Precision Arithmetic"):
 *  KC_FP64  - every step in double precision.
 *  KC_MIXED - the phase frac((t-t0)/P) in pair-of-single (double-single)
 *             arithmetic, Kepler's equation, the velocities and the residuals
 *             in single precision, with compensated (Kahan) sums for the
 *             planet velocities and for chi2 (Sec. 4.4).
 *  KC_FP32  - every step in single precision, observation times and periods
 *             included: Sec. 5's pure single-precision variant, whose worst
 *             chi2 error the paper puts at one part in ten.  Accepted by
 *             kc_chi2_eval_ex only (float output), for precision comparisons;
 *             not an accurate path for absolute times t/P >> 1e3. */
typedef enum kc_mode { KC_FP64 = 0, KC_MIXED = 1, KC_FP32 = 2 } kc_mode;

#define KC_MAX_PLANETS 8        /* n_pl range: 1 .. KC_MAX_PLANETS           */
#define KC_MAX_OBS (1 << 24)    /* n_obs range: 0 .. KC_MAX_OBS              */

/* ------------------------------------------------------------- chi-square */

/* FP64 chi2 of n_sys systems with epoch t0 = 0 and no jitter (the paper's
 * setting, Eq. 4 with t=0 as epoch and sigma_j = 0 in Eq. 5).
 *   params [n_sys][5*n_pl+1], t/v_obs/sigma [n_obs], out [n_sys] (double). */
kc_status kc_chi2_eval(const double *params, const double *t,
                       const double *v_obs, const double *sigma,
                       int64_t n_sys, int32_t n_pl, int32_t n_obs,
                       double *out, kc_stream stream);

/* Mixed-precision chi2 (KC_MIXED arithmetic), t0 = 0, no jitter.
 *   out [n_sys] (float).  max_kepler_resid [n_sys] (float, may be NULL):
 *   per system, max over its (planet, observation) pairs of
 *   |E - e sin E - M| evaluated in single precision at the returned E. */
kc_status kc_chi2_eval_mixed(const double *params, const double *t,
                             const double *v_obs, const double *sigma,
                             int64_t n_sys, int32_t n_pl, int32_t n_obs,
                             float *out, float *max_kepler_resid,
                             kc_stream stream);

/* General form: epoch t0 of M0 (Eq. 4) and jitter sigma_j (Eq. 5).
 * out is double* for KC_FP64 and float* for KC_MIXED.  max_kepler_resid
 * (float [n_sys], may be NULL) is filled in either mode.
 * kc_chi2_eval(...) == kc_chi2_eval_ex(..., 0.0, 0.0, KC_FP64, out, NULL, s). */
kc_status kc_chi2_eval_ex(const double *params, const double *t,
                          const double *v_obs, const double *sigma,
                          int64_t n_sys, int32_t n_pl, int32_t n_obs,
                          double t0, double jitter, kc_mode mode, void *out,
                          float *max_kepler_resid, kc_stream stream);

/* Gradient of chi2 with respect to all 5*n_pl+1 parameters of every system,
 * by a hand-written adjoint (Sec. 6 suggests evaluating partial derivatives
 * in parallel): E is recomputed, not stored, and Kepler's equation is
 * differentiated implicitly, dE = (dM + sin E de)/(1 - e cos E);
 * dM/dP = -2 pi (t - t0)/P^2 (jumps of frac() ignored).
 *   chi2_out [n_sys] (may be NULL), grad_out [n_sys][5*n_pl+1]; both double
 *   for KC_FP64 and float for KC_MIXED. */
kc_status kc_chi2_grad(const double *params, const double *t,
                       const double *v_obs, const double *sigma,
                       int64_t n_sys, int32_t n_pl, int32_t n_obs, double t0,
                       double jitter, kc_mode mode, void *chi2_out,
                       void *grad_out, kc_stream stream);

/* Gauss-Newton normal matrix (derivatives for least-squares refinement,
 * which Sec. 6 lists as future work): for every system
 *   H = sum_k w_k J_k J_k^T,  J_k = dV_k/dtheta over its n = 5*n_pl + 1
 *   parameters, w_k = 1/(sigma_k^2 + jitter^2),
 * the matrix of a Levenberg-Marquardt step (the chi2 Hessian is 2H plus a
 * term proportional to the residuals), together with chi2 and its gradient
 * from the same pass (chi2_out and grad_out may be NULL; grad_out as in
 * kc_chi2_grad).  jtj_out: [n_sys][n (n + 1)/2], the upper triangle packed
 * row by row (H[0][0..n-1], H[1][1..n-1], ...); float for KC_MIXED, double
 * for KC_FP64.  KC_MIXED forms the per-batch update H += U^T U (U: 32
 * observations x n, rows sqrt(w_k) J_k) on the tensor cores with TF32
 * inputs split in two (error about 1e-6 of sqrt(H_pp H_qq)), by warp-level
 * mma.sync or by tcgen05 MMAs with the accumulator in tensor memory, as
 * the tile table's KC_KERNEL_GN entry says.  Invalid systems give NaN in
 * all their outputs.  Errors as kc_chi2_grad. */
kc_status kc_chi2_gauss_newton(const double *params, const double *t,
                               const double *v_obs, const double *sigma,
                               int64_t n_sys, int32_t n_pl, int32_t n_obs,
                               double t0, double jitter, kc_mode mode,
                               void *chi2_out, void *grad_out, void *jtj_out,
                               kc_stream stream);

/* Free jitter: each system carries its own jitter sigma_j after gamma
 * (params [n_sys][5*n_pl + 2]) and the statistic is the Gaussian negative
 * log-likelihood whose exponent is Eq. 5's chi2 with that sigma_j,
 *   nll = 1/2 sum_k [ r_k^2/(sigma_k^2 + sigma_j^2)
 *                     + ln(2 pi (sigma_k^2 + sigma_j^2)) ],
 * which, unlike chi2, has a finite optimum in sigma_j (the paper fixes
 * sigma_j = 0 and keeps it as a variable, Sec. 2.2).  out [n_sys]: double
 * for KC_FP64, float for KC_MIXED.  A non-positive or NaN variance makes the
 * system NaN; an infinite one makes its nll infinite. */
kc_status kc_nll_eval(const double *params, const double *t,
                      const double *v_obs, const double *sigma, int64_t n_sys,
                      int32_t n_pl, int32_t n_obs, double t0, kc_mode mode,
                      void *out, kc_stream stream);

/* nll and its gradient with respect to all 5*n_pl + 2 parameters (adjoint
 * as kc_chi2_grad; d nll / d sigma_j = sigma_j sum_k w_k (1 - w_k r_k^2)
 * with w_k = 1/(sigma_k^2 + sigma_j^2)).  nll_out may be NULL. */
kc_status kc_nll_grad(const double *params, const double *t,
                      const double *v_obs, const double *sigma, int64_t n_sys,
                      int32_t n_pl, int32_t n_obs, double t0, kc_mode mode,
                      void *nll_out, void *grad_out, kc_stream stream);

/* Allocation-free form of kc_chi2_eval_mixed (with t0 and jitter as in
 * kc_chi2_eval_ex).  The paper has no counterpart: this exists for callers
 * that must not allocate device memory while they evaluate (all memory
 * reserved up front, or no allocator calls allowed at that point).  It runs
 * the two-pass variant of the mixed kernel with its intermediate data in a
 * fixed array of KC_NOALLOC_SCRATCH_BYTES compiled into libkc.so, which every
 * GPU that loads the library keeps until the process exits; the call itself
 * never calls cudaMalloc, cudaFree or a memory pool.
 *  - Limit: 32 B per (system, planet), 4 B per system and 20 B per
 *    observation (each part rounded up to 256 B) must fit in the array,
 *    e.g. 4096 systems x 4 planets x 256 observations uses ~540 KB.  Larger
 *    problems return KC_ERR_ARG with the byte counts, before any launch.
 *  - The first call on a device looks up the array's device address (once
 *    per device); make that first call before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents:
 *    calls that overlap on the GPU (different streams, or other host
 *    threads) race and must be serialised by the caller.  Nothing in the
 *    array needs to start at zero: each call writes all it reads.
 *  - Results equal kc_chi2_eval_mixed's within rounding (same arithmetic,
 *    possibly a different summation order). */
#define KC_NOALLOC_SCRATCH_BYTES (4u << 20)

kc_status kc_chi2_eval_mixed_noalloc(const double *params, const double *t,
                                     const double *v_obs, const double *sigma,
                                     int64_t n_sys, int32_t n_pl, int32_t n_obs,
                                     double t0, double jitter, float *out,
                                     float *max_kepler_resid, kc_stream stream);

/* --------------------------------------------------------- DE-MC step */

/* One step of differential-evolution MCMC (ter Braak 2006; the population
 * MCMC the paper proposes to drive the evaluator, Sec. 6) for chains
 * first .. first+count-1 of a population of n_chains parameter vectors
 * (states [n_chains][5*n_pl+1], device, updated in place; chi2 [n_chains]
 * their current chi2, double for KC_FP64, float for KC_MIXED).  Chain
 * i = first + c proposes
 *   x*_p = x_ip + gamma (x_r1,p - x_r2,p) + (eps_scale[p] |x_ip|) z[c][p]
 * (each operation rounded in that order, no fused operations), evaluates
 * chi2(x*) with the kernels of kc_chi2_eval_ex (epoch t0, jitter, mode) and
 * accepts iff ln u[c][0] < -(chi2(x*) - chi2(x_i))/2 (flat prior; invalid
 * parameters give NaN chi2 and are rejected; u = 0 accepts any finite
 * chi2).  The random numbers are inputs: z [count][5*n_pl+1] standard
 * normal draws, u [count][3] uniform draws in [0, 1).  The partners are two
 * distinct chains of the range partner_first .. partner_first+m-1
 * (m = partner_count >= 2), uniform over ordered pairs:
 *   k1 = floor(u[c][1] m) clamped to 0 .. m - 1,
 *   k2 = floor(u[c][2] (m - 1)) clamped to 0 .. m - 2, k2 += (k2 >= k1),
 *   r1 = partner_first + k1, r2 = partner_first + k2
 * (in double; a NaN draw counts as 0, so no draw indexes outside the
 * range).  The partner range must lie inside the population and not
 * overlap the updated range (their states stay fixed during the step, which
 * keeps detailed balance), else KC_ERR_ARG.  eps_scale [5*n_pl+1] (device)
 * scales the perturbation per parameter (0 with equal values in every chain
 * holds a parameter fixed).  The caller supplies the workspaces
 * proposals [count][5*n_pl+1] and chi2_prop [count] (chi2's type);
 * accepted [count] (may be NULL) receives 1/0. */
kc_status kc_demcmc_step(double *states, void *chi2, int64_t n_chains,
                         int32_t n_pl, const double *t, const double *v_obs,
                         const double *sigma, int32_t n_obs, double t0,
                         double jitter, kc_mode mode, int64_t first,
                         int64_t count, int64_t partner_first,
                         int64_t partner_count, double gamma,
                         const double *eps_scale, const double *z,
                         const double *u, double *proposals,
                         void *chi2_prop, int32_t *accepted, kc_stream stream);

/* -------------------------------------------------------- model, Kepler */

/* FP64 model velocities V(t_k) = gamma + sum_j v_j(t_k) (Eq. 2):
 *   v_out [n_sys][n_obs] (double).  Used to synthesise observations and
 *   for predictive distributions (Sec. 6). */
kc_status kc_rv_predict(const double *params, const double *t, int64_t n_sys,
                        int32_t n_pl, int32_t n_obs, double t0, double *v_out,
                        kc_stream stream);

/* FP64 model velocities of a ragged batch (device arrays): system s has
 * n_pl[s] planets at params[par_off[s]] and its own times
 * t[obs_off[s] .. obs_off[s+1]); v_out has the layout of t. */
kc_status kc_rv_predict_ragged(const double *params, const int64_t *par_off,
                               const int32_t *n_pl, const double *t,
                               const int64_t *obs_off, int64_t n_sys, double t0,
                               double *v_out, kc_stream stream);

/* Elementwise Kepler solve with the same device solver the chi2 kernels use
 * (Sec. 4.3): E_out[i] with E - e sin E = M for M[i] in any range and
 * 0 <= e[i] < 1.  KC_FP64: M, e, E_out are double.  KC_MIXED: float.
 * E_out is reduced to the branch of M reduced to [-pi, pi]. */
kc_status kc_kepler_solve(const void *M, const void *e, int64_t n,
                          kc_mode mode, void *E_out, kc_stream stream);

/* ------------------------------------------------------------- ragged */

/* A plan for a ragged batch: systems with their own planet count and their
 * own observations, evaluated by one persistent kernel that takes whole
 * systems from a device work queue (longest first) and is replayed as a CUDA
 * graph.  The observations are fixed for the plan (as the paper treats them,
 * Sec. 4.1); the parameters change from run to run.
 *   obs_off [n_sys+1] host int64: system s owns observations
 *                     obs_off[s] .. obs_off[s+1] (obs_off[0] == 0,
 *                     non-decreasing; empty systems allowed).
 *   n_pl    [n_sys]   host int32 in 1 .. KC_MAX_PLANETS.
 * Parameters are packed: system s's 5*n_pl[s]+1 values (same layout as the
 * uniform calls) follow those of system s-1.  The plan copies the
 * descriptors to the current device and owns that memory, the converted
 * observations and its work queue until kc_plan_destroy.  Creation
 * allocates and synchronises; KC_ERR_NOMEM if the device is out of memory. */
typedef struct kc_plan kc_plan;

kc_status kc_plan_create_ragged(kc_plan **plan, const int64_t *obs_off,
                                const int32_t *n_pl, int64_t n_sys, double t0,
                                double jitter, kc_mode mode, int want_grad);

/* Total number of packed parameters (sum of 5*n_pl[s]+1) and of
 * observations of the plan. */
kc_status kc_plan_sizes(const kc_plan *plan, int64_t *n_params,
                        int64_t *n_obs);

/* Converts the observations (device [n_obs] doubles t, v_obs, sigma) into
 * the plan's own arrays, on `stream`.  Must precede kc_plan_run; later runs
 * on other streams must be ordered after it by the caller. */
kc_status kc_plan_set_observations(kc_plan *plan, const double *t,
                                   const double *v_obs, const double *sigma,
                                   kc_stream stream);

/* chi2_out [n_sys] (float for KC_MIXED, double for KC_FP64) and, for a plan
 * created with want_grad, grad_out laid out like the packed parameters
 * (same type), else NULL.  The first run captures the queue reset and the
 * kernel into a CUDA graph (on a stream private to the plan); every run
 * launches that graph on `stream`, retargeted to the given pointers.  When
 * `stream` is itself being captured the two operations are recorded into
 * the caller's graph instead.  Every stream a plan runs on gets its own work
 * queue and graph (up to 64 streams per plan, kept until kc_plan_destroy;
 * KC_ERR_UNSUPPORTED beyond), so runs on different streams may overlap on
 * the device; runs on one stream are ordered by it. */
kc_status kc_plan_run(kc_plan *plan, const double *params, void *chi2_out,
                      void *grad_out, kc_stream stream);

/* Times persistent launch shapes (threads per CTA x CTAs per SM) on these
 * parameters and keeps the fastest for later runs.  Blocking; not during
 * stream capture.  Outputs are overwritten.  *block / *ctas_per_sm (may
 * be NULL) receive the choice. */
kc_status kc_plan_autotune(kc_plan *plan, const double *params, void *chi2_out,
                           void *grad_out, int32_t *block, int32_t *ctas_per_sm,
                           kc_stream stream);

void kc_plan_destroy(kc_plan *plan);

/* ------------------------------------------------------------ tiling */

/* Launch shape of the uniform-batch kernels: each system is handled by
 * threads_per_system consecutive threads (1..block and a divisor of block;
 * a power of two except for the mixed chi2 kernel; at most 32 for the
 * gradient kernel), `block` threads per CTA (32..256, a multiple of 32;
 * up to 1024 for split = 3).  split (mixed chi2 only) selects a
 * two-pass variant for small batches: a preparation pass first writes every
 * per-(system, planet) constant and the converted observations to
 * stream-ordered scratch from a library memory pool, then the main kernel
 * (programmatic dependent launch) only reads them.  split = 1: CTAs as
 * above.  split = 2: one warp per (system, chunk of observations);
 * threads_per_system = 32 x chunks (32..1024), any block; the last warp of a
 * system merges the chunks' partial sums in chunk order.  While the stream is
 * being captured into a CUDA graph the split variants are replaced by the
 * fused kernel (no allocation inside a graph).
 * split = 3 (mixed chi2 only): the warp-per-system kernel,
 * threads_per_system = 8, 16, 32, 64 or 128 lanes per system (64 and 128:
 * the system's observations split over two or four warps, whose sums are
 * combined through shared memory), block a multiple of 32 and of
 * threads_per_system, up to 1024; one CTA per block / threads_per_system
 * systems.  Allocates nothing, so it also runs under stream capture.  With
 * no tuned entry the mixed chi2 (and the mixed DE-MC step) uses this
 * variant with the lanes per system and block that spread the work most
 * evenly over the SMs. */
typedef struct kc_tile {
    int32_t threads_per_system;
    int32_t block;
    int32_t split;
} kc_tile;

/* KC_KERNEL_GN (KC_MIXED only): the Gauss-Newton kernel of
 * kc_chi2_gauss_newton, one warp per system and four per CTA
 * (threads_per_system = 32, block = 128); split chooses how it adds U^T U:
 * 0 = warp-level mma.sync (TF32), 32 observations per batch; 4 = tcgen05
 * MMAs for the CTA's four systems stacked in one M = 64, N = 64 tile (one
 * issuing thread, two accumulators in 128 TMEM columns per CTA), 64
 * observations per batch, n_pl <= 3 only.  Without a tuned entry split 4 is used for
 * n_pl <= 3 and split 0 above. */
typedef enum kc_kernel {
    KC_KERNEL_CHI2 = 0,
    KC_KERNEL_GRAD = 1,
    KC_KERNEL_GN = 2
} kc_kernel;

/* Tiles are looked up by (kernel, mode, n_pl, power-of-two bucket of n_sys,
 * power-of-two bucket of n_obs, SM count of the current device) in a
 * process-wide table; a missing entry uses a built-in heuristic.  kc_set_tile (tile == NULL removes the entry)
 * and kc_get_tile (the tile that would be used) act on that table. */
kc_status kc_set_tile(kc_kernel kernel, kc_mode mode, int64_t n_sys,
                      int32_t n_pl, int32_t n_obs, const kc_tile *tile);
kc_status kc_get_tile(kc_kernel kernel, kc_mode mode, int64_t n_sys,
                      int32_t n_pl, int32_t n_obs, kc_tile *tile);

/* Autotuner: times every admissible tile on the given problem (device
 * arrays as for kc_chi2_eval_ex / kc_chi2_grad / kc_chi2_gauss_newton;
 * t0 = 0, no jitter; per launch, the mean of four launches back to back,
 * the best of three), stores the fastest in the table (the built-in tile
 * unless another is at least 1 % faster, so that shapes within timing
 * noise of each other do not trade places from run to run) and returns it
 * in *best (and its time in *best_ms, may be NULL).  Blocking: synchronises `stream`; must not be
 * called while the stream is being captured.  Allocates and frees its own
 * output buffers (stream-ordered). */
kc_status kc_autotune(const double *params, const double *t,
                      const double *v_obs, const double *sigma, int64_t n_sys,
                      int32_t n_pl, int32_t n_obs, kc_kernel kernel,
                      kc_mode mode, kc_tile *best, float *best_ms,
                      kc_stream stream);

/* --------------------------------------------------------------- misc */

const char *kc_status_string(kc_status status);

/* Detail of the calling thread's last non-OK status ("" if none). */
const char *kc_last_error(void);

/* Number of systems whose result came out NaN (invalid parameters or
 * observations, convention above) in every evaluation on the current device
 * since the previous call, then resets that count to zero.  The paper has no
 * counterpart (its kernels return chi2 only); the count lets a caller notice
 * invalid models without scanning the outputs.  Synchronises the current
 * device first, so an asynchronous fault of an earlier launch is reported
 * here as KC_ERR_CUDA (with *n_invalid = 0).  Evaluations made by
 * kc_demcmc_step on its proposals are counted too.  n_invalid must not be
 * NULL (KC_ERR_ARG). */
kc_status kc_last_device_error(int64_t *n_invalid);

/* Measured throughput of one arithmetic pipe of the current GPU, in
 * operations per SM per SM-clock cycle: pipe 0 = FP32 FMA, 1 = FP64 FMA.
 * The roofline denominators of the two paths (the paper quotes none; the
 * FP64 rate of this part is 1/64 of its FP32 rate).  Runs one CTA of 1024
 * threads per SM with eight independent FMA chains per thread and divides
 * the FMAs each CTA executed by its SM-clock cycles (clock64), so the result
 * does not depend on the clock frequency.  Blocking: synchronises `stream`;
 * allocates and frees its own scratch.  KC_ERR_ARG for another pipe or a
 * NULL result pointer. */
kc_status kc_measure_pipe_rate(int32_t pipe, double *ops_per_sm_clock, kc_stream stream);

/* First failed device index check of a KC_DEBUG build of the library
 * (compiled with -DKC_DEBUG; the paper has no counterpart: it stands in for
 * a memory checker).  Such a build checks, in its kernels, every index that
 * reaches memory through caller data or launch arithmetic (parameter and
 * observation indices, shared-memory slots, a ragged plan's queue entries,
 * planet counts and offsets); a failed check skips its access or substitutes
 * an index known to be in range, so nothing traps or faults.  *word
 * receives the first failure since the previous call on the current device
 * (bit 63 set, site in bits 48-55, the low 48 bits of the index; zero if
 * none) and the word is reset.  Synchronises the device.  A normal build
 * returns KC_ERR_UNSUPPORTED with *word = 0.  KC_ERR_ARG for NULL. */
kc_status kc_debug_word(uint64_t *word);

/* Library version as 10000*major + 100*minor + patch. */
int32_t kc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KC_H */
