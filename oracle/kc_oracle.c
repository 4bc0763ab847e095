/*
 * kc_oracle.c -- FP64 CPU oracle for the batched Keplerian radial-velocity
 * chi-square of Ford (2008), "Parallel Algorithm for Solving Kepler's Equation
 * on Graphics Processing Units".
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything here is the plain definition of the quantity, in double
 * precision, written for a reader to check against the paper by eye:
 *
 *   mean anomaly     M = 2*pi*frac((t - t0)/P) + M0         (Eqs. 4 and 6)
 *   Kepler's eq.     E - e sin E = M                         (Eq. 1, Sec. 4.3)
 *   true anomaly     f = 2 atan2(sqrt(1+e) sin(E/2), sqrt(1-e) cos(E/2))
 *   velocity         v = K [cos(omega + f) + e cos(omega)]   (Eq. 3, standard
 *                                                            convention)
 *   model            V(t_k) = gamma + sum_j v_j(t_k)         (Eq. 2)
 *   chi-square       chi2 = sum_k (V(t_k) - v_k)^2 / (sigma_j^2 + sigma_k^2)
 *                                                            (Eq. 5)
 *
 * Readings taken where the paper is ambiguous (each also listed in the design
 * notes): +M0 as in Eq. 4 (Eq. 6 prints -M0); the velocity in
 * the K[cos(omega+f) + e cos(omega)] form, because Eq. 3's printed prefactor
 * K' = K/sqrt(1-e^2) does not match its bracket; a per-system offset gamma
 * appended after the planets; epoch t0 as an argument (the paper fixes t=0).
 *
 * Kepler's equation has a unique root for 0 <= e < 1 (f' = 1 - e cos E > 0),
 * bracketed by [M - e, M + e] because |E - M| = e |sin E| <= e.  The oracle
 * finds it with Newton steps kept inside that bracket (bisection when a step
 * leaves it) until the iterate stops moving: the definition of E to FP64
 * rounding, not the paper's fixed-count Danby iteration.
 *
 * Sums over observations use Neumaier's compensated summation (an
 * improvement of the Kahan summation the paper uses in Sec. 4.4).
 *
 * Parameter layout (one system): (P, K, e, omega, M0) for each planet j, then
 * gamma; 5*n_pl + 1 doubles.  Invalid parameters (P <= 0, e outside [0,1),
 * non-finite values) or a non-positive (or NaN) variance give NaN for that
 * system; an infinite variance is a zero weight.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC
 * (no -ffast-math: the compensated sums need IEEE semantics).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KCO_TWO_PI 6.28318530717958647692528676655900577

/* ---------------------------------------------------------------- threads */

void kco_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int kco_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------- Neumaier summing */

typedef struct { double s, c; } kco_sum;

static void kco_sum_add(kco_sum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}

static double kco_sum_value(const kco_sum *a) { return a->s + a->c; }

/* --------------------------------------------------------------- Eqs. 4, 6 */

/* Mean anomaly of a planet with period P and mean anomaly M0 at epoch t0,
 * at time t, reduced to [-pi, pi].  frac((t-t0)/P) is formed as
 * fmod(t-t0, P)/P: fmod is exact in IEEE arithmetic, so the phase carries a
 * single rounding even when (t-t0)/P is of order 1e6 (the precision problem
 * Sec. 5, 'Mixed Precision Arithmetic', describes). */
double kco_mean_anomaly(double t, double t0, double P, double M0)
{
    double phase = fmod(t - t0, P) / P;          /* in (-1, 1) cycles   */
    double cyc = phase + M0 / KCO_TWO_PI;        /* total, in cycles    */
    cyc -= floor(cyc + 0.5);                     /* to [-1/2, 1/2)      */
    return KCO_TWO_PI * cyc;
}

/* ------------------------------------------------------------- Eq. 1, 4.3 */

/* Eccentric anomaly E with E - e sin E = M, for 0 <= e < 1.  *n_iter (if not
 * NULL) receives the number of steps taken. */
double kco_kepler_E(double M, double e, int *n_iter)
{
    double lo = M - e, hi = M + e;
    /* the paper's starting guess (Sec. 4.3); it lies inside the bracket */
    double E = M + 0.85 * e * (sin(M) >= 0.0 ? 1.0 : -1.0);
    int it = 0;
    if (e == 0.0) { if (n_iter) *n_iter = 0; return M; }
    if (!(E > lo && E < hi)) E = 0.5 * (lo + hi);
    for (it = 1; it <= 200; ++it) {
        double f = E - e * sin(E) - M;
        double En;
        if (f == 0.0) break;
        if (f < 0.0) lo = E; else hi = E;       /* root stays in [lo, hi] */
        En = E - f / (1.0 - e * cos(E));        /* Newton step            */
        if (!(En > lo && En < hi)) En = 0.5 * (lo + hi);   /* bisect     */
        if (En == E) break;
        E = En;
    }
    if (n_iter) *n_iter = it;
    return E;
}

/* True anomaly from the eccentric anomaly (standard half-angle relation). */
double kco_true_anomaly(double E, double e)
{
    return 2.0 * atan2(sqrt(1.0 + e) * sin(0.5 * E), sqrt(1.0 - e) * cos(0.5 * E));
}

/* ------------------------------------------------------------------ Eq. 3 */

static int kco_planet_valid(const double *p)
{
    double P = p[0], K = p[1], e = p[2], w = p[3], M0 = p[4];
    return isfinite(P) && P > 0.0 && isfinite(K) && isfinite(e) &&
           e >= 0.0 && e < 1.0 && isfinite(w) && isfinite(M0);
}

/* Radial velocity of one planet p = (P, K, e, omega, M0) at time t. */
double kco_planet_velocity(const double *p, double t, double t0)
{
    double P = p[0], K = p[1], e = p[2], w = p[3], M0 = p[4];
    double M = kco_mean_anomaly(t, t0, P, M0);
    double E = kco_kepler_E(M, e, NULL);
    double f = kco_true_anomaly(E, e);
    return K * (cos(w + f) + e * cos(w));
}

/* Partial derivatives of one planet's velocity with respect to
 * (P, K, e, omega, M0), by the chain rule through Kepler's equation:
 *   dE/dM = 1/D,  dE/de|M = sin E / D,        D = 1 - e cos E
 *   df/dE = beta/D,  df/de|E = sin E/(beta D),  beta = sqrt(1 - e^2)
 *   dM/dM0 = 1,  dM/dP = -2 pi (t - t0)/P^2   (jumps of frac() ignored). */
static double kco_planet_velocity_grad(const double *p, double t, double t0,
                                       double g[5])
{
    double P = p[0], K = p[1], e = p[2], w = p[3], M0 = p[4];
    double M = kco_mean_anomaly(t, t0, P, M0);
    double E = kco_kepler_E(M, e, NULL);
    double f = kco_true_anomaly(E, e);
    double D = 1.0 - e * cos(E);
    double beta = sqrt((1.0 - e) * (1.0 + e));
    double c_wf = cos(w + f), s_wf = sin(w + f);
    double dv_df = -K * s_wf;
    double df_dE = beta / D;
    double dv_dM = dv_df * df_dE / D;
    double df_de = sin(E) / (beta * D) + df_dE * sin(E) / D;
    g[0] = dv_dM * (-KCO_TWO_PI * (t - t0) / (P * P));       /* dv/dP     */
    g[1] = c_wf + e * cos(w);                                /* dv/dK     */
    g[2] = K * cos(w) + dv_df * df_de;                       /* dv/de     */
    g[3] = -K * (s_wf + e * sin(w));                         /* dv/domega */
    g[4] = dv_dM;                                            /* dv/dM0    */
    return K * (c_wf + e * cos(w));
}

/* ------------------------------------------------------- one system, Eq.5 */

/* chi-square of one system (and, when grad != NULL, its gradient with
 * respect to the 5*n_pl + 1 parameters; when gabs != NULL also the sum over
 * observations of the absolute value of each observation's term of the
 * gradient, the scale of the cancellation in each gradient sum). */
static double kco_system(const double *par, int n_pl, const double *t,
                         const double *v, const double *sigma, int64_t n_obs,
                         double t0, double jitter, double *grad, double *gabs)
{
    int n_par = 5 * n_pl + 1;
    double gamma = par[5 * n_pl];
    kco_sum chi2 = {0.0, 0.0};
    kco_sum gsum[5 * 16 + 1];
    int j, q;
    int64_t k;
    int valid = isfinite(gamma);
    for (j = 0; j < n_pl; ++j) valid = valid && kco_planet_valid(par + 5 * j);
    for (q = 0; q < n_par; ++q) { gsum[q].s = 0.0; gsum[q].c = 0.0; }
    if (gabs) for (q = 0; q < n_par; ++q) gabs[q] = 0.0;
    if (!valid) {
        if (grad) for (q = 0; q < n_par; ++q) grad[q] = NAN;
        if (gabs) for (q = 0; q < n_par; ++q) gabs[q] = NAN;
        return NAN;
    }
    for (k = 0; k < n_obs; ++k) {
        double var = sigma[k] * sigma[k] + jitter * jitter;
        double wk = 1.0 / var;
        double V = gamma, r;
        double g[16][5];
        if (!(var > 0.0)) {              /* var = +inf: weight 0 (Eq. 5) */
            if (grad) for (q = 0; q < n_par; ++q) grad[q] = NAN;
            return NAN;
        }
        for (j = 0; j < n_pl; ++j) {
            if (grad) V += kco_planet_velocity_grad(par + 5 * j, t[k], t0, g[j]);
            else      V += kco_planet_velocity(par + 5 * j, t[k], t0);
        }
        r = V - v[k];
        kco_sum_add(&chi2, wk * r * r);
        if (grad) {
            double a = 2.0 * wk * r;
            for (j = 0; j < n_pl; ++j)
                for (q = 0; q < 5; ++q) kco_sum_add(&gsum[5 * j + q], a * g[j][q]);
            kco_sum_add(&gsum[5 * n_pl], a);                 /* dchi2/dgamma */
            if (gabs) {
                for (j = 0; j < n_pl; ++j)
                    for (q = 0; q < 5; ++q) gabs[5 * j + q] += fabs(a * g[j][q]);
                gabs[5 * n_pl] += fabs(a);
            }
        }
    }
    if (grad) for (q = 0; q < n_par; ++q) grad[q] = kco_sum_value(&gsum[q]);
    return kco_sum_value(&chi2);
}

/* ------------------------------------------- free jitter, log-likelihood */

/* Negative log-likelihood of one system whose jitter sigma_j is a free
 * parameter, appended after gamma (5*n_pl + 2 values):
 *   nll = 1/2 sum_k [ r_k^2/(sigma_k^2 + sigma_j^2) + ln(2 pi (sigma_k^2 + sigma_j^2)) ]
 * (the Gaussian likelihood whose exponent is Eq. 5's chi2 with sigma_j
 * included).  Gradient (when grad != NULL) with respect to all 5*n_pl + 2
 * parameters; d nll / d sigma_j = sigma_j sum_k w_k (1 - w_k r_k^2). */
static double kco_nll_system(const double *par, int n_pl, const double *t,
                             const double *v, const double *sigma, int64_t n_obs,
                             double t0, double *grad, double *gabs)
{
    int n_par = 5 * n_pl + 2;
    double gamma = par[5 * n_pl], sj = par[5 * n_pl + 1];
    kco_sum nll = {0.0, 0.0};
    kco_sum gsum[5 * 16 + 2];
    int j, q;
    int64_t k;
    int valid = isfinite(gamma) && isfinite(sj);
    for (j = 0; j < n_pl; ++j) valid = valid && kco_planet_valid(par + 5 * j);
    for (q = 0; q < n_par; ++q) { gsum[q].s = 0.0; gsum[q].c = 0.0; }
    if (gabs) for (q = 0; q < n_par; ++q) gabs[q] = 0.0;
    if (!valid) {
        if (grad) for (q = 0; q < n_par; ++q) grad[q] = NAN;
        if (gabs) for (q = 0; q < n_par; ++q) gabs[q] = NAN;
        return NAN;
    }
    for (k = 0; k < n_obs; ++k) {
        double var = sigma[k] * sigma[k] + sj * sj;
        double wk = 1.0 / var;
        double V = gamma, r;
        double g[16][5];
        if (!(var > 0.0)) {
            if (grad) for (q = 0; q < n_par; ++q) grad[q] = NAN;
            return NAN;
        }
        for (j = 0; j < n_pl; ++j) {
            if (grad) V += kco_planet_velocity_grad(par + 5 * j, t[k], t0, g[j]);
            else      V += kco_planet_velocity(par + 5 * j, t[k], t0);
        }
        r = V - v[k];
        kco_sum_add(&nll, 0.5 * (wk * r * r + log(KCO_TWO_PI * var)));
        if (grad) {
            double a = wk * r;
            for (j = 0; j < n_pl; ++j)
                for (q = 0; q < 5; ++q) kco_sum_add(&gsum[5 * j + q], a * g[j][q]);
            kco_sum_add(&gsum[5 * n_pl], a);
            kco_sum_add(&gsum[5 * n_pl + 1], sj * wk * (1.0 - wk * r * r));
            if (gabs) {
                for (j = 0; j < n_pl; ++j)
                    for (q = 0; q < 5; ++q) gabs[5 * j + q] += fabs(a * g[j][q]);
                gabs[5 * n_pl] += fabs(a);
                gabs[5 * n_pl + 1] += fabs(sj * wk * (1.0 - wk * r * r));
            }
        }
    }
    if (grad) for (q = 0; q < n_par; ++q) grad[q] = kco_sum_value(&gsum[q]);
    return kco_sum_value(&nll);
}

/* ------------------------------------------------------ public entry points */

/* Uniform batch: all n_sys systems have n_pl planets and share the n_obs
 * observations (t, v, sigma).  params is [n_sys][5*n_pl+1], out is [n_sys],
 * grad and gabs (may be NULL; gabs needs grad) are [n_sys][5*n_pl+1].
 * Returns 0, or -1 on bad sizes. */
int kco_chi2(const double *params, const double *t, const double *v,
             const double *sigma, int64_t n_sys, int n_pl, int64_t n_obs,
             double t0, double jitter, double *out, double *grad, double *gabs)
{
    int64_t s;
    int n_par = 5 * n_pl + 1;
    if (n_pl < 1 || n_pl > 16 || n_obs < 0 || n_sys < 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (s = 0; s < n_sys; ++s)
        out[s] = kco_system(params + s * n_par, n_pl, t, v, sigma, n_obs, t0,
                            jitter, grad ? grad + s * n_par : NULL,
                            grad && gabs ? gabs + s * n_par : NULL);
    return 0;
}

/* Uniform batch with a free jitter per system: params [n_sys][5*n_pl+2],
 * out [n_sys] negative log-likelihoods, grad and gabs (may be NULL) like
 * params. */
int kco_nll(const double *params, const double *t, const double *v,
            const double *sigma, int64_t n_sys, int n_pl, int64_t n_obs,
            double t0, double *out, double *grad, double *gabs)
{
    int64_t s;
    int n_par = 5 * n_pl + 2;
    if (n_pl < 1 || n_pl > 16 || n_obs < 0 || n_sys < 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (s = 0; s < n_sys; ++s)
        out[s] = kco_nll_system(params + s * n_par, n_pl, t, v, sigma, n_obs, t0,
                                grad ? grad + s * n_par : NULL,
                                grad && gabs ? gabs + s * n_par : NULL);
    return 0;
}

/* Ragged batch: system s has n_pl[s] planets whose parameters start at
 * params[par_off[s]] (5*n_pl[s]+1 doubles) and its own observations
 * t/v/sigma[obs_off[s] .. obs_off[s+1]).  grad and gabs (may be NULL) use
 * the same offsets as params. */
int kco_chi2_ragged(const double *params, const int64_t *par_off,
                    const int32_t *n_pl, const double *t, const double *v,
                    const double *sigma, const int64_t *obs_off, int64_t n_sys,
                    double t0, double jitter, double *out, double *grad, double *gabs)
{
    int64_t s;
    int bad = 0;
    for (s = 0; s < n_sys; ++s)
        if (n_pl[s] < 1 || n_pl[s] > 16 || obs_off[s + 1] < obs_off[s]) bad = 1;
    if (bad || n_sys < 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (s = 0; s < n_sys; ++s)
        out[s] = kco_system(params + par_off[s], n_pl[s], t + obs_off[s],
                            v + obs_off[s], sigma + obs_off[s],
                            obs_off[s + 1] - obs_off[s], t0, jitter,
                            grad ? grad + par_off[s] : NULL,
                            grad && gabs ? gabs + par_off[s] : NULL);
    return 0;
}

/* Model velocities V(t_k) = gamma + sum_j v_j(t_k) for every system (Eq. 2):
 * out is [n_sys][n_obs]. */
int kco_predict(const double *params, const double *t, int64_t n_sys, int n_pl,
                int64_t n_obs, double t0, double *out)
{
    int64_t s;
    int n_par = 5 * n_pl + 1;
    if (n_pl < 1 || n_pl > 16 || n_obs < 0 || n_sys < 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (s = 0; s < n_sys; ++s) {
        const double *par = params + s * n_par;
        int64_t k;
        int j;
        int valid = isfinite(par[5 * n_pl]);
        for (j = 0; j < n_pl; ++j) valid = valid && kco_planet_valid(par + 5 * j);
        for (k = 0; k < n_obs; ++k) {
            double V = par[5 * n_pl];
            for (j = 0; j < n_pl; ++j) V += kco_planet_velocity(par + 5 * j, t[k], t0);
            out[s * n_obs + k] = valid ? V : NAN;
        }
    }
    return 0;
}

/* Model velocities of a ragged batch: system s (n_pl[s] planets at
 * params[par_off[s]]) at its own times t[obs_off[s] .. obs_off[s+1]);
 * out has the layout of t. */
int kco_predict_ragged(const double *params, const int64_t *par_off,
                       const int32_t *n_pl, const double *t,
                       const int64_t *obs_off, int64_t n_sys, double t0,
                       double *out)
{
    int64_t s;
    for (s = 0; s < n_sys; ++s)
        if (n_pl[s] < 1 || n_pl[s] > 16 || obs_off[s + 1] < obs_off[s]) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (s = 0; s < n_sys; ++s) {
        const double *par = params + par_off[s];
        int J = n_pl[s], j;
        int64_t k;
        int valid = isfinite(par[5 * J]);
        for (j = 0; j < J; ++j) valid = valid && kco_planet_valid(par + 5 * j);
        for (k = obs_off[s]; k < obs_off[s + 1]; ++k) {
            double V = par[5 * J];
            for (j = 0; j < J; ++j) V += kco_planet_velocity(par + 5 * j, t[k], t0);
            out[k] = valid ? V : NAN;
        }
    }
    return 0;
}

/* floor(f) clamped to 0 .. hi, NaN to 0. */
static int64_t kco_clamp_index(double f, int64_t hi)
{
    f = floor(f);
    return f >= 0.0 ? (f < (double)hi ? (int64_t)f : hi) : 0;
}

/* One differential-evolution MCMC step (ter Braak 2006) for chains
 * first .. first+count-1 (see the library's kc_demcmc_step).  Chain
 * i = first + c takes two distinct partners of the range
 * pfirst .. pfirst+m-1 (m = pcount >= 2) from its uniform draws
 * u[c][1], u[c][2]: k1 = floor(u1 m) and k2 = floor(u2 (m - 1)) (each
 * clamped into its range), k2 += (k2 >= k1), which is uniform over ordered
 * pairs of distinct chains; proposes
 *   x*_p = x_ip + gamma (x_r1,p - x_r2,p) + (eps_scale_p |x_ip|) z[c][p]
 * (each operation rounded in that order, no fused operations); evaluates
 * chi2 of the proposals in FP64 and accepts iff
 * ln u[c][0] < -(chi2* - chi2_i)/2.  Accepted states and chi2 replace the
 * current ones.  proposals [count][n_par], chi2_prop [count] and
 * accepted [count] are outputs.  Returns -1 on a bad range (the partner
 * range outside the population, shorter than 2 or overlapping the updated
 * chains). */
int kco_demcmc_step(double *states, double *chi2, int64_t n_chains, int n_pl,
                    const double *t, const double *v, const double *sigma,
                    int64_t n_obs, double t0, double jitter, int64_t first,
                    int64_t count, int64_t pfirst, int64_t pcount, double gamma,
                    const double *eps_scale, const double *z, const double *u,
                    double *proposals, double *chi2_prop, int32_t *accepted)
{
    int n_par = 5 * n_pl + 1, p;
    int64_t c;
    if (first < 0 || count < 0 || first + count > n_chains) return -1;
    if (pfirst < 0 || pcount < 2 || pfirst + pcount > n_chains) return -1;
    if (count > 0 && pfirst < first + count && first < pfirst + pcount) return -1;
    for (c = 0; c < count; ++c) {
        int64_t i = first + c;
        int64_t k1 = kco_clamp_index(u[3 * c + 1] * (double)pcount, pcount - 1);
        int64_t k2 = kco_clamp_index(u[3 * c + 2] * (double)(pcount - 1), pcount - 2);
        int64_t r1, r2;
        if (k2 >= k1) k2 += 1;
        r1 = pfirst + k1;
        r2 = pfirst + k2;
        for (p = 0; p < n_par; ++p) {
            double xi = states[i * n_par + p];
            double d = states[r1 * n_par + p] - states[r2 * n_par + p];
            double eps = (eps_scale[p] * fabs(xi)) * z[c * n_par + p];
            proposals[c * n_par + p] = (xi + gamma * d) + eps;
        }
    }
    if (kco_chi2(proposals, t, v, sigma, count, n_pl, n_obs, t0, jitter, chi2_prop,
                 NULL, NULL) != 0)
        return -1;
    for (c = 0; c < count; ++c) {
        int64_t i = first + c;
        int acc = log(u[3 * c]) < -0.5 * (chi2_prop[c] - chi2[i]);
        if (acc) {
            for (p = 0; p < n_par; ++p) states[i * n_par + p] = proposals[c * n_par + p];
            chi2[i] = chi2_prop[c];
        }
        accepted[c] = acc;
    }
    return 0;
}

/* ------------------------------------------- Gauss-Newton normal matrix */

/* H = sum_k w_k J_k J_k^T of one system, J_k = dV_k/dtheta over its
 * 5*n_pl + 1 parameters (the planets' (P, K, e, omega, M0), then gamma),
 * w_k = 1/(sigma_k^2 + jitter^2): the matrix of the normal equations of a
 * Gauss-Newton / Levenberg-Marquardt step (derivatives for least-squares
 * refinement, Sec. 6).  The Hessian of chi2 is 2 H + 2 sum_k w_k r_k
 * d2V_k/dtheta2, so at zero residuals it is 2 H.  Written as the packed
 * upper triangle, row by row: H[0][0..n-1], H[1][1..n-1], ...
 * (n (n + 1)/2 values).  NaN everywhere for invalid parameters or a
 * non-positive variance; an infinite variance is a zero weight. */
static void kco_gn_system(const double *par, int n_pl, const double *t,
                          const double *sigma, int64_t n_obs, double t0,
                          double jitter, double *H)
{
    int n_par = 5 * n_pl + 1, n_tri = n_par * (n_par + 1) / 2;
    kco_sum acc[(5 * 8 + 1) * (5 * 8 + 2) / 2];
    double J[5 * 8 + 1];
    int j, p, q, i;
    int64_t k;
    int valid = isfinite(par[5 * n_pl]);
    for (j = 0; j < n_pl; ++j) valid = valid && kco_planet_valid(par + 5 * j);
    if (!valid) {
        for (i = 0; i < n_tri; ++i) H[i] = NAN;
        return;
    }
    for (i = 0; i < n_tri; ++i) { acc[i].s = 0.0; acc[i].c = 0.0; }
    for (k = 0; k < n_obs; ++k) {
        double var = sigma[k] * sigma[k] + jitter * jitter;
        double wk = 1.0 / var;
        if (!(var > 0.0)) {
            for (i = 0; i < n_tri; ++i) H[i] = NAN;
            return;
        }
        for (j = 0; j < n_pl; ++j) kco_planet_velocity_grad(par + 5 * j, t[k], t0, J + 5 * j);
        J[5 * n_pl] = 1.0;                                        /* dV/dgamma */
        i = 0;
        for (p = 0; p < n_par; ++p)
            for (q = p; q < n_par; ++q) kco_sum_add(&acc[i++], wk * J[p] * J[q]);
    }
    for (i = 0; i < n_tri; ++i) H[i] = kco_sum_value(&acc[i]);
}

/* Uniform batch: H [n_sys][n (n + 1)/2] with n = 5*n_pl + 1 (n_pl <= 8). */
int kco_gauss_newton(const double *params, const double *t, const double *sigma,
                     int64_t n_sys, int n_pl, int64_t n_obs, double t0,
                     double jitter, double *H)
{
    int64_t s;
    int n_par = 5 * n_pl + 1, n_tri = n_par * (n_par + 1) / 2;
    if (n_pl < 1 || n_pl > 8 || n_obs < 0 || n_sys < 0) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (s = 0; s < n_sys; ++s)
        kco_gn_system(params + s * n_par, n_pl, t, sigma, n_obs, t0, jitter,
                      H + s * n_tri);
    return 0;
}

/* Elementwise Kepler solve (E for each (M, e) pair). */
void kco_kepler_batch(const double *M, const double *e, int64_t n, double *E,
                      int32_t *n_iter)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        int it = 0;
        E[i] = kco_kepler_E(M[i], e[i], &it);
        if (n_iter) n_iter[i] = it;
    }
}

/* Elementwise mean anomaly, true anomaly and single-planet velocity, for the
 * pin tests. */
void kco_mean_anomaly_batch(const double *t, double t0, const double *P,
                            const double *M0, int64_t n, double *M)
{
    int64_t i;
    for (i = 0; i < n; ++i) M[i] = kco_mean_anomaly(t[i], t0, P[i], M0[i]);
}

void kco_true_anomaly_batch(const double *E, const double *e, int64_t n, double *f)
{
    int64_t i;
    for (i = 0; i < n; ++i) f[i] = kco_true_anomaly(E[i], e[i]);
}
