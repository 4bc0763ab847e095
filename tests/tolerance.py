"""Parity bound of a computed gradient component, derived from the arithmetic.

Each component of the chi2 (or nll) gradient is a sum over observations,
g_i = sum_k c_ik with c_ik = 2 w_k r_k d_ik (d_ik = dV_k/dtheta_i, r_k the
residual).  The base bound,

    rel * max(|g_i|, 1e-3 ||g||)        (rel = 1e-3 single, 1e-9 double),

holds on every component whose terms do not cancel (sum_k |c_ik| <= 10 |g_i|):
there the rounding errors below are five orders of magnitude smaller.  When
the terms cancel (the period and phase derivatives near a good fit: sum_k
|c_ik| up to 1e5 |g_i|), the computed sum's forward error bound (Higham,
Accuracy and Stability of Numerical Algorithms, Sec. 4) is added, from the
kernels' own operations rather than from measured errors:

  term formation, KAPPA_FORM u sum_k |c_ik|.  The longest chain is the
    period term: sin/cos of E (sin/cos to an ulp, the angle-addition update:
    about 5 u), cos f and sin f (one product, one subtraction and the
    approximate reciprocal of D, relative error 2^-22 = 4 u: 7 u more),
    sin(w + f) (two products and an addition: 3 u), K sin(w + f)/D (two
    products and the reciprocal: 6 u), beta/D (product, reciprocal: 5 u),
    the factor 2 pi (t - t0)/P^2 (t - t0 and 1/P rounded to float, P^-2, two
    products: 5 u), then 2 w r (the weight and a product: 2 u) and the
    product with the partial (1 u): KAPPA_FORM = 34, which also covers the
    other partials (fewer operations);
  accumulation, KAPPA_SUM u sum_k |c_ik|: 2 for a compensated (Kahan) sum,
    else the terms one lane adds in order plus the levels of the lanes'
    pairwise combination, ceil(n_obs / lanes) + log2(lanes);
  the residual's own error, sum_k 2 w_k |d_ik| eps_k <= 2 sqrt(H_ii)
    sqrt(sum_k w_k eps_k^2) (Cauchy-Schwarz; H = sum_k w_k d_k d_k^T, the
    oracle's Gauss-Newton matrix), with eps_k bounding the computed
    residual's absolute error: M's float error, KAPPA_M u (below), moves
    v_j by at most KAPPA_M u K_j / D_jk^2 (|dv/dM| <= K/D^2), the Kepler
    solve's rounding of f (3 u) moves E by 3 u / D and v by 3 u K / D^2,
    sin/cos and the velocity's evaluation (products, the reciprocal) by at
    most 18 u K / D, and the planet sum and the residual add
    3 u (|V_k| + |v_k|):
        eps_k = u [sum_j K_j ((KAPPA_M + 3) / D_jk^2 + 18 / D_jk)
                   + 3 (|V_k| + |v_k|)].
  M's error, from the mixed path's operations: the phase sum
    u = frac(tau/P) + c rounds once (|u| < 1: 2^-25 cycles, 2 pi 2^-25 =
    pi u rad), the float 2 pi differs from 2 pi by 1.75e-7 (times
    |u| <= 1/2: 1.47 u), the final FMA rounds once (|M| <= pi: 2 u), the
    low part and the phase offset are exact to ~1e-14 cycles:
    KAPPA_M = pi + 3.5.

The same eps_k bounds the chi2 of the mixed path: |d chi2| <= 1e-5
max(chi2, 1) (the relative bound of the mixed path, which covers the weights and
the compensated sums) + 2 sum_k w_k |r_k| eps_k, the second term mattering
only where chi2 is small and the amplitudes large (a model at its truth,
few observations).

A component whose bound is zero (an all-zero oracle row, e.g. a system
without observations) must match exactly, and a NaN on one side only (the
GPU's value or the oracle's) always fails: both helpers return inf for it
rather than letting the comparison drop it.
"""
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53
KAPPA_FORM = 34.0
KAPPA_M = math.pi + 3.5
CANCELLING = 10.0       # sum_k |c_ik| above this multiple of |g_i|: cancellation


@dataclass
class Arith:
    """How a kernel formed and summed the gradient of a batch.

    lanes: threads that share one system's observations; n_obs: observations
    of the system (or a per-system array); compensated: mask over the
    parameter columns summed with Kahan compensation (or None); resid:
    [n_sys, n_par] the residual-error term 2 sqrt(H_ii) sqrt(sum_k w_k
    eps_k^2) (or None to leave it out)."""
    lanes: int
    n_obs: object
    compensated: Optional[np.ndarray] = None
    resid: Optional[np.ndarray] = None


def kappa_sum(arith: Arith, n_par: int) -> np.ndarray:
    """[n_sys or 1, n_par] accumulation constant."""
    n_obs = np.atleast_1d(np.asarray(arith.n_obs, np.float64))[:, None]
    plain = np.ceil(n_obs / arith.lanes) + math.log2(max(arith.lanes, 1))
    comp = np.zeros(n_par, bool) if arith.compensated is None else np.asarray(arith.compensated)
    return np.where(comp[None, :], 2.0, plain)


def grad_bound(ref, gabs, rel, u, arith: Optional[Arith] = None):
    """Per-component bound (arrays [n_sys, n_par])."""
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    gabs = np.atleast_2d(np.asarray(gabs, np.float64)).reshape(ref.shape)
    with np.errstate(invalid="ignore", over="ignore"):
        norm = np.sqrt(np.nansum(ref * ref, axis=1, keepdims=True))
        core = rel * np.maximum(np.abs(ref), 1e-3 * norm)
        if arith is None:
            return core
        extra = (KAPPA_FORM + kappa_sum(arith, ref.shape[1])) * u * gabs
        if arith.resid is not None:
            extra = extra + np.asarray(arith.resid, np.float64).reshape(ref.shape)
        cancel = gabs > CANCELLING * np.abs(ref)
        return core + np.where(cancel, extra, 0.0)


def grad_ratios(got, ref, gabs, rel, u, arith: Optional[Arith] = None):
    """Per-component ratio of the error to its bound (arrays [n_sys, n_par]):
    0 where both sides are NaN or the bound is zero and the values are equal,
    inf where only one side is NaN or a zero bound is exceeded."""
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    got = np.asarray(got, np.float64).reshape(ref.shape)
    bound = grad_bound(ref, gabs, rel, u, arith)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        err = np.abs(got - ref)
        ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0),
                         np.where(err == 0, 0.0, np.inf))
    got_nan, ref_nan = np.isnan(got), np.isnan(ref)
    ratio = np.where(got_nan & ref_nan, 0.0, ratio)
    ratio = np.where(got_nan ^ ref_nan, np.inf, ratio)
    # anything still NaN (a NaN bound from a NaN gabs with finite values) fails
    return np.where(np.isnan(ratio), np.inf, ratio)


def grad_excess(got, ref, gabs, rel, u, arith: Optional[Arith] = None):
    """Largest ratio of a component's error to its bound over all rows
    (arrays [n_sys, n_par]); <= 1 passes."""
    r = grad_ratios(got, ref, gabs, rel, u, arith)
    return float(np.max(r)) if r.size else 0.0


def grad_excess_ragged(got, ref, gabs, par_off, rel, u, ariths=None):
    """grad_excess for a ragged batch (parameters packed at par_off): the
    bound's norm is taken per system, the worst ratio over all of them.
    ariths: one Arith per system (its resid laid out [1, n_par]) or None."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    gabs = np.asarray(gabs, np.float64)
    worst = [grad_ratios(got[a:b][None, :], ref[a:b][None, :], gabs[a:b][None, :], rel, u,
                         None if ariths is None else ariths[s]).max(initial=0.0)
             for s, (a, b) in enumerate(zip(par_off[:-1], par_off[1:]))]
    return float(np.max(np.asarray(worst))) if worst else 0.0


# ------------------------------------------------------------ residual term

def residual_error(oracle, params, t, v_obs, n_pl, t0, u):
    """eps_k of every (system, observation): the bound on the computed
    residual's absolute error stated above.  params [n_sys, >= 5 n_pl + 1]."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    t = np.asarray(t, np.float64)
    n_sys = params.shape[0]
    V = oracle.predict(params[:, :5 * n_pl + 1], t, n_pl, t0)
    scale = np.zeros((n_sys, t.size))
    for j in range(n_pl):
        P, K, e, M0 = (params[:, 5 * j + q][:, None] for q in (0, 1, 2, 4))
        M = oracle.mean_anomaly(np.broadcast_to(t[None, :], (n_sys, t.size)), t0,
                                np.broadcast_to(P, (n_sys, t.size)),
                                np.broadcast_to(M0, (n_sys, t.size)))
        E = oracle.kepler_E(M, np.broadcast_to(e, M.shape))
        D = 1.0 - e * np.cos(E)
        scale += np.abs(K) * ((KAPPA_M + 3.0) / D ** 2 + 18.0 / D)
    return u * (scale + 3.0 * (np.abs(V) + np.abs(np.asarray(v_obs, np.float64))[None, :]))


def chi2_rounding_term(oracle, params, t, v_obs, sigma, n_pl, t0, jitter, u):
    """[n_sys] 2 sum_k w_k |r_k| eps_k: the computed residuals' error carried
    into chi2 (first order), r_k from the oracle's model."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    v_obs = np.asarray(v_obs, np.float64)
    w = 1.0 / (np.asarray(sigma, np.float64) ** 2 + jitter ** 2)
    eps = residual_error(oracle, params, t, v_obs, n_pl, t0, u)
    r = np.abs(oracle.predict(params[:, :5 * n_pl + 1], t, n_pl, t0) - v_obs[None, :])
    return 2.0 * np.sum(w[None, :] * r * eps, axis=1)


def residual_term(oracle, params, t, v_obs, sigma, n_pl, t0, jitter, u):
    """[n_sys, 5 n_pl + 1] the residual-error term 2 sqrt(H_ii) sqrt(sum_k
    w_k eps_k^2) of a uniform batch (H from the oracle's Gauss-Newton
    matrix).  Free-jitter batches pass their planets and gamma; the jitter
    column then takes 2 sigma_j sqrt(sum_k w_k^3 r_k^2) sqrt(sum_k w_k eps_k^2)
    (the same Cauchy-Schwarz step on its terms sigma_j w_k (1 - w_k r_k^2))."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    n = 5 * n_pl + 1
    w = 1.0 / (np.asarray(sigma, np.float64) ** 2 + jitter ** 2)
    eps = residual_error(oracle, params, t, v_obs, n_pl, t0, u)
    rms = np.sqrt(np.sum(w[None, :] * eps ** 2, axis=1))
    H = oracle.gauss_newton(params[:, :n], t, sigma, n_pl, t0=t0, jitter=jitter, packed=False)
    return 2.0 * np.sqrt(np.maximum(np.diagonal(H, axis1=1, axis2=2), 0.0)) * rms[:, None]


def nll_residual_term(oracle, params, t, v_obs, sigma, n_pl, t0, u):
    """residual_term for free-jitter parameters [n_sys, 5 n_pl + 2]: the
    weights taken at zero jitter (larger than the system's own, so the term
    only grows), and the jitter column's term as stated above."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    n = 5 * n_pl + 1
    base = residual_term(oracle, params[:, :n], t, v_obs, sigma, n_pl, t0, 0.0, u)
    w0 = 1.0 / np.asarray(sigma, np.float64) ** 2
    eps = residual_error(oracle, params[:, :n], t, v_obs, n_pl, t0, u)
    rms = np.sqrt(np.sum(w0[None, :] * eps ** 2, axis=1))
    r = oracle.predict(params[:, :n], t, n_pl, t0) - np.asarray(v_obs, np.float64)[None, :]
    sj = np.abs(params[:, n])
    jit = 2.0 * sj * np.sqrt(np.sum(w0[None, :] ** 3 * r ** 2, axis=1)) * rms
    return np.concatenate([base, jit[:, None]], axis=1)


def uniform_arith(kc, oracle, params, t, v_obs, sigma, n_pl, t0, jitter, mode, kind="grad",
                  n_sys_launch=None):
    """The Arith of a uniform batch's gradient: the lanes per system of the
    tile the library launched (kc_get_tile; the Gauss-Newton kernel runs a
    warp per system), the period columns compensated in the mixed kernels,
    and the residual term.  kind: 'grad', 'nll' (free jitter) or 'gn'."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    n_obs = int(np.asarray(t).size)
    u = U32 if mode == "mixed" else U64
    if kind == "gn":
        lanes = 32
    else:
        n_sys = n_sys_launch if n_sys_launch is not None else params.shape[0]
        lanes = kc.kc_get_tile("grad", mode, n_sys, n_pl, n_obs)[0]
    comp = np.zeros(params.shape[1], bool)
    if mode == "mixed":
        comp[0:5 * n_pl:5] = True
    if kind == "nll":
        resid = nll_residual_term(oracle, params, t, v_obs, sigma, n_pl, t0, u)
    else:
        resid = residual_term(oracle, params, t, v_obs, sigma, n_pl, t0, jitter, u)
    return Arith(lanes, n_obs, comp, resid)


def ragged_ariths(oracle, params, par_off, n_pl, t, v_obs, sigma, obs_off, t0, jitter, mode):
    """One Arith per system of a ragged batch: a warp per system, the period
    columns compensated in the mixed kernel."""
    u = U32 if mode == "mixed" else U64
    out = []
    for s in range(len(n_pl)):
        J = int(n_pl[s])
        a, b = par_off[s], par_off[s + 1]
        o0, o1 = obs_off[s], obs_off[s + 1]
        comp = np.zeros(b - a, bool)
        if mode == "mixed":
            comp[0:5 * J:5] = True
        resid = None
        if o1 > o0:
            resid = residual_term(oracle, params[a:b][None, :], t[o0:o1], v_obs[o0:o1],
                                  sigma[o0:o1], J, t0, jitter, u)
        out.append(Arith(32, o1 - o0, comp, resid))
    return out
