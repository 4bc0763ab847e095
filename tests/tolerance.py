"""Parity bound of a computed gradient component, derived from the arithmetic.

Each component of the chi2 (or nll) gradient is a sum over observations,
g_i = sum_k c_ik.  Computed in a working precision with unit roundoff u,
every term c_ik carries a relative error of a few u from the arithmetic
that forms it (the partial derivatives, the residual), and the sum's error
is bounded by that error times sum_k |c_ik| (the standard forward bound of
a floating-point sum, Higham, Accuracy and Stability of Numerical
Algorithms, Sec. 4).  When the terms cancel (the period and phase
derivatives near a good fit: sum_k |c_ik| up to 1e5 |g_i|), that bound, not
|g_i|, sets how close single precision can come.  A component passes if

    |g_i - g_i(oracle)| <= rel * max(|g_i(oracle)|, 1e-3 ||g(oracle)||)
                           + 16 u sum_k |c_ik|,

rel being the path's relative tolerance (1e-3 single precision, 1e-9
double) and u = 2^-24 or 2^-53; sum_k |c_ik| comes from the oracle (gabs).
16 u leaves a factor 5 over the largest error measured on the GPU
(3.2 u sum_k |c_ik|, 3000-system gradient workload).

A component whose bound is zero (an all-zero oracle row, e.g. a system
without observations) must match exactly, and a NaN on one side only
(the GPU's value or the oracle's) always fails: both helpers return inf
for it rather than letting the comparison drop it.
"""
import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def grad_ratios(got, ref, gabs, rel, u):
    """Per-component ratio of the error to its bound (arrays [n_sys, n_par]):
    0 where both sides are NaN or the bound is zero and the values are equal,
    inf where only one side is NaN or a zero bound is exceeded."""
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    gabs = np.atleast_2d(np.asarray(gabs, np.float64))
    got = np.asarray(got, np.float64).reshape(ref.shape)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        norm = np.sqrt(np.nansum(ref * ref, axis=1, keepdims=True))
        scale = np.maximum(np.abs(ref), 1e-3 * norm)
        bound = rel * scale + 16.0 * u * gabs
        err = np.abs(got - ref)
        ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0),
                         np.where(err == 0, 0.0, np.inf))
    got_nan, ref_nan = np.isnan(got), np.isnan(ref)
    ratio = np.where(got_nan & ref_nan, 0.0, ratio)
    ratio = np.where(got_nan ^ ref_nan, np.inf, ratio)
    # anything still NaN (a NaN bound from a NaN gabs with finite values) fails
    return np.where(np.isnan(ratio), np.inf, ratio)


def grad_excess(got, ref, gabs, rel, u):
    """Largest ratio of a component's error to its bound over all rows
    (arrays [n_sys, n_par]); <= 1 passes."""
    r = grad_ratios(got, ref, gabs, rel, u)
    return float(np.max(r)) if r.size else 0.0


def grad_excess_ragged(got, ref, gabs, par_off, rel, u):
    """grad_excess for a ragged batch (parameters packed at par_off): the
    bound's norm is taken per system, the worst ratio over all of them."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    gabs = np.asarray(gabs, np.float64)
    worst = [grad_ratios(got[a:b][None, :], ref[a:b][None, :], gabs[a:b][None, :], rel, u)
             .max(initial=0.0) for a, b in zip(par_off[:-1], par_off[1:])]
    return float(np.max(np.asarray(worst))) if worst else 0.0
