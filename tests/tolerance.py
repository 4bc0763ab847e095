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
"""
import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def grad_excess(got, ref, gabs, rel, u):
    """Largest ratio of a component's error to its bound, per system row
    (arrays [n_sys, n_par]); <= 1 passes."""
    got = np.asarray(got, np.float64)
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    gabs = np.atleast_2d(np.asarray(gabs, np.float64))
    got = got.reshape(ref.shape)
    scale = np.maximum(np.abs(ref), 1e-3 * np.linalg.norm(ref, axis=1, keepdims=True))
    bound = rel * scale + 16.0 * u * gabs
    return float(np.max(np.abs(got - ref) / bound))


def grad_excess_ragged(got, ref, gabs, par_off, rel, u):
    """grad_excess for a ragged batch (parameters packed at par_off)."""
    worst = 0.0
    for s in range(len(par_off) - 1):
        sl = slice(par_off[s], par_off[s + 1])
        worst = max(worst, grad_excess(np.asarray(got)[sl][None, :], ref[sl][None, :],
                                       gabs[sl][None, :], rel, u))
    return worst
