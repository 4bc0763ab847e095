"""FP64 CPU oracle for the batched Keplerian radial-velocity chi-square.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import this
module.  It wraps ``kc_oracle.c`` (plain C, double precision) through ctypes
and shares no code with the CUDA path.

Every function takes and returns numpy float64 arrays.  Parameters of one
system are laid out as (P, K, e, omega, M0) per planet followed by the
offset gamma (``5*n_pl + 1`` values), the same order as Sec. 4.1 lists them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkc_oracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU needed); returns the .so path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = bind(ctypes.CDLL(build()))
        return _lib


def compile_variant(source: str, path: str):
    """Compile another version of the oracle's C source (used by the tests
    that plant mistakes to check that the pins catch them) and return it
    bound like the real one; install it with ``use(lib)``."""
    src = path + ".c"
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(["gcc", *_CFLAGS, src, "-o", path, "-lm"], check=True)
    return bind(ctypes.CDLL(path))


def use(lib) -> None:
    """Make every function of this module call ``lib`` (None: the real one)."""
    global _lib
    _lib = lib


def bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    d = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.kco_set_threads.argtypes = [ctypes.c_int]
    lib.kco_max_threads.restype = ctypes.c_int
    lib.kco_mean_anomaly.restype = ctypes.c_double
    lib.kco_mean_anomaly.argtypes = [ctypes.c_double] * 4
    lib.kco_kepler_E.restype = ctypes.c_double
    lib.kco_kepler_E.argtypes = [ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(ctypes.c_int)]
    lib.kco_true_anomaly.restype = ctypes.c_double
    lib.kco_true_anomaly.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.kco_planet_velocity.restype = ctypes.c_double
    lib.kco_planet_velocity.argtypes = [d, ctypes.c_double, ctypes.c_double]
    lib.kco_chi2.restype = ctypes.c_int
    lib.kco_chi2.argtypes = [d, d, d, d, i64, ctypes.c_int, i64,
                             ctypes.c_double, ctypes.c_double, d, d, d]
    lib.kco_nll.restype = ctypes.c_int
    lib.kco_nll.argtypes = [d, d, d, d, i64, ctypes.c_int, i64, ctypes.c_double, d, d, d]
    lib.kco_chi2_ragged.restype = ctypes.c_int
    lib.kco_chi2_ragged.argtypes = [d, i64p, i32p, d, d, d, i64p, i64,
                                    ctypes.c_double, ctypes.c_double, d, d, d]
    lib.kco_predict.restype = ctypes.c_int
    lib.kco_predict.argtypes = [d, d, i64, ctypes.c_int, i64,
                                ctypes.c_double, d]
    lib.kco_predict_ragged.restype = ctypes.c_int
    lib.kco_predict_ragged.argtypes = [d, i64p, i32p, d, i64p, i64, ctypes.c_double, d]
    lib.kco_demcmc_step.restype = ctypes.c_int
    lib.kco_demcmc_step.argtypes = [d, d, i64, ctypes.c_int, d, d, d, i64, ctypes.c_double,
                                    ctypes.c_double, i64, i64, i64, i64, ctypes.c_double, d, d,
                                    d, d, d, i32p]
    lib.kco_gauss_newton.argtypes = [d, d, d, i64, ctypes.c_int, i64, ctypes.c_double,
                                     ctypes.c_double, d]
    lib.kco_gauss_newton.restype = ctypes.c_int
    lib.kco_kepler_batch.argtypes = [d, d, i64, d, i32p]
    lib.kco_mean_anomaly_batch.argtypes = [d, ctypes.c_double, d, d, i64, d]
    lib.kco_true_anomaly_batch.argtypes = [d, d, i64, d]
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's batch loops use."""
    _load().kco_set_threads(int(n))


def max_threads() -> int:
    return int(_load().kco_max_threads())


def mean_anomaly(t, t0, P, M0) -> np.ndarray:
    """M = 2 pi frac((t - t0)/P) + M0 reduced to [-pi, pi] (Eqs. 4, 6)."""
    t, P, M0 = np.broadcast_arrays(_f64(t), _f64(P), _f64(M0))
    t, P, M0 = _f64(t), _f64(P), _f64(M0)
    out = np.empty_like(t)
    _load().kco_mean_anomaly_batch(_p(t.ravel()), float(t0), _p(P.ravel()),
                                   _p(M0.ravel()), t.size, _p(out))
    return out


def kepler_E(M, e, return_iters: bool = False):
    """Root E of E - e sin E = M (Eq. 1), elementwise."""
    M, e = np.broadcast_arrays(_f64(M), _f64(e))
    M, e = _f64(M), _f64(e)
    E = np.empty_like(M)
    it = np.empty(M.shape, dtype=np.int32)
    _load().kco_kepler_batch(_p(M), _p(e), M.size, _p(E),
                             _p(it, ctypes.c_int32))
    return (E, it) if return_iters else E


def true_anomaly(E, e) -> np.ndarray:
    E, e = np.broadcast_arrays(_f64(E), _f64(e))
    E, e = _f64(E), _f64(e)
    f = np.empty_like(E)
    _load().kco_true_anomaly_batch(_p(E), _p(e), E.size, _p(f))
    return f


def planet_velocity(p5, t, t0: float = 0.0) -> np.ndarray:
    """Velocity of one planet (P, K, e, omega, M0) at each time t (Eq. 3)."""
    p5 = _f64(p5)
    lib = _load()
    return np.array([lib.kco_planet_velocity(_p(p5), float(tk), float(t0))
                     for tk in np.asarray(t, dtype=np.float64).ravel()])


def predict(params, t, n_pl: int, t0: float = 0.0) -> np.ndarray:
    """Model velocities gamma + sum_j v_j(t_k): [n_sys, n_obs] (Eq. 2)."""
    params, t = _f64(params), _f64(t)
    n_par = 5 * n_pl + 1
    params = params.reshape(-1, n_par)
    out = np.empty((params.shape[0], t.size))
    rc = _load().kco_predict(_p(params), _p(t), params.shape[0], int(n_pl),
                             t.size, float(t0), _p(out))
    if rc != 0:
        raise ValueError("oracle.predict: bad sizes")
    return out


def chi2(params, t, v, sigma, n_pl: int, t0: float = 0.0,
         jitter: float = 0.0, grad: bool = False, gabs: bool = False):
    """chi-square of every system against shared data (Eq. 5).

    Returns chi2 [n_sys], or (chi2, grad [n_sys, 5*n_pl+1]) when grad=True,
    or (chi2, grad, gabs) when gabs=True as well: gabs = sum over the
    observations of |each observation's term of the gradient|, the scale of
    the cancellation in each component's sum (Higham's bound of a computed
    sum is proportional to it).
    """
    params, t, v, sigma = _f64(params), _f64(t), _f64(v), _f64(sigma)
    n_par = 5 * n_pl + 1
    params = params.reshape(-1, n_par)
    n_sys = params.shape[0]
    out = np.empty(n_sys)
    grad = grad or gabs
    g = np.empty((n_sys, n_par)) if grad else None
    ga = np.empty((n_sys, n_par)) if gabs else None
    rc = _load().kco_chi2(_p(params), _p(t), _p(v), _p(sigma), n_sys,
                          int(n_pl), t.size, float(t0), float(jitter), _p(out),
                          _p(g) if grad else None, _p(ga) if gabs else None)
    if rc != 0:
        raise ValueError("oracle.chi2: bad sizes")
    if gabs:
        return out, g, ga
    return (out, g) if grad else out


def gauss_newton(params, t, sigma, n_pl: int, t0: float = 0.0, jitter: float = 0.0,
                 packed: bool = True):
    """Gauss-Newton matrix H = sum_k w_k J_k J_k^T of every system (J_k =
    dV_k/dtheta over the 5*n_pl + 1 parameters): [n_sys, n(n+1)/2] packed
    upper triangle row by row, or [n_sys, n, n] with packed=False."""
    params, t, sigma = _f64(params), _f64(t), _f64(sigma)
    n_par = 5 * n_pl + 1
    params = params.reshape(-1, n_par)
    n_sys = params.shape[0]
    H = np.empty((n_sys, n_par * (n_par + 1) // 2))
    rc = _load().kco_gauss_newton(_p(params), _p(t), _p(sigma), n_sys, int(n_pl), t.size,
                                  float(t0), float(jitter), _p(H))
    if rc != 0:
        raise ValueError("oracle.gauss_newton: bad sizes")
    return H if packed else unpack_symmetric(H, n_par)


def unpack_symmetric(H, n: int):
    """[..., n(n+1)/2] packed upper triangle (row by row) -> [..., n, n]."""
    H = np.asarray(H)
    iu = np.triu_indices(n)
    full = np.zeros(H.shape[:-1] + (n, n))
    full[..., iu[0], iu[1]] = H
    full[..., iu[1], iu[0]] = H
    return full


def nll(params, t, v, sigma, n_pl: int, t0: float = 0.0, grad: bool = False,
        gabs: bool = False):
    """Negative log-likelihood with a free jitter per system (parameters
    [n_sys, 5*n_pl+2]: planets, gamma, sigma_j):
    1/2 sum_k [r_k^2/(sigma_k^2+sigma_j^2) + ln(2 pi (sigma_k^2+sigma_j^2))].
    grad and gabs as for chi2."""
    params, t, v, sigma = _f64(params), _f64(t), _f64(v), _f64(sigma)
    n_par = 5 * n_pl + 2
    params = params.reshape(-1, n_par)
    n_sys = params.shape[0]
    out = np.empty(n_sys)
    grad = grad or gabs
    g = np.empty((n_sys, n_par)) if grad else None
    ga = np.empty((n_sys, n_par)) if gabs else None
    rc = _load().kco_nll(_p(params), _p(t), _p(v), _p(sigma), n_sys, int(n_pl), t.size,
                         float(t0), _p(out), _p(g) if grad else None,
                         _p(ga) if gabs else None)
    if rc != 0:
        raise ValueError("oracle.nll: bad sizes")
    if gabs:
        return out, g, ga
    return (out, g) if grad else out


def chi2_ragged(params, par_off, n_pl, t, v, sigma, obs_off, t0: float = 0.0,
                jitter: float = 0.0, grad: bool = False, gabs: bool = False):
    """chi-square of systems with their own planet counts and observations.

    System s: parameters params[par_off[s] : par_off[s] + 5*n_pl[s] + 1],
    observations t/v/sigma[obs_off[s] : obs_off[s+1]].  grad and gabs as
    for chi2 (laid out like params).
    """
    params, t, v, sigma = _f64(params), _f64(t), _f64(v), _f64(sigma)
    par_off = np.ascontiguousarray(par_off, dtype=np.int64)
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    n_pl = np.ascontiguousarray(n_pl, dtype=np.int32)
    n_sys = n_pl.size
    out = np.empty(n_sys)
    grad = grad or gabs
    g = np.empty_like(params) if grad else None
    ga = np.empty_like(params) if gabs else None
    rc = _load().kco_chi2_ragged(
        _p(params), _p(par_off, ctypes.c_int64), _p(n_pl, ctypes.c_int32),
        _p(t), _p(v), _p(sigma), _p(obs_off, ctypes.c_int64), n_sys,
        float(t0), float(jitter), _p(out), _p(g) if grad else None,
        _p(ga) if gabs else None)
    if rc != 0:
        raise ValueError("oracle.chi2_ragged: bad sizes")
    if gabs:
        return out, g, ga
    return (out, g) if grad else out


def predict_ragged(params, par_off, n_pl, t, obs_off, t0: float = 0.0) -> np.ndarray:
    """Model velocities of a ragged batch, laid out like t (Eq. 2)."""
    params, t = _f64(params), _f64(t)
    par_off = np.ascontiguousarray(par_off, dtype=np.int64)
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    n_pl = np.ascontiguousarray(n_pl, dtype=np.int32)
    out = np.empty_like(t)
    rc = _load().kco_predict_ragged(_p(params), _p(par_off, ctypes.c_int64),
                                    _p(n_pl, ctypes.c_int32), _p(t),
                                    _p(obs_off, ctypes.c_int64), n_pl.size, float(t0),
                                    _p(out))
    if rc != 0:
        raise ValueError("oracle.predict_ragged: bad sizes")
    return out


def demcmc_step(states, chi2_cur, t, v, sigma, n_pl: int, first: int, count: int,
                pfirst: int, pcount: int, gamma: float, eps_scale, z, u, t0: float = 0.0,
                jitter: float = 0.0):
    """One DE-MC step of chains first .. first+count-1 (ter Braak 2006), the
    partners drawn from chains pfirst .. pfirst+pcount-1; z [count, n_par]
    standard normal and u [count, 3] uniform draws.  Returns (states, chi2,
    accepted, proposals, chi2_of_proposals); the inputs are not modified."""
    states = _f64(states).copy()
    chi2_cur = _f64(chi2_cur).copy()
    t, v, sigma = _f64(t), _f64(v), _f64(sigma)
    n_par = 5 * n_pl + 1
    n_chains = states.size // n_par
    eps_scale = np.ascontiguousarray(np.broadcast_to(_f64(eps_scale), (n_par,)))
    z, u = _f64(z), _f64(u)
    prop = np.empty((count, n_par))
    chi2_prop = np.empty(count)
    acc = np.empty(count, dtype=np.int32)
    rc = _load().kco_demcmc_step(_p(states), _p(chi2_cur), n_chains, int(n_pl), _p(t), _p(v),
                                 _p(sigma), t.size, float(t0), float(jitter), int(first),
                                 int(count), int(pfirst), int(pcount), float(gamma),
                                 _p(eps_scale), _p(z), _p(u), _p(prop), _p(chi2_prop),
                                 _p(acc, ctypes.c_int32))
    if rc != 0:
        raise ValueError("oracle.demcmc_step: bad range")
    return states.reshape(-1, n_par), chi2_cur, acc, prop, chi2_prop
