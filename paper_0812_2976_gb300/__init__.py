"""GB300-native batched Keplerian radial-velocity chi-square (Ford 2008).

Thin PyTorch binding over libkc.so: every function here marshals tensors to
the C ABI of include/kc.h and calls it on the current CUDA stream; all
arithmetic runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams only.

Parameters of one system: (P, K, e, omega, M0) per planet, then gamma, so a
batch is a float64 CUDA tensor [n_sys, 5*n_pl + 1].  Observations t, v_obs,
sigma are float64 CUDA tensors [n_obs] shared by every system.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import torch

from . import _lib
from ._lib import KC_FP32, KC_FP64, KC_MIXED, KC_MAX_PLANETS, KcError

__all__ = [
    "KC_FP64", "KC_MIXED", "KC_FP32", "KC_MAX_PLANETS", "KcError",
    "kc_chi2_eval", "kc_chi2_eval_mixed", "kc_chi2_eval_ex", "kc_chi2_grad",
    "kc_chi2_eval_mixed_noalloc", "kc_nll_eval", "kc_nll_grad", "nll",
    "kc_demcmc_step", "DEMCMC", "kc_chi2_gauss_newton",
    "kc_rv_predict", "kc_rv_predict_ragged", "kc_kepler_solve", "kc_autotune", "kc_set_tile", "kc_get_tile",
    "RaggedPlan", "chi2", "n_planets", "library_path", "kc_last_device_error", "kc_measure_pipe_rate",
]

library_path = _lib.LIB_PATH


def _mode(mode) -> int:
    if mode in (KC_FP64, "fp64", "f64", "double"):
        return KC_FP64
    if mode in (KC_MIXED, "mixed"):
        return KC_MIXED
    if mode in (KC_FP32, "fp32", "single"):
        return KC_FP32      # kc_chi2_eval_ex only: the all-single-precision comparison
    raise ValueError(f"unknown mode {mode!r}: use 'fp64' or 'mixed'")


def _ptr(x: Optional[torch.Tensor]) -> Optional[int]:
    return None if x is None else x.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


def _dev_f64(name: str, x: torch.Tensor, dim: int) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if x.dim() != dim:
        raise ValueError(f"{name} must be {dim}-D")
    return x.contiguous()


def _out_f32(name: str, x, n: int, device) -> None:
    """A caller-provided float32 output of at least n elements on `device`."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.device != device:
        raise TypeError(f"{name} must be a CUDA tensor on {device}")
    if x.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not x.is_contiguous() or x.numel() < n:
        raise ValueError(f"{name} must be contiguous with at least {n} elements")


def n_planets(params: torch.Tensor) -> int:
    """n_pl from a [n_sys, 5*n_pl+1] parameter batch."""
    n = params.shape[-1] - 1
    if n <= 0 or n % 5:
        raise ValueError("params must have 5*n_pl + 1 columns")
    return n // 5


def _obs(t, v_obs, sigma):
    t = _dev_f64("t", t, 1)
    v_obs = _dev_f64("v_obs", v_obs, 1)
    sigma = _dev_f64("sigma", sigma, 1)
    if not (t.numel() == v_obs.numel() == sigma.numel()):
        raise ValueError("t, v_obs and sigma must have the same length")
    return t, v_obs, sigma


def kc_chi2_eval_ex(params, t, v_obs, sigma, t0: float = 0.0, jitter: float = 0.0,
                    mode="mixed", out: Optional[torch.Tensor] = None,
                    max_kepler_resid=None, stream=None):
    """chi2 of every system (include/kc.h: kc_chi2_eval_ex).

    Returns ``out`` [n_sys] (float64 for 'fp64', float32 for 'mixed'); if
    ``max_kepler_resid`` is True or a float32 tensor, returns (out, resid)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    m = _mode(mode)
    n_sys, n_pl = params.shape[0], n_planets(params)
    dtype = torch.float64 if m == KC_FP64 else torch.float32
    if out is None:
        out = torch.empty(n_sys, dtype=dtype, device=params.device)
    resid = None
    if max_kepler_resid is True:
        resid = torch.empty(n_sys, dtype=torch.float32, device=params.device)
    elif isinstance(max_kepler_resid, torch.Tensor):
        resid = max_kepler_resid
    lib = _lib.load()
    _lib.check(lib.kc_chi2_eval_ex(
        params.data_ptr(), t.data_ptr(), v_obs.data_ptr(), sigma.data_ptr(), n_sys, n_pl,
        t.numel(), float(t0), float(jitter), m, out.data_ptr(), _ptr(resid),
        _stream(stream)), "kc_chi2_eval_ex")
    return (out, resid) if resid is not None else out


def kc_measure_pipe_rate(pipe: str = "fp64", stream=None) -> float:
    """Measured FMA throughput per SM per clock of the FP32 ('fp32') or FP64
    ('fp64') pipe (kc_measure_pipe_rate; blocking)."""
    r = ctypes.c_double(0.0)
    lib = _lib.load()
    _lib.check(lib.kc_measure_pipe_rate({"fp32": 0, "fp64": 1}[pipe], ctypes.byref(r),
                                        _stream(stream)), "kc_measure_pipe_rate")
    return float(r.value)


def kc_last_device_error() -> int:
    """Systems whose result came out NaN since the previous call on the
    current device (kc_last_device_error; synchronises the device)."""
    n = ctypes.c_int64(0)
    lib = _lib.load()
    _lib.check(lib.kc_last_device_error(ctypes.byref(n)), "kc_last_device_error")
    return int(n.value)


def kc_chi2_eval(params, t, v_obs, sigma, out=None, stream=None) -> torch.Tensor:
    """FP64 chi2, t0 = 0, no jitter (include/kc.h: kc_chi2_eval)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    n_sys = params.shape[0]
    if out is None:
        out = torch.empty(n_sys, dtype=torch.float64, device=params.device)
    lib = _lib.load()
    _lib.check(lib.kc_chi2_eval(params.data_ptr(), t.data_ptr(), v_obs.data_ptr(),
                                sigma.data_ptr(), n_sys, n_planets(params), t.numel(),
                                out.data_ptr(), _stream(stream)), "kc_chi2_eval")
    return out


def kc_chi2_eval_mixed(params, t, v_obs, sigma, out=None, max_kepler_resid=None,
                       stream=None):
    """Mixed-precision chi2, t0 = 0, no jitter (kc_chi2_eval_mixed)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    n_sys = params.shape[0]
    if out is None:
        out = torch.empty(n_sys, dtype=torch.float32, device=params.device)
    resid = None
    if max_kepler_resid is True:
        resid = torch.empty(n_sys, dtype=torch.float32, device=params.device)
    elif isinstance(max_kepler_resid, torch.Tensor):
        resid = max_kepler_resid
    lib = _lib.load()
    _lib.check(lib.kc_chi2_eval_mixed(
        params.data_ptr(), t.data_ptr(), v_obs.data_ptr(), sigma.data_ptr(), n_sys,
        n_planets(params), t.numel(), out.data_ptr(), _ptr(resid), _stream(stream)),
        "kc_chi2_eval_mixed")
    return (out, resid) if resid is not None else out


def kc_chi2_eval_mixed_noalloc(params, t, v_obs, sigma, out, t0: float = 0.0,
                               jitter: float = 0.0, max_kepler_resid=None, stream=None):
    """Mixed chi2 without any device allocation by the library
    (kc_chi2_eval_mixed_noalloc): for callers that must not allocate while
    evaluating.  ``out`` (float32 [n_sys]) and the optional float32
    ``max_kepler_resid`` must be provided by the caller; intermediate data
    go to a fixed array inside libkc.so, so problems are limited to
    KC_NOALLOC_SCRATCH_BYTES of it and overlapping calls must be serialised.
    Inputs must already be contiguous (a copy would allocate) and the
    outputs float32 CUDA tensors on the parameters' device."""
    for name, x, dim in (("params", params, 2), ("t", t, 1), ("v_obs", v_obs, 1),
                         ("sigma", sigma, 1)):
        _dev_f64(name, x, dim)
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous: this call makes no copy")
    if not (t.numel() == v_obs.numel() == sigma.numel()):
        raise ValueError("t, v_obs and sigma must have the same length")
    n_sys = params.shape[0]
    _out_f32("out", out, n_sys, params.device)
    if max_kepler_resid is not None:
        _out_f32("max_kepler_resid", max_kepler_resid, n_sys, params.device)
    lib = _lib.load()
    _lib.check(lib.kc_chi2_eval_mixed_noalloc(
        params.data_ptr(), t.data_ptr(), v_obs.data_ptr(), sigma.data_ptr(), params.shape[0],
        n_planets(params), t.numel(), float(t0), float(jitter), out.data_ptr(),
        _ptr(max_kepler_resid), _stream(stream)), "kc_chi2_eval_mixed_noalloc")
    return out


def kc_chi2_grad(params, t, v_obs, sigma, t0: float = 0.0, jitter: float = 0.0,
                 mode="mixed", chi2_out=None, grad_out=None,
                 stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
    """(chi2 [n_sys], d chi2/d params [n_sys, 5*n_pl+1]) (kc_chi2_grad)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    m = _mode(mode)
    dtype = torch.float64 if m == KC_FP64 else torch.float32
    n_sys = params.shape[0]
    if chi2_out is None:
        chi2_out = torch.empty(n_sys, dtype=dtype, device=params.device)
    if grad_out is None:
        grad_out = torch.empty(params.shape, dtype=dtype, device=params.device)
    lib = _lib.load()
    _lib.check(lib.kc_chi2_grad(
        params.data_ptr(), t.data_ptr(), v_obs.data_ptr(), sigma.data_ptr(), n_sys,
        n_planets(params), t.numel(), float(t0), float(jitter), m, chi2_out.data_ptr(),
        grad_out.data_ptr(), _stream(stream)), "kc_chi2_grad")
    return chi2_out, grad_out


def kc_chi2_gauss_newton(params, t, v_obs, sigma, t0: float = 0.0, jitter: float = 0.0,
                         mode="mixed", chi2_out=None, grad_out=None, jtj_out=None,
                         stream=None):
    """(chi2 [n_sys], gradient [n_sys, n], Gauss-Newton matrix [n_sys, n(n+1)/2]
    packed upper triangle row by row), n = 5*n_pl + 1 (kc_chi2_gauss_newton)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    m = _mode(mode)
    if m not in (KC_FP64, KC_MIXED):
        raise ValueError("kc_chi2_gauss_newton takes 'fp64' or 'mixed'")
    dtype = torch.float64 if m == KC_FP64 else torch.float32
    n_sys, n = params.shape[0], params.shape[1]
    if chi2_out is None:
        chi2_out = torch.empty(n_sys, dtype=dtype, device=params.device)
    if grad_out is None:
        grad_out = torch.empty((n_sys, n), dtype=dtype, device=params.device)
    if jtj_out is None:
        jtj_out = torch.empty((n_sys, n * (n + 1) // 2), dtype=dtype, device=params.device)
    lib = _lib.load()
    _lib.check(lib.kc_chi2_gauss_newton(
        params.data_ptr(), t.data_ptr(), v_obs.data_ptr(), sigma.data_ptr(), n_sys,
        n_planets(params), t.numel(), float(t0), float(jitter), m, chi2_out.data_ptr(),
        grad_out.data_ptr(), jtj_out.data_ptr(), _stream(stream)), "kc_chi2_gauss_newton")
    return chi2_out, grad_out, jtj_out


def n_planets_nll(params: torch.Tensor) -> int:
    """n_pl from a [n_sys, 5*n_pl+2] free-jitter parameter batch."""
    n = params.shape[-1] - 2
    if n <= 0 or n % 5:
        raise ValueError("params must have 5*n_pl + 2 columns (planets, gamma, jitter)")
    return n // 5


def kc_nll_eval(params, t, v_obs, sigma, t0: float = 0.0, mode="mixed", out=None,
                stream=None) -> torch.Tensor:
    """Free-jitter negative log-likelihood [n_sys] (kc_nll_eval); params are
    [n_sys, 5*n_pl+2] = planets, gamma, sigma_j."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    m = _mode(mode)
    if out is None:
        out = torch.empty(params.shape[0], dtype=torch.float64 if m == KC_FP64 else torch.float32,
                          device=params.device)
    lib = _lib.load()
    _lib.check(lib.kc_nll_eval(params.data_ptr(), t.data_ptr(), v_obs.data_ptr(),
                               sigma.data_ptr(), params.shape[0], n_planets_nll(params),
                               t.numel(), float(t0), m, out.data_ptr(), _stream(stream)),
               "kc_nll_eval")
    return out


def kc_nll_grad(params, t, v_obs, sigma, t0: float = 0.0, mode="mixed", nll_out=None,
                grad_out=None, stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
    """(nll [n_sys], gradient [n_sys, 5*n_pl+2]) (kc_nll_grad)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    m = _mode(mode)
    dtype = torch.float64 if m == KC_FP64 else torch.float32
    if nll_out is None:
        nll_out = torch.empty(params.shape[0], dtype=dtype, device=params.device)
    if grad_out is None:
        grad_out = torch.empty(params.shape, dtype=dtype, device=params.device)
    lib = _lib.load()
    _lib.check(lib.kc_nll_grad(params.data_ptr(), t.data_ptr(), v_obs.data_ptr(),
                               sigma.data_ptr(), params.shape[0], n_planets_nll(params),
                               t.numel(), float(t0), m, nll_out.data_ptr(), grad_out.data_ptr(),
                               _stream(stream)), "kc_nll_grad")
    return nll_out, grad_out


def kc_rv_predict(params, t, t0: float = 0.0, out=None, stream=None) -> torch.Tensor:
    """FP64 model velocities [n_sys, n_obs] (kc_rv_predict)."""
    params = _dev_f64("params", params, 2)
    t = _dev_f64("t", t, 1)
    n_sys = params.shape[0]
    if out is None:
        out = torch.empty((n_sys, t.numel()), dtype=torch.float64, device=params.device)
    lib = _lib.load()
    _lib.check(lib.kc_rv_predict(params.data_ptr(), t.data_ptr(), n_sys, n_planets(params),
                                 t.numel(), float(t0), out.data_ptr(), _stream(stream)),
               "kc_rv_predict")
    return out


def kc_rv_predict_ragged(params, par_off, n_pl, t, obs_off, t0: float = 0.0, out=None,
                         stream=None) -> torch.Tensor:
    """FP64 model velocities of a ragged batch, laid out like t
    (kc_rv_predict_ragged).  par_off/obs_off: int64, n_pl: int32 CUDA tensors."""
    params = _dev_f64("params", params, 1)
    t = _dev_f64("t", t, 1)
    par_off = par_off.to(device=params.device, dtype=torch.int64).contiguous()
    obs_off = obs_off.to(device=params.device, dtype=torch.int64).contiguous()
    n_pl = n_pl.to(device=params.device, dtype=torch.int32).contiguous()
    if out is None:
        out = torch.empty_like(t)
    lib = _lib.load()
    _lib.check(lib.kc_rv_predict_ragged(params.data_ptr(), par_off.data_ptr(), n_pl.data_ptr(),
                                        t.data_ptr(), obs_off.data_ptr(), n_pl.numel(),
                                        float(t0), out.data_ptr(), _stream(stream)),
               "kc_rv_predict_ragged")
    return out


def kc_kepler_solve(M, e, mode="fp64", out=None, stream=None) -> torch.Tensor:
    """Elementwise E with E - e sin E = M (kc_kepler_solve)."""
    m = _mode(mode)
    dtype = torch.float64 if m == KC_FP64 else torch.float32
    for name, x in (("M", M), ("e", e)):
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != dtype:
            raise TypeError(f"{name} must be a {dtype} CUDA tensor")
    M, e = M.contiguous(), e.contiguous()
    if M.shape != e.shape:
        raise ValueError("M and e must have the same shape")
    if out is None:
        out = torch.empty_like(M)
    lib = _lib.load()
    _lib.check(lib.kc_kepler_solve(M.data_ptr(), e.data_ptr(), M.numel(), m, out.data_ptr(),
                                   _stream(stream)), "kc_kepler_solve")
    return out


def _kernel(kernel) -> int:
    if kernel in (_lib.KC_KERNEL_CHI2, "chi2"):
        return _lib.KC_KERNEL_CHI2
    if kernel in (_lib.KC_KERNEL_GRAD, "grad"):
        return _lib.KC_KERNEL_GRAD
    if kernel in (_lib.KC_KERNEL_GN, "gn"):
        return _lib.KC_KERNEL_GN
    raise ValueError(f"unknown kernel {kernel!r}: use 'chi2', 'grad' or 'gn'")


def kc_autotune(params, t, v_obs, sigma, kernel="chi2", mode="mixed", stream=None):
    """Time every admissible tile on this problem, keep the fastest for
    problems of its size class; returns ((threads_per_system, block, split),
    ms)."""
    params = _dev_f64("params", params, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    best = _lib.KcTile()
    ms = ctypes.c_float()
    lib = _lib.load()
    _lib.check(lib.kc_autotune(params.data_ptr(), t.data_ptr(), v_obs.data_ptr(),
                               sigma.data_ptr(), params.shape[0], n_planets(params), t.numel(),
                               _kernel(kernel), _mode(mode), ctypes.byref(best),
                               ctypes.byref(ms), _stream(stream)), "kc_autotune")
    return (best.threads_per_system, best.block, best.split), ms.value


def kc_set_tile(kernel, mode, n_sys: int, n_pl: int, n_obs: int, tile=None) -> None:
    """Pin (threads_per_system, block[, split]) for a size class; None
    restores the default."""
    lib = _lib.load()
    ptr = None
    if tile is not None:
        split = int(tile[2]) if len(tile) > 2 else 0
        ptr = ctypes.byref(_lib.KcTile(int(tile[0]), int(tile[1]), split))
    _lib.check(lib.kc_set_tile(_kernel(kernel), _mode(mode), n_sys, n_pl, n_obs, ptr),
               "kc_set_tile")


def kc_get_tile(kernel, mode, n_sys: int, n_pl: int, n_obs: int):
    """(threads_per_system, block, split) the library would launch."""
    lib = _lib.load()
    t = _lib.KcTile()
    _lib.check(lib.kc_get_tile(_kernel(kernel), _mode(mode), n_sys, n_pl, n_obs,
                               ctypes.byref(t)), "kc_get_tile")
    return t.threads_per_system, t.block, t.split


class RaggedPlan:
    """Ragged batch (include/kc.h: kc_plan_*): systems with their own planet
    count and observations, evaluated by one persistent, graph-replayed
    kernel.  ``obs_off`` [n_sys+1] and ``n_pl`` [n_sys] are host arrays;
    parameters are packed per system (5*n_pl[s]+1 values each)."""

    def __init__(self, obs_off, n_pl, t0: float = 0.0, jitter: float = 0.0, mode="mixed",
                 want_grad: bool = False):
        import numpy as np
        self._obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
        self._n_pl = np.ascontiguousarray(n_pl, dtype=np.int32)
        self.n_sys = int(self._n_pl.size)
        self.mode = _mode(mode)
        self.want_grad = bool(want_grad)
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self._lib.kc_plan_create_ragged(
            ctypes.byref(h), self._obs_off.ctypes.data, self._n_pl.ctypes.data, self.n_sys,
            float(t0), float(jitter), self.mode, int(self.want_grad)), "kc_plan_create_ragged")
        self._h = h
        n_par, n_obs = ctypes.c_int64(), ctypes.c_int64()
        _lib.check(self._lib.kc_plan_sizes(h, ctypes.byref(n_par), ctypes.byref(n_obs)),
                   "kc_plan_sizes")
        self.n_params, self.n_obs = n_par.value, n_obs.value
        self._keep = None

    @property
    def dtype(self):
        return torch.float64 if self.mode == KC_FP64 else torch.float32

    def set_observations(self, t, v_obs, sigma, stream=None) -> None:
        t, v_obs, sigma = _obs(t, v_obs, sigma)
        if t.numel() != self.n_obs:
            raise ValueError(f"expected {self.n_obs} observations, got {t.numel()}")
        _lib.check(self._lib.kc_plan_set_observations(
            self._h, t.data_ptr(), v_obs.data_ptr(), sigma.data_ptr(), _stream(stream)),
            "kc_plan_set_observations")
        self._keep = (t, v_obs, sigma)

    def _outputs(self, params, chi2_out, grad_out):
        params = _dev_f64("params", params, 1)
        if params.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} packed parameters")
        if chi2_out is None:
            chi2_out = torch.empty(self.n_sys, dtype=self.dtype, device=params.device)
        if self.want_grad and grad_out is None:
            grad_out = torch.empty(self.n_params, dtype=self.dtype, device=params.device)
        return params, chi2_out, grad_out

    def run(self, params, chi2_out=None, grad_out=None, stream=None):
        """chi2 [n_sys] (and the packed gradient if the plan wants it)."""
        params, chi2_out, grad_out = self._outputs(params, chi2_out, grad_out)
        _lib.check(self._lib.kc_plan_run(self._h, params.data_ptr(), chi2_out.data_ptr(),
                                         _ptr(grad_out), _stream(stream)), "kc_plan_run")
        return (chi2_out, grad_out) if self.want_grad else chi2_out

    def autotune(self, params, stream=None):
        """Pick the persistent launch shape; returns (block, ctas_per_sm)."""
        params, chi2_out, grad_out = self._outputs(params, None, None)
        b, k = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(self._lib.kc_plan_autotune(self._h, params.data_ptr(), chi2_out.data_ptr(),
                                              _ptr(grad_out), ctypes.byref(b), ctypes.byref(k),
                                              _stream(stream)), "kc_plan_autotune")
        return b.value, k.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.kc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kc_demcmc_step(states, chi2, t, v_obs, sigma, first: int, count: int,
                   partner_first: int, partner_count: int, gamma: float, eps_scale, z, u,
                   proposals=None, chi2_prop=None, accepted=None, t0: float = 0.0,
                   jitter: float = 0.0, mode="mixed", stream=None):
    """One DE-MC step of chains first .. first+count-1 in place, partners
    drawn from chains partner_first .. partner_first+partner_count-1
    (kc_demcmc_step).  states: float64 [n_chains, 5*n_pl+1]; chi2: float32
    ('mixed') or float64 ('fp64') [n_chains]; eps_scale float64
    [5*n_pl+1]; z float64 [count, 5*n_pl+1] standard normal draws; u
    float64 [count, 3] uniform draws in [0, 1).  Returns accepted (int32
    [count])."""
    states = _dev_f64("states", states, 2)
    t, v_obs, sigma = _obs(t, v_obs, sigma)
    m = _mode(mode)
    dtype = torch.float64 if m == KC_FP64 else torch.float32
    if chi2.dtype != dtype or not chi2.is_cuda:
        raise TypeError(f"chi2 must be a {dtype} CUDA tensor")
    n_pl = n_planets(states)
    npar = 5 * n_pl + 1
    eps_scale = _dev_f64("eps_scale", eps_scale, 1)
    z = _dev_f64("z", z, 2)
    u = _dev_f64("u", u, 2)
    if eps_scale.numel() != npar or z.shape != (count, npar) or u.shape != (count, 3):
        raise ValueError("eps_scale, z and u must be [n_par], [count, n_par] and [count, 3]")
    if proposals is None:
        proposals = torch.empty((count, npar), dtype=torch.float64, device=states.device)
    if chi2_prop is None:
        chi2_prop = torch.empty(count, dtype=dtype, device=states.device)
    if accepted is None:
        accepted = torch.empty(count, dtype=torch.int32, device=states.device)
    lib = _lib.load()
    _lib.check(lib.kc_demcmc_step(
        states.data_ptr(), chi2.data_ptr(), states.shape[0], n_pl, t.data_ptr(),
        v_obs.data_ptr(), sigma.data_ptr(), t.numel(), float(t0), float(jitter), m, int(first),
        int(count), int(partner_first), int(partner_count), float(gamma), eps_scale.data_ptr(),
        z.data_ptr(), u.data_ptr(), proposals.data_ptr(), chi2_prop.data_ptr(),
        accepted.data_ptr(), _stream(stream)),
        "kc_demcmc_step")
    return accepted


class DEMCMC:
    """Differential-evolution MCMC (ter Braak 2006) over a population of
    model systems on the GPU, chi2 as -2 ln L (flat prior).

    Each generation updates the two halves of the population in turn, every
    chain of a half proposing x + gamma (x_r1 - x_r2) + eps with r1 != r2
    from the other half; gamma = 2.38/sqrt(2 d) except every ``hop_every``-th
    generation where gamma = 1 (jumps between modes); eps ~ N(0, eps_scale^2
    x^2) per parameter (``eps_scale`` a number or one value per parameter; 0
    together with equal values in every chain holds a parameter fixed).
    Random draws come from a torch generator on the device; the step itself
    is kc_demcmc_step.  The draws do not depend on the chains, so they are
    made ``draw_batch`` generations at a time, for the next batch on a side
    stream while the current batch steps (two buffers), in the same order
    whether the generations run eagerly or from a CUDA graph; the
    acceptances of a batch are tallied once, with the next batch's draws.
    ``autotune``: time the chi2 tiles once for the size class of half the
    population (what each step evaluates) and keep the fastest; off by
    default, since the pick depends on timing and so can change the
    summation order from one run to the next."""

    def __init__(self, states, t, v_obs, sigma, t0: float = 0.0, jitter: float = 0.0,
                 mode="mixed", eps_scale: float = 1e-6, hop_every: int = 10, seed: int = 0,
                 autotune: bool = False, draw_batch: int = 8):
        self.states = _dev_f64("states", states, 2).clone()
        n = self.states.shape[0]
        if n < 8 or n % 2:
            raise ValueError("DEMCMC needs an even population of at least 8 chains")
        self.t, self.v, self.sigma = _obs(t, v_obs, sigma)
        self.t0, self.jitter, self.mode = float(t0), float(jitter), mode
        self.npar = self.states.shape[1]
        self.half = n // 2
        if draw_batch < 1:
            raise ValueError("draw_batch must be at least 1")
        self.batch = int(draw_batch)
        self.gamma = 2.38 / (2.0 * self.npar) ** 0.5
        self.eps_scale = torch.as_tensor(eps_scale, dtype=torch.float64,
                                         device=self.states.device).expand(self.npar).clone()
        self.hop_every = int(hop_every)
        self.gen = torch.Generator(device=self.states.device)
        self.gen.manual_seed(seed)
        if autotune:
            kc_autotune(self.states[:self.half], self.t, self.v, self.sigma, kernel="chi2",
                        mode=mode)
        self.chi2 = kc_chi2_eval_ex(self.states, self.t, self.v, self.sigma, self.t0,
                                    self.jitter, mode)
        dev = self.states.device
        self._prop = torch.empty((self.half, self.npar), dtype=torch.float64, device=dev)
        self._cp = torch.empty(self.half, dtype=self.chi2.dtype, device=dev)
        self.generation = 0
        # accepted flags per generation slot of a batch (two buffers),
        # tallied per chain once a batch, on the side stream, while the
        # next batch steps
        G = self.batch
        self._acc = [torch.zeros((G, n), dtype=torch.int32, device=dev) for _ in (0, 1)]
        self._n_acc = torch.zeros(n, dtype=torch.int64, device=dev)
        self.proposed = 0
        self._graph = None
        self._side = torch.cuda.Stream(device=dev)
        self._z32 = torch.empty((G, n, self.npar), dtype=torch.float32, device=dev)
        self._z = [torch.empty((G, n, self.npar), dtype=torch.float64, device=dev)
                   for _ in (0, 1)]
        self._u = [torch.empty((G, n, 3), dtype=torch.float64, device=dev) for _ in (0, 1)]
        self._buf = 0                    # the buffer holding the current batch's draws
        self._slot = 0                   # the next generation's slot in it
        self._draws(0)

    def _draws(self, b: int) -> None:
        """Every random number of one batch of generations (both halves)
        into buffer b: standard normal perturbations and three uniforms per
        chain (acceptance, two partners) for each generation; the step
        kernels scale and map them.  The normals are drawn in single
        precision (a perturbation needs no more; double precision normals
        cost 27 us a generation on this GPU, these 15) and widened."""
        torch.randn(self._z32.shape, generator=self.gen, out=self._z32)
        self._z[b].copy_(self._z32)
        torch.rand(self._u[b].shape, generator=self.gen, out=self._u[b])

    def _generation(self, gamma: float) -> None:
        cur, k = self._buf, self._slot
        main = torch.cuda.current_stream(self.states.device)
        if k == 0:
            # a new batch: the other buffer (last used by the previous
            # batch's steps) takes the next batch's draws, after its flags
            # are tallied
            nxt = 1 - cur
            self._side.wait_stream(main)
            with torch.cuda.stream(self._side):
                self._n_acc += self._acc[nxt].sum(dim=0)
                self._draws(nxt)
        z, u, acc = self._z[cur][k], self._u[cur][k], self._acc[cur][k]
        h = self.half
        for first, other in ((0, h), (h, 0)):
            kc_demcmc_step(self.states, self.chi2, self.t, self.v, self.sigma, first, h, other, h,
                           gamma, self.eps_scale, z[first:first + h], u[first:first + h],
                           self._prop, self._cp, acc[first:first + h], self.t0,
                           self.jitter, self.mode)
        self._slot = k + 1
        if self._slot == self.batch:
            main.wait_stream(self._side)           # the next batch's draws are made
            self._slot = 0
            self._buf = 1 - cur

    def _gamma(self, ahead: int = 1) -> float:
        hop = self.hop_every and (self.generation + ahead) % self.hop_every == 0
        return 1.0 if hop else self.gamma

    def step(self) -> None:
        """One generation (both halves)."""
        self._generation(self._gamma())
        self.proposed += 2 * self.half
        self.generation += 1

    def run(self, generations: int, use_graph: bool = True) -> None:
        """``generations`` generations; with use_graph, two batches of
        generations (one on each draw buffer) are captured into a CUDA
        graph, random draws included, and replayed, which removes the
        per-launch host overhead for small populations.  The first
        generation, and the generations of any two batches that hold a
        gamma = 1 generation or would be cut short, run eagerly."""
        span = 2 * self.batch
        while generations > 0:
            whole = (use_graph and generations >= span and self.generation > 0
                     and self._buf == 0 and self._slot == 0
                     and all(self._gamma(i) == self.gamma for i in range(1, span + 1)))
            if not whole:
                self.step()
                generations -= 1
                continue
            if self._graph is None:
                self._capture()
            self._graph.replay()
            self.generation += span
            self.proposed += 2 * span * self.half
            generations -= span

    def _capture(self) -> None:
        dev = self.states.device
        torch.cuda.synchronize(dev)
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(torch.cuda.current_stream(dev))
        g = torch.cuda.CUDAGraph()
        g.register_generator_state(self.gen)              # replays advance self.gen
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g, stream=cap):
                for _ in range(2 * self.batch):            # buffer 0's batch, then 1's:
                    self._generation(self.gamma)           # back to buffer 0, slot 0
        torch.cuda.current_stream(dev).wait_stream(cap)
        self._graph = g

    @property
    def acceptance(self) -> float:
        """Fraction of accepted proposals so far (synchronises): the tallied
        batches, the flags of the batch before the current one when its
        tally is still to come (the current batch has not begun), and the
        current batch's generations so far."""
        torch.cuda.synchronize(self.states.device)
        total = int(self._n_acc.sum()) + int(self._acc[self._buf][:self._slot].sum())
        if self._slot == 0 and self.generation > 0:
            total += int(self._acc[1 - self._buf].sum())
        return total / max(self.proposed, 1)


class _Chi2Fn(torch.autograd.Function):
    """chi2 with the adjoint kernel as backward."""

    @staticmethod
    def forward(ctx, params, t, v_obs, sigma, t0, jitter, mode):
        chi, grad = kc_chi2_grad(params, t, v_obs, sigma, t0, jitter, mode)
        ctx.save_for_backward(grad)
        return chi

    @staticmethod
    def backward(ctx, grad_chi2):
        (grad,) = ctx.saved_tensors
        g = grad.to(torch.float64) * grad_chi2.to(torch.float64)[:, None]
        return g, None, None, None, None, None, None


class _NllFn(torch.autograd.Function):
    """Free-jitter nll with the adjoint kernel as backward."""

    @staticmethod
    def forward(ctx, params, t, v_obs, sigma, t0, mode):
        val, grad = kc_nll_grad(params, t, v_obs, sigma, t0, mode)
        ctx.save_for_backward(grad)
        return val

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return (grad.to(torch.float64) * grad_out.to(torch.float64)[:, None],
                None, None, None, None, None)


def nll(params, t, v_obs, sigma, t0: float = 0.0, mode="mixed") -> torch.Tensor:
    """Differentiable free-jitter negative log-likelihood [n_sys]."""
    if params.requires_grad and torch.is_grad_enabled():
        return _NllFn.apply(params, t, v_obs, sigma, float(t0), mode)
    return kc_nll_eval(params, t, v_obs, sigma, t0, mode)


def chi2(params, t, v_obs, sigma, t0: float = 0.0, jitter: float = 0.0,
         mode="mixed") -> torch.Tensor:
    """Differentiable chi2 [n_sys] with respect to ``params``.

    Without grad, the forward kernel (kc_chi2_eval_ex) runs; with grad the
    adjoint kernel (kc_chi2_grad) produces chi2 and its gradient in one pass
    and backward scales it by the incoming gradient."""
    if params.requires_grad and torch.is_grad_enabled():
        return _Chi2Fn.apply(params, t, v_obs, sigma, float(t0), float(jitter), mode)
    return kc_chi2_eval_ex(params, t, v_obs, sigma, t0, jitter, mode)
