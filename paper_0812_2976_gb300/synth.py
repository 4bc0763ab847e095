"""Seeded synthetic workloads shaped like the paper's benchmarks.

The paper's radial-velocity data set is not available, so these generators
stand in for it.  They follow the parameter distributions of Table 2 (periods
and amplitudes log-uniform, eccentricity and angles uniform, n_pl = 4,
n_obs = 256) and the five workload shapes this package is measured on.

This module draws random numbers only.  It evaluates no part of the
Keplerian model: the observed velocities are ``truth model + noise`` and the
caller forms the truth-model velocities with whichever implementation it is
testing or timing (the FP64 CPU oracle in the tests, ``kc.rv_predict`` on the
GPU in the benchmark), then adds ``noise``.

Parameter layout of one system: (P, K, e, omega, M0) per planet, then the
offset gamma.  Units: days, m/s, radians.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 20081209
EPOCH = 2450000.0
TWO_PI = 2.0 * np.pi


@dataclass(frozen=True)
class Shape:
    name: str
    n_sys: int
    n_pl: int
    n_obs: int
    span: float            # days covered by the observations
    p_range: tuple         # log-uniform period range (days)
    k_range: tuple         # log-uniform amplitude range (m/s)
    e_max: float           # truth eccentricity ~ U[0, e_max)
    rel_perturb: float     # model = truth * (1 + rel_perturb * N(0,1))
    e_clip: float          # model eccentricities clipped to [0, e_clip]
    sort_periods: bool
    t0: float              # epoch of M0 passed to the evaluator
    description: str = ""


# The five workload shapes.  0-3 share one star's observations across every
# model system; 4 is ragged (own observations and planet count per system).
SHAPES = {
    0: Shape("fp64-small", 64, 1, 32, 2000.0, (2.0, 1000.0), (1.0, 100.0),
             0.8, 1e-2, 0.95, False, 0.0,
             "plain FP64 chi2: n_sys=64, n_pl=1, n_obs=32"),
    1: Shape("paper-batch", 4096, 4, 256, 4000.0, (1.0, 4000.0), (1.0, 100.0),
             0.8, 1e-2, 0.95, True, 0.0,
             "paper-shaped batch: n_sys=4096, n_pl=4, n_obs=256"),
    2: Shape("grid-sweep", 1 << 20, 4, 256, 4000.0, (1.0, 4000.0),
             (1.0, 100.0), 0.95, 1e-1, 0.95, True, 0.0,
             "large grid sweep: n_sys=2^20, n_pl=4, n_obs=256, e<=0.95"),
    3: Shape("gradient", 65536, 3, 512, 4000.0, (1.0, 4000.0), (1.0, 100.0),
             0.8, 1e-2, 0.95, True, EPOCH,
             "gradient: n_sys=65536, n_pl=3, n_obs=512, t0=2450000"),
}


@dataclass
class UniformWorkload:
    """Systems sharing one star's observations (configs 0-3)."""
    shape: Shape
    t: np.ndarray          # [n_obs] absolute times (days)
    sigma: np.ndarray      # [n_obs] measurement uncertainties (m/s)
    noise: np.ndarray      # [n_obs] N(0, sigma^2) draws
    truth: np.ndarray      # [5*n_pl+1] parameters that generate the data
    params: np.ndarray     # [n_sys, 5*n_pl+1] model systems to evaluate
    t0: float = 0.0
    jitter: float = 0.0

    @property
    def n_sys(self) -> int:
        return self.params.shape[0]

    @property
    def n_pl(self) -> int:
        return self.shape.n_pl

    @property
    def n_obs(self) -> int:
        return self.t.size


def _draw_planets(rng, n, n_pl, sh: Shape, e_max=None):
    """[n, n_pl, 5] truth-like draws of (P, K, e, omega, M0)."""
    e_max = sh.e_max if e_max is None else e_max
    lp = rng.uniform(np.log(sh.p_range[0]), np.log(sh.p_range[1]), (n, n_pl))
    P = np.exp(lp)
    if sh.sort_periods:
        P = np.sort(P, axis=1)
    K = np.exp(rng.uniform(np.log(sh.k_range[0]), np.log(sh.k_range[1]),
                           (n, n_pl)))
    e = rng.uniform(0.0, e_max, (n, n_pl))
    w = rng.uniform(0.0, TWO_PI, (n, n_pl))
    M0 = rng.uniform(0.0, TWO_PI, (n, n_pl))
    return np.stack([P, K, e, w, M0], axis=-1)


def _perturb(rng, truth_rows: np.ndarray, n_pl: int, rel: float,
             e_clip: float) -> np.ndarray:
    """model = truth * (1 + rel * N(0,1)) per parameter; then clip."""
    m = truth_rows * (1.0 + rel * rng.standard_normal(truth_rows.shape))
    _clip_rows(m, n_pl, e_clip)
    return m


def _clip_rows(m: np.ndarray, n_pl: int, e_clip: float) -> None:
    """In place, on rows laid out (P, K, e, omega, M0)*n_pl + gamma."""
    end = 5 * n_pl
    m[:, 0:end:5] = np.maximum(m[:, 0:end:5], 1e-3)             # P > 0
    m[:, 1:end:5] = np.maximum(m[:, 1:end:5], 0.0)              # K >= 0
    m[:, 2:end:5] = np.clip(m[:, 2:end:5], 0.0, e_clip)         # e range


def uniform(cfg: int, n_sys: Optional[int] = None,
            seed: Optional[int] = None) -> UniformWorkload:
    """Workload of config ``cfg`` (0-3).  ``n_sys`` truncates the batch: the
    first n systems are identical to the first n of the full batch."""
    sh = SHAPES[cfg]
    rng = np.random.default_rng(SEED_BASE + cfg if seed is None else seed)
    t = np.sort(rng.uniform(EPOCH, EPOCH + sh.span, sh.n_obs))
    sigma = rng.uniform(1.0, 5.0, sh.n_obs)
    noise = sigma * rng.standard_normal(sh.n_obs)
    planets = _draw_planets(rng, 1, sh.n_pl, sh)[0]
    gamma = rng.uniform(-10.0, 10.0)
    truth = np.concatenate([planets.ravel(), [gamma]])
    full = sh.n_sys
    rows = np.broadcast_to(truth, (full, truth.size)).copy()
    params = _perturb(rng, rows, sh.n_pl, sh.rel_perturb, sh.e_clip)
    if n_sys is not None:
        params = params[:n_sys].copy()
    return UniformWorkload(sh, t, sigma, noise, truth, params, t0=sh.t0)


@dataclass
class RaggedWorkload:
    """Systems with their own planet count and observations (config 4)."""
    n_pl: np.ndarray       # [n_sys] int32, 1..6
    par_off: np.ndarray    # [n_sys+1] int64 offsets into params
    params: np.ndarray     # [par_off[-1]] model parameters
    truth: np.ndarray      # [par_off[-1]] generating parameters
    obs_off: np.ndarray    # [n_sys+1] int64 offsets into t/sigma/noise
    t: np.ndarray          # [obs_off[-1]] absolute times
    sigma: np.ndarray
    noise: np.ndarray
    t0: float = 0.0
    jitter: float = 0.0

    @property
    def n_sys(self) -> int:
        return self.n_pl.size

    def evals(self) -> int:
        """Planet-observation evaluations: sum_s n_pl[s] * n_obs[s]."""
        return int(np.sum(self.n_pl.astype(np.int64) * np.diff(self.obs_off)))


RAGGED_N_SYS = 200000


def _sorted_uniform_segments(rng, n_obs: np.ndarray) -> np.ndarray:
    """Concatenated sorted U[0,1) samples, n_obs[s] of them per segment.

    The order statistics of n uniforms are the first n partial sums of n+1
    exponential draws divided by their total, which avoids a sort."""
    seg = n_obs.astype(np.int64) + 1
    ends = np.cumsum(seg)
    starts = ends - seg
    ex = rng.standard_exponential(int(ends[-1])) if ends.size else np.zeros(0)
    cs = np.cumsum(ex)
    base = np.where(starts > 0, cs[np.maximum(starts - 1, 0)], 0.0)
    seg_id = np.repeat(np.arange(n_obs.size), seg)
    within = cs - base[seg_id]
    total = within[ends - 1]
    u = within / total[seg_id]
    keep = np.ones(u.size, dtype=bool)
    keep[ends - 1] = False
    return np.minimum(u[keep], np.nextafter(1.0, 0.0))


def ragged(n_sys: int = RAGGED_N_SYS, seed: Optional[int] = None,
           obs_range=(16, 1024), pl_range=(1, 6),
           span_range=(500.0, 6000.0)) -> RaggedWorkload:
    """Config 4: n_obs ~ U[16, 1024], n_pl ~ U{1..6}, each system with its own
    times EPOCH + sorted U[0, span], span ~ U[500, 6000] days; parameter
    distributions as config 1 and 1% model perturbation."""
    sh = SHAPES[1]
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    n_pl = rng.integers(pl_range[0], pl_range[1] + 1, n_sys).astype(np.int32)
    n_obs = rng.integers(obs_range[0], obs_range[1] + 1, n_sys).astype(np.int64)
    span = rng.uniform(span_range[0], span_range[1], n_sys)
    obs_off = np.zeros(n_sys + 1, dtype=np.int64)
    np.cumsum(n_obs, out=obs_off[1:])
    n_tot = int(obs_off[-1])
    t = EPOCH + _sorted_uniform_segments(rng, n_obs) * np.repeat(span, n_obs)
    sigma = rng.uniform(1.0, 5.0, n_tot)
    noise = sigma * rng.standard_normal(n_tot)
    n_par = 5 * n_pl.astype(np.int64) + 1
    par_off = np.zeros(n_sys + 1, dtype=np.int64)
    np.cumsum(n_par, out=par_off[1:])
    maxpl = pl_range[1]
    planets = _draw_planets(rng, n_sys, maxpl, sh)       # [n_sys, 6, 5]
    gamma = rng.uniform(-10.0, 10.0, n_sys)
    pert = 1.0 + sh.rel_perturb * rng.standard_normal((n_sys, 5 * maxpl + 1))
    truth = np.empty(int(par_off[-1]))
    params = np.empty_like(truth)
    for J in range(pl_range[0], pl_range[1] + 1):
        idx = np.nonzero(n_pl == J)[0]
        if idx.size == 0:
            continue
        # periods of a J-planet system: the J draws, sorted
        pj = planets[idx, :J, :].copy()
        pj[..., 0] = np.sort(pj[..., 0], axis=1)
        rows = np.concatenate([pj.reshape(idx.size, 5 * J),
                               gamma[idx, None]], axis=1)
        m = rows * np.concatenate([pert[idx, :5 * J], pert[idx, -1:]], axis=1)
        _clip_rows(m, J, sh.e_clip)
        cols = par_off[idx, None] + np.arange(5 * J + 1)[None, :]
        truth[cols] = rows
        params[cols] = m
    return RaggedWorkload(n_pl, par_off, params, truth, obs_off, t, sigma,
                          noise)


def subset_ragged(w: RaggedWorkload, idx: np.ndarray) -> RaggedWorkload:
    """The systems ``idx`` of a ragged workload, repacked."""
    idx = np.asarray(idx, dtype=np.int64)
    n_pl = w.n_pl[idx]
    n_par = 5 * n_pl.astype(np.int64) + 1
    par_off = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(n_par, out=par_off[1:])
    n_obs = (w.obs_off[idx + 1] - w.obs_off[idx])
    obs_off = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(n_obs, out=obs_off[1:])
    pcols = np.concatenate([np.arange(w.par_off[s], w.par_off[s + 1])
                            for s in idx]) if idx.size else np.zeros(0, np.int64)
    ocols = np.concatenate([np.arange(w.obs_off[s], w.obs_off[s + 1])
                            for s in idx]) if idx.size else np.zeros(0, np.int64)
    return RaggedWorkload(n_pl, par_off, w.params[pcols], w.truth[pcols],
                          obs_off, w.t[ocols], w.sigma[ocols], w.noise[ocols],
                          w.t0, w.jitter)


def pad_ragged(w: RaggedWorkload, v_obs: np.ndarray, n_pl: Optional[int] = None,
               n_obs: Optional[int] = None):
    """The same batch padded to a uniform size: every system gets n_pl
    planets (the added ones with K = 0, so they contribute nothing) and n_obs
    observations (the added ones with sigma = inf, i.e. zero weight).
    Returns (padded workload, padded v_obs)."""
    J = int(w.n_pl.max()) if n_pl is None else int(n_pl)
    cnt = np.diff(w.obs_off)
    N = int(cnt.max()) if n_obs is None else int(n_obs)
    S = w.n_sys
    npar = 5 * J + 1
    params = np.zeros((S, npar))
    truth = np.zeros((S, npar))
    params[:, 0:5 * J:5] = 1.0                # P = 1 d for the empty planets
    truth[:, 0:5 * J:5] = 1.0
    for Jo in np.unique(w.n_pl):
        idx = np.nonzero(w.n_pl == Jo)[0]
        cols = w.par_off[idx, None] + np.arange(5 * Jo + 1)[None, :]
        params[idx, :5 * Jo] = w.params[cols[:, :5 * Jo]]
        params[idx, -1] = w.params[cols[:, -1]]
        truth[idx, :5 * Jo] = w.truth[cols[:, :5 * Jo]]
        truth[idx, -1] = w.truth[cols[:, -1]]
    t = np.empty((S, N))
    sg = np.full((S, N), np.inf)
    vv = np.zeros((S, N))
    nz = np.zeros((S, N))
    k = np.arange(N)[None, :]
    valid = k < cnt[:, None]
    src = w.obs_off[:-1, None] + np.minimum(k, np.maximum(cnt[:, None] - 1, 0))
    has = cnt[:, None] > 0
    t[:] = np.where(has, w.t[np.minimum(src, max(w.t.size - 1, 0))], EPOCH)
    sg[valid] = w.sigma[src[valid]]
    vv[valid] = v_obs[src[valid]]
    nz[valid] = w.noise[src[valid]]
    out = RaggedWorkload(np.full(S, J, np.int32), np.arange(S + 1, dtype=np.int64) * npar,
                         params.ravel(), truth.ravel(), np.arange(S + 1, dtype=np.int64) * N,
                         t.ravel(), sg.ravel(), nz.ravel(), w.t0, w.jitter)
    return out, vv.ravel()
