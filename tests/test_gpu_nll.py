"""Free-jitter negative log-likelihood (kc_nll_eval / kc_nll_grad) vs the FP64
CPU oracle, through the C ABI.  Tolerances as for chi2 (relative to
max(|nll|, 1)); gradient per component normalised by max(|g|, 1e-3 |g|),
plus the sum's cancellation term (tests/tolerance.py)."""
import numpy as np
import pytest
import torch
from tolerance import U32, U64, grad_excess, uniform_arith

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5
GRAD_MIXED_TOL = 1e-3
GRAD_F64_TOL = 1e-9


@pytest.fixture(scope="module")
def kc():
    import paper_0812_2976_gb300 as kc
    from paper_0812_2976_gb300 import build
    build.build()
    kc._lib.load()
    return kc


def dev(*arrs):
    return [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
            for a in arrs]


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1.0)


def grad_err(got, ref, gabs, mode="mixed", arith=None):
    """Largest error of a gradient component over its bound (<= 1 passes);
    arith: how the kernel formed and summed it (tests/tolerance.py)."""
    rel, u = (GRAD_MIXED_TOL, U32) if mode == "mixed" else (GRAD_F64_TOL, U64)
    return grad_excess(got, ref, gabs, rel, u, arith)


def workload(oracle_mod, n_sys=3000, seed=21):
    """Config-3-shaped data (n_pl 3, n_obs 512, t0 = 2450000) with a jitter
    of its own for every model system."""
    from paper_0812_2976_gb300 import synth
    w = synth.uniform(3, n_sys=n_sys)
    v = oracle_mod.predict(w.truth, w.t, w.n_pl, w.t0)[0] + w.noise
    rng = np.random.default_rng(seed)
    params = np.concatenate([w.params, rng.uniform(0.0, 5.0, (n_sys, 1))], axis=1)
    return w, v, params


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_nll_and_gradient_vs_oracle(kc, oracle_mod, mode):
    w, v, params = workload(oracle_mod)
    ref, gref, gabs = oracle_mod.nll(params, w.t, v, w.sigma, w.n_pl, t0=w.t0, gabs=True)
    P, T, V, S = dev(params, w.t, v, w.sigma)
    tol = MIXED_TOL if mode == "mixed" else FP64_TOL
    got = kc.kc_nll_eval(P, T, V, S, t0=w.t0, mode=mode).cpu().numpy()
    assert rel_err(got, ref).max() <= tol
    val, g = kc.kc_nll_grad(P, T, V, S, t0=w.t0, mode=mode)
    assert rel_err(val.cpu().numpy(), ref).max() <= tol
    ar = uniform_arith(kc, oracle_mod, params, w.t, v, w.sigma, w.n_pl, w.t0, 0.0, mode, "nll")
    assert grad_err(g.cpu().numpy(), gref, gabs, mode, ar) <= 1.0


@pytest.mark.parametrize("n_pl", [1, 4, 7])
def test_nll_planet_counts_and_invalid(kc, oracle_mod, n_pl):
    rng = np.random.default_rng(30 + n_pl)
    n_sys, n_obs = 333, 211
    cols = []
    for _ in range(n_pl):
        cols += [np.exp(rng.uniform(0, np.log(4000), n_sys)), rng.uniform(1, 100, n_sys),
                 rng.uniform(0, 0.9, n_sys), rng.uniform(0, 2 * np.pi, n_sys),
                 rng.uniform(0, 2 * np.pi, n_sys)]
    params = np.stack(cols + [rng.uniform(-10, 10, n_sys), rng.uniform(-4, 4, n_sys)], axis=1)
    params[5, -1] = np.nan                       # invalid jitter
    t = np.sort(rng.uniform(2450000, 2455000, n_obs))
    v = rng.normal(0, 40, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    ref, gref, gabs = oracle_mod.nll(params, t, v, sig, n_pl, gabs=True)
    P, T, V, S = dev(params, t, v, sig)
    ok = np.setdiff1d(np.arange(n_sys), [5])
    for mode, tol in (("mixed", MIXED_TOL), ("fp64", FP64_TOL)):
        got = kc.kc_nll_eval(P, T, V, S, mode=mode).cpu().numpy()
        assert np.isnan(got[5]) and rel_err(got[ok], ref[ok]).max() <= tol
    _, g = kc.kc_nll_grad(P, T, V, S, mode="fp64")
    g = g.cpu().numpy()
    ar = uniform_arith(kc, oracle_mod, params[ok], t, v, sig, n_pl, 0.0, 0.0, "fp64", "nll",
                       n_sys_launch=n_sys)
    assert np.all(np.isnan(g[5])) and grad_err(g[ok], gref[ok], gabs[ok], "fp64", ar) <= 1.0
    # Gradients in single precision at the gradient workload's epoch as well
    # (with t0 = 0 the cancellation term dominates the period components).
    for t0 in (0.0, 2450000.0):
        ref, gref, gabs = oracle_mod.nll(params, t, v, sig, n_pl, t0=t0, gabs=True)
        for mode, tol in (("mixed", MIXED_TOL), ("fp64", FP64_TOL)):
            val, g = kc.kc_nll_grad(P, T, V, S, t0=t0, mode=mode)
            g = g.cpu().numpy()
            assert rel_err(val.cpu().numpy()[ok], ref[ok]).max() <= tol
            ar = uniform_arith(kc, oracle_mod, params[ok], t, v, sig, n_pl, t0, 0.0, mode, "nll",
                               n_sys_launch=n_sys)
            assert np.all(np.isnan(g[5])) and grad_err(g[ok], gref[ok], gabs[ok], mode, ar) <= 1.0


def test_nll_autograd(kc, oracle_mod):
    w, v, params = workload(oracle_mod, n_sys=64)
    P, T, V, S = dev(params, w.t, v, w.sigma)
    Pg = P.clone().requires_grad_(True)
    kc.nll(Pg, T, V, S, t0=w.t0, mode="fp64").sum().backward()
    _, gref, gabs = oracle_mod.nll(params, w.t, v, w.sigma, w.n_pl, t0=w.t0, gabs=True)
    ar = uniform_arith(kc, oracle_mod, params, w.t, v, w.sigma, w.n_pl, w.t0, 0.0, "fp64", "nll")
    assert grad_err(Pg.grad.cpu().numpy(), gref, gabs, "fp64", ar) <= 1.0
