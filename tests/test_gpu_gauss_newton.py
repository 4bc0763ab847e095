"""Gauss-Newton normal matrix H = sum_k w_k J_k J_k^T with chi2 and its
gradient from one pass (kc_chi2_gauss_newton) against the FP64 oracle.

H entries are compared on the correlation scale: |dH_pq| / sqrt(H_pp H_qq)
(an entry that cancels to ~0 cannot carry relative accuracy).  Tolerances:
the mixed path forms J_k in FP32 (relative error ~1e-6, the period column
~1e-5 through (t - t0)/P^2) and the update on the tensor cores with the
two-term TF32 split by truncation (< 3 * 2^-20 ~ 3e-6 per product), so 1e-4
leaves an order of magnitude; FP64: 1e-10."""
import contextlib

import numpy as np
import pytest
import torch
from tolerance import U32, U64, grad_excess, uniform_arith

pytestmark = pytest.mark.gpu

H_MIXED_TOL = 1e-4
H_F64_TOL = 1e-10
CHI2_MIXED_TOL, CHI2_F64_TOL = 1e-5, 1e-12
GRAD_MIXED_TOL, GRAD_F64_TOL = 1e-3, 1e-9


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


def h_err(got, ref, n):
    import oracle
    G = oracle.unpack_symmetric(np.asarray(got, np.float64), n)
    R = oracle.unpack_symmetric(ref, n)
    d = np.sqrt(np.abs(np.diagonal(R, axis1=1, axis2=2)))
    scale = np.maximum(d[:, :, None] * d[:, None, :], 1e-30)
    return np.abs(G - R) / scale


@contextlib.contextmanager
def gn_variant(kc, split, n_sys, n_pl, n_obs):
    """Runs the mixed Gauss-Newton kernel's U^T U update by mma.sync (split
    0) or tcgen05 (4: four systems stacked in an M = 64 tile) for this size
    class."""
    kc.kc_set_tile("gn", "mixed", n_sys, n_pl, n_obs, (32, 128, split))
    try:
        yield
    finally:
        kc.kc_set_tile("gn", "mixed", n_sys, n_pl, n_obs, None)


def rel(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1.0)


def grad_err(got, ref, gabs, mode="mixed", arith=None):
    """Largest error of a gradient component over its bound (<= 1 passes;
    arith: how the kernel formed and summed it, tests/tolerance.py)."""
    rel, u = (GRAD_MIXED_TOL, U32) if mode == "mixed" else (GRAD_F64_TOL, U64)
    return grad_excess(got, ref, gabs, rel, u, arith)


@pytest.mark.parametrize("mode,split", [("mixed", 0), ("mixed", 4), ("fp64", 0)])
def test_gradient_workload_sampled(kc, oracle_mod, mode, split):
    """Config-3 shapes (n_pl 3, n_obs 512, t0 = 2450000) on 2048 systems;
    mixed with each way of adding U^T U."""
    from paper_0812_2976_gb300 import synth
    w = synth.uniform(3, n_sys=2048)
    v = oracle_mod.predict(w.truth, w.t, w.n_pl, w.t0)[0] + w.noise
    chi_ref, g_ref, g_abs = oracle_mod.chi2(w.params, w.t, v, w.sigma, w.n_pl, t0=w.t0,
                                            gabs=True)
    H_ref = oracle_mod.gauss_newton(w.params, w.t, w.sigma, w.n_pl, t0=w.t0)
    P, T, V, S = dev(w.params, w.t, v, w.sigma)
    ctx = gn_variant(kc, split, 2048, w.n_pl, w.t.size) if mode == "mixed" else \
        contextlib.nullcontext()
    with ctx:
        chi, g, H = kc.kc_chi2_gauss_newton(P, T, V, S, t0=w.t0, mode=mode)
    tol = (CHI2_MIXED_TOL, GRAD_MIXED_TOL, H_MIXED_TOL) if mode == "mixed" else \
        (CHI2_F64_TOL, GRAD_F64_TOL, H_F64_TOL)
    assert rel(chi.cpu().numpy(), chi_ref).max() <= tol[0]
    ar = uniform_arith(kc, oracle_mod, w.params, w.t, v, w.sigma, w.n_pl, w.t0, 0.0, mode, "gn")
    assert grad_err(g.cpu().numpy(), g_ref, g_abs, mode, ar) <= 1.0
    e = h_err(H.cpu().numpy(), H_ref, 5 * w.n_pl + 1)
    assert e.max() <= tol[2], e.max()


@pytest.mark.parametrize("n_pl,n_obs", [(1, 33), (2, 300), (4, 77), (5, 129), (7, 64), (8, 257)])
def test_planet_counts_ragged_tails_invalid(kc, oracle_mod, n_pl, n_obs):
    rng = np.random.default_rng(40 + n_pl)
    n_sys = 37
    cols = []
    for _ in range(n_pl):
        cols += [np.exp(rng.uniform(0, np.log(3000), n_sys)), rng.uniform(1, 80, n_sys),
                 rng.uniform(0, 0.85, n_sys), rng.uniform(0, 2 * np.pi, n_sys),
                 rng.uniform(0, 2 * np.pi, n_sys)]
    par = np.stack(cols + [rng.uniform(-10, 10, n_sys)], axis=1)
    par[4, 2] = 1.5                                   # e > 1: invalid
    t = np.sort(rng.uniform(2450000, 2453000, n_obs))
    v = rng.normal(0, 30, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    t0 = 2450500.0
    chi_ref, g_ref, g_abs = oracle_mod.chi2(par, t, v, sig, n_pl, t0=t0, gabs=True)
    H_ref = oracle_mod.gauss_newton(par, t, sig, n_pl, t0=t0)
    P, T, V, S = dev(par, t, v, sig)
    ok = np.setdiff1d(np.arange(n_sys), [4])
    kc.kc_last_device_error()
    for mode, tol in (("mixed", (CHI2_MIXED_TOL, GRAD_MIXED_TOL, H_MIXED_TOL)),
                      ("fp64", (CHI2_F64_TOL, GRAD_F64_TOL, H_F64_TOL))):
        chi, g, H = kc.kc_chi2_gauss_newton(P, T, V, S, t0=t0, mode=mode)
        chi, g, H = chi.cpu().numpy(), g.cpu().numpy(), H.cpu().numpy()
        assert np.isnan(chi[4]) and np.all(np.isnan(g[4])) and np.all(np.isnan(H[4]))
        assert rel(chi[ok], chi_ref[ok]).max() <= tol[0]
        ar = uniform_arith(kc, oracle_mod, par[ok], t, v, sig, n_pl, t0, 0.0, mode, "gn")
        assert grad_err(g[ok], g_ref[ok], g_abs[ok], mode, ar) <= 1.0
        assert h_err(H[ok], H_ref[ok], 5 * n_pl + 1).max() <= tol[2]
        assert kc.kc_last_device_error() == 1


@pytest.mark.parametrize("split", [4])
@pytest.mark.parametrize("n_pl,n_obs,n_sys", [(1, 33, 37), (2, 300, 9), (3, 1000, 6),
                                              (3, 1, 5), (3, 0, 3), (3, 97, 4097),
                                              (3, 64, 8), (2, 513, 4)])
def test_tcgen05_variants(kc, oracle_mod, split, n_pl, n_obs, n_sys):
    """The tcgen05 form of the U^T U update against the oracle and against
    the mma.sync form, element by element: partial last CTAs (n_sys not a
    multiple of four), a partial last batch of 64 observations (one lane's
    second observation only, or neither), exactly one batch, several
    observation tiles of 512 and many batches through the one operand tile,
    one observation, none (H = 0), and an invalid system beside valid ones
    in one M = 64 tile (its NaN rows must not reach the others' blocks)."""
    rng = np.random.default_rng(100 * n_pl + n_obs)
    cols = []
    for _ in range(n_pl):
        cols += [np.exp(rng.uniform(0, np.log(3000), n_sys)), rng.uniform(1, 80, n_sys),
                 rng.uniform(0, 0.85, n_sys), rng.uniform(0, 2 * np.pi, n_sys),
                 rng.uniform(0, 2 * np.pi, n_sys)]
    par = np.stack(cols + [rng.uniform(-10, 10, n_sys)], axis=1)
    bad = [1] if n_sys > 1 else []
    par[bad, 2] = 1.5                                    # e > 1: invalid
    t = np.sort(rng.uniform(2450000, 2453000, n_obs))
    v = rng.normal(0, 30, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    t0 = 2450500.0
    n = 5 * n_pl + 1
    chi_ref, g_ref, g_abs = oracle_mod.chi2(par, t, v, sig, n_pl, t0=t0, gabs=True)
    H_ref = oracle_mod.gauss_newton(par, t, sig, n_pl, t0=t0)
    P, T, V, S = dev(par, t, v, sig)
    ok = np.setdiff1d(np.arange(n_sys), bad)
    with gn_variant(kc, 0, n_sys, n_pl, n_obs):
        chi0, g0, H0 = [x.cpu().numpy() for x in kc.kc_chi2_gauss_newton(P, T, V, S, t0=t0,
                                                                          mode="mixed")]
    kc.kc_last_device_error()
    with gn_variant(kc, split, n_sys, n_pl, n_obs):
        chi, g, H = [x.cpu().numpy() for x in kc.kc_chi2_gauss_newton(P, T, V, S, t0=t0,
                                                                       mode="mixed")]
    assert kc.kc_last_device_error() == len(bad)
    assert np.all(np.isnan(chi[bad])) and np.all(np.isnan(g[bad])) and np.all(np.isnan(H[bad]))
    assert np.all(np.isfinite(H[ok]))
    if n_obs == 0:
        assert np.all(H[ok] == 0) and np.all(chi[ok] == 0) and np.all(g[ok] == 0)
        return
    assert rel(chi[ok], chi_ref[ok]).max() <= CHI2_MIXED_TOL
    ar = uniform_arith(kc, oracle_mod, par[ok], t, v, sig, n_pl, t0, 0.0, "mixed", "gn")
    assert grad_err(g[ok], g_ref[ok], g_abs[ok], "mixed", ar) <= 1.0
    assert h_err(H[ok], H_ref[ok], n).max() <= H_MIXED_TOL
    # the same split products as the mma.sync form: both within a few 2^-20
    # of the exact matrix on the correlation scale
    assert h_err(H[ok], H0[ok].astype(np.float64), n).max() <= 2e-5
    np.testing.assert_array_equal(chi[ok], chi0[ok])


def test_high_eccentricity(kc, oracle_mod):
    """One planet of each system at 0.96 <= e <= 0.99 (the FP64 solver's
    second step).  FP64: H, chi2 and gradient at the usual tolerances.  Mixed:
    chi2 within 1e-5 plus the single-precision conditioning bound of the
    velocity near pericentre, |dv| <= 4e-7 K / (1 - e), carried through
    2 sum_k w_k |r_k| |dv|."""
    rng = np.random.default_rng(71)
    n_sys, n_pl, n_obs = 64, 2, 200
    cols = []
    for j in range(n_pl):
        cols += [np.exp(rng.uniform(0, np.log(3000), n_sys)), rng.uniform(1, 80, n_sys),
                 rng.uniform(0.96, 0.99, n_sys) if j == 0 else rng.uniform(0, 0.8, n_sys),
                 rng.uniform(0, 2 * np.pi, n_sys), rng.uniform(0, 2 * np.pi, n_sys)]
    par = np.stack(cols + [rng.uniform(-5, 5, n_sys)], axis=1)
    t = np.sort(rng.uniform(2450000, 2453000, n_obs))
    sig = rng.uniform(1, 4, n_obs)
    v = oracle_mod.predict(par[:1], t, n_pl, 2450000.0)[0] + sig * rng.standard_normal(n_obs)
    chi_ref, g_ref, g_abs = oracle_mod.chi2(par, t, v, sig, n_pl, t0=2450000.0, gabs=True)
    H_ref = oracle_mod.gauss_newton(par, t, sig, n_pl, t0=2450000.0)
    P, T, V, S = dev(par, t, v, sig)
    chi, g, H = kc.kc_chi2_gauss_newton(P, T, V, S, t0=2450000.0, mode="fp64")
    assert rel(chi.cpu().numpy(), chi_ref).max() <= CHI2_F64_TOL
    ar = uniform_arith(kc, oracle_mod, par, t, v, sig, n_pl, 2450000.0, 0.0, "fp64", "gn")
    assert grad_err(g.cpu().numpy(), g_ref, g_abs, "fp64", ar) <= 1.0
    assert h_err(H.cpu().numpy(), H_ref, 5 * n_pl + 1).max() <= H_F64_TOL
    chi32, _, _ = kc.kc_chi2_gauss_newton(P, T, V, S, t0=2450000.0, mode="mixed")
    r = np.abs(oracle_mod.predict(par, t, n_pl, 2450000.0) - v[None, :])
    dv = sum(par[:, 5 * j + 1] * 4e-7 / (1 - par[:, 5 * j + 2]) for j in range(n_pl))
    bound = 1e-5 * np.maximum(chi_ref, 1.0) + 2 * (r / sig[None, :] ** 2).sum(axis=1) * dv
    assert np.all(np.abs(chi32.cpu().numpy().astype(np.float64) - chi_ref) <= bound)


def test_levenberg_marquardt_step_reduces_chi2(kc, oracle_mod):
    """One damped Gauss-Newton step built from the GPU outputs lowers chi2
    of perturbed models of noise-free data (the matrix is the one a fitter
    needs, not only numerically close to the oracle's)."""
    from paper_0812_2976_gb300 import synth
    w = synth.uniform(0, n_sys=64)
    t0 = float(w.t[0])
    v = oracle_mod.predict(w.truth, w.t, w.n_pl, t0)[0]
    rng = np.random.default_rng(5)
    params = w.truth * (1 + 1e-4 * rng.standard_normal((64, w.truth.size)))
    P, T, V, S = dev(params, w.t, v, w.sigma)
    chi, g, H = kc.kc_chi2_gauss_newton(P, T, V, S, t0=t0, mode="mixed")
    import oracle
    n = 5 * w.n_pl + 1
    Hf = oracle.unpack_symmetric(H.cpu().numpy().astype(np.float64), n)
    g = g.cpu().numpy().astype(np.float64)
    base = oracle_mod.chi2(params, w.t, v, w.sigma, w.n_pl, t0=t0)
    better = 0
    for s in range(params.shape[0]):
        A = Hf[s] + 1e-3 * np.diag(np.diag(Hf[s]))
        step = np.linalg.solve(A, -0.5 * g[s])
        new = oracle_mod.chi2((params[s] + step)[None], w.t, v, w.sigma, w.n_pl, t0=t0)[0]
        better += new < 0.5 * base[s]
    assert better >= 0.9 * params.shape[0]
