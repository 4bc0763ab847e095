"""Pins for the FP64 CPU oracle against facts other than itself.

Each test checks the oracle against something the paper or the mathematics
fixes: brute-force bisection of Kepler's equation, exact rational phases,
the circular-orbit closed form, the radial velocity as the time derivative
of the line-of-sight position, invariances of chi-square, and central finite
differences for the gradient.  None of these re-types the oracle's own
formulas.
"""
from fractions import Fraction

import numpy as np
import pytest

TWO_PI = 2.0 * np.pi


# ----------------------------------------------------------------- helpers

def bisect_kepler(M, e, iters=200):
    """Brute force: bisection of E - e sin E - M on [M - e, M + e]."""
    M = np.asarray(M, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    lo, hi = M - e, M + e
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        neg = (mid - e * np.sin(mid) - M) < 0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    return 0.5 * (lo + hi)


def exact_cycles(t, t0, P):
    """frac((t - t0)/P) computed exactly from the binary doubles."""
    q = (Fraction(float(t)) - Fraction(float(t0))) / Fraction(float(P))
    return q - (q.numerator // q.denominator)


def wrap_pi(x):
    return (np.asarray(x) + np.pi) % TWO_PI - np.pi


def angle_diff(a, b):
    return np.abs(wrap_pi(np.asarray(a) - np.asarray(b)))


# ------------------------------------------------------------ Kepler, Eq.1

def test_kepler_matches_bisection(oracle_mod):
    e = np.repeat(np.linspace(0.0, 0.99, 34), 41)
    M = np.tile(np.linspace(-np.pi, np.pi, 41), 34)
    E = oracle_mod.kepler_E(M, e)
    Eb = bisect_kepler(M, e)
    # the root is conditioned by 1/(1 - e cos E) <= 100 here
    assert np.max(np.abs(E - Eb)) < 5e-14


def test_kepler_special_cases(oracle_mod):
    for e in (0.0, 0.1, 0.5, 0.9, 0.999):
        assert abs(oracle_mod.kepler_E([0.0], [e])[0]) < 1e-300
        assert abs(oracle_mod.kepler_E([np.pi], [e])[0] - np.pi) < 1e-15
        assert abs(oracle_mod.kepler_E([-np.pi], [e])[0] + np.pi) < 1e-15
    M = np.linspace(-3, 3, 13)
    assert np.array_equal(oracle_mod.kepler_E(M, np.zeros_like(M)), M)


def test_kepler_residual_and_iterations(oracle_mod):
    rng = np.random.default_rng(1)
    M = rng.uniform(-np.pi, np.pi, 20000)
    e = rng.uniform(0.0, 0.999, 20000)
    E, it = oracle_mod.kepler_E(M, e, return_iters=True)
    resid = np.abs(E - e * np.sin(E) - M)
    assert resid.max() < 1e-15
    assert it.max() < 60


def test_kepler_odd_symmetry(oracle_mod):
    rng = np.random.default_rng(2)
    M = rng.uniform(0, np.pi, 500)
    e = rng.uniform(0, 0.95, 500)
    assert np.max(np.abs(oracle_mod.kepler_E(M, e) + oracle_mod.kepler_E(-M, e))) < 1e-15


# ----------------------------------------------------- mean anomaly, Eq. 4/6

def test_mean_anomaly_exact_phase(oracle_mod):
    """Against exact rational arithmetic at absolute epochs ~2.45e6 d, where
    single precision fails (Sec. 5, mixed precision)."""
    rng = np.random.default_rng(3)
    n = 300
    t = rng.uniform(2450000.0, 2456000.0, n)
    P = np.exp(rng.uniform(np.log(0.5), np.log(4000.0), n))
    M0 = rng.uniform(0, TWO_PI, n)
    for t0 in (0.0, 2450000.0, 1234.5):
        M = oracle_mod.mean_anomaly(t, t0, P, M0)
        assert np.all(M >= -np.pi) and np.all(M <= np.pi)
        for i in range(n):
            cyc = exact_cycles(t[i], t0, P[i])
            ref = TWO_PI * float(cyc) + M0[i]
            assert angle_diff(M[i], ref) < 4e-15 * 8, (i, t0)


def test_mean_anomaly_periodic(oracle_mod):
    P = np.array([3.7, 17.25, 411.0])
    M0 = np.array([0.3, 2.0, 5.9])
    t = np.array([100.0, 250.0, 999.0])
    a = oracle_mod.mean_anomaly(t, 0.0, P, M0)
    b = oracle_mod.mean_anomaly(t + P, 0.0, P, M0)
    assert np.max(angle_diff(a, b)) < 1e-12
    assert np.max(angle_diff(oracle_mod.mean_anomaly(t, 0.0, P, M0 + TWO_PI), a)) < 1e-14
    # at the epoch the mean anomaly is M0
    for i in range(3):
        at_epoch = oracle_mod.mean_anomaly(t[i:i + 1], t[i], P[i:i + 1], M0[i:i + 1])
        assert angle_diff(at_epoch[0], M0[i]) < 1e-15


# --------------------------------------------------- true anomaly, velocity

def test_true_anomaly_matches_cartesian_form(oracle_mod):
    rng = np.random.default_rng(4)
    E = rng.uniform(-np.pi, np.pi, 5000)
    e = rng.uniform(0, 0.99, 5000)
    f = oracle_mod.true_anomaly(E, e)
    D = 1 - e * np.cos(E)
    cf = (np.cos(E) - e) / D
    sf = np.sqrt((1 - e) * (1 + e)) * np.sin(E) / D
    assert np.max(angle_diff(f, np.arctan2(sf, cf))) < 1e-13


def test_velocity_is_derivative_of_line_of_sight_position(oracle_mod):
    """Independent of Eq. 3's printed form: with a = 1 the line-of-sight
    position is z = (cos E - e) sin w + sqrt(1-e^2) sin E cos w, and
    v = K sqrt(1-e^2)/n * dz/dt with n = 2 pi/P.  dz/dt by central
    differences, E by bisection, M = n t + M0 directly."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        P = np.exp(rng.uniform(np.log(2.0), np.log(1000.0)))
        K = rng.uniform(1, 100)
        e = rng.uniform(0, 0.9)
        w = rng.uniform(0, TWO_PI)
        M0 = rng.uniform(0, TWO_PI)
        n = TWO_PI / P
        t = rng.uniform(0, 3 * P, 8)
        h = P * 1e-5

        def z(tt):
            E = bisect_kepler(wrap_pi(n * tt + M0), np.full_like(tt, e))
            return (np.cos(E) - e) * np.sin(w) + np.sqrt(1 - e * e) * np.sin(E) * np.cos(w)

        dzdt = (z(t + h) - z(t - h)) / (2 * h)
        v_ref = K * np.sqrt(1 - e * e) / n * dzdt
        v = oracle_mod.planet_velocity([P, K, e, w, M0], t, 0.0)
        assert np.max(np.abs(v - v_ref)) < 1e-6 * K, (P, K, e, w, M0)


def test_velocity_circular_closed_form(oracle_mod):
    rng = np.random.default_rng(6)
    for _ in range(20):
        P, K = rng.uniform(2, 500), rng.uniform(1, 100)
        w, M0 = rng.uniform(0, TWO_PI, 2)
        t = rng.uniform(0, 1000, 16)
        v = oracle_mod.planet_velocity([P, K, 0.0, w, M0], t, 0.0)
        assert np.max(np.abs(v - K * np.cos(w + TWO_PI * t / P + M0))) < 1e-11 * K


# ------------------------------------------------------------- chi2, Eq. 5

def _random_systems(rng, n_sys, n_pl, e_max=0.9):
    rows = []
    for _ in range(n_sys):
        r = []
        for _ in range(n_pl):
            r += [np.exp(rng.uniform(0, np.log(4000))), rng.uniform(1, 100),
                  rng.uniform(0, e_max), rng.uniform(0, TWO_PI),
                  rng.uniform(0, TWO_PI)]
        rows.append(r + [rng.uniform(-10, 10)])
    return np.array(rows)


def test_chi2_circular_closed_form(oracle_mod):
    rng = np.random.default_rng(7)
    n_pl, n_obs = 3, 40
    par = _random_systems(rng, 6, n_pl)
    par[:, 2:5 * n_pl:5] = 0.0                     # e = 0
    t = np.sort(rng.uniform(0, 800, n_obs))
    v = rng.normal(0, 30, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    got = oracle_mod.chi2(par, t, v, sig, n_pl)
    for s in range(par.shape[0]):
        V = np.full(n_obs, par[s, -1])
        for j in range(n_pl):
            P, K, _, w, M0 = par[s, 5 * j:5 * j + 5]
            V += K * np.cos(w + TWO_PI * t / P + M0)
        ref = np.sum((V - v) ** 2 / sig ** 2)
        assert abs(got[s] - ref) <= 1e-12 * ref


def test_chi2_zero_for_noise_free_data(oracle_mod):
    rng = np.random.default_rng(8)
    par = _random_systems(rng, 1, 4)
    t = np.sort(rng.uniform(2450000, 2454000, 256))
    v = oracle_mod.predict(par, t, 4)[0]
    sig = rng.uniform(1, 5, 256)
    assert oracle_mod.chi2(par, t, v, sig, 4)[0] < 1e-20


def test_chi2_invariances(oracle_mod):
    rng = np.random.default_rng(9)
    n_pl, n_obs = 4, 128
    par = _random_systems(rng, 8, n_pl)
    t = np.sort(rng.uniform(2450000, 2454000, n_obs))
    v = rng.normal(0, 50, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    base = oracle_mod.chi2(par, t, v, sig, n_pl)
    # planet permutation
    perm = par.copy()
    order = [2, 0, 3, 1]
    for dst, src in enumerate(order):
        perm[:, 5 * dst:5 * dst + 5] = par[:, 5 * src:5 * src + 5]
    assert np.allclose(oracle_mod.chi2(perm, t, v, sig, n_pl), base, rtol=1e-13)
    # common offset on model and data
    shift = par.copy()
    shift[:, -1] += 7.5
    assert np.allclose(oracle_mod.chi2(shift, t, v + 7.5, sig, n_pl), base, rtol=1e-10)
    # M0 -> M0 + 2 pi
    m0 = par.copy()
    m0[:, 4:5 * n_pl:5] += TWO_PI
    assert np.allclose(oracle_mod.chi2(m0, t, v, sig, n_pl), base, rtol=1e-12)
    # jitter adds in quadrature to sigma (Eq. 5)
    jit = 2.5
    assert np.allclose(oracle_mod.chi2(par, t, v, sig, n_pl, jitter=jit),
                       oracle_mod.chi2(par, t, v, np.sqrt(sig ** 2 + jit ** 2), n_pl),
                       rtol=1e-13)


def test_chi2_time_shift_by_period(oracle_mod):
    rng = np.random.default_rng(10)
    par = _random_systems(rng, 5, 1)
    t = np.sort(rng.uniform(2450000, 2452000, 32))
    v = rng.normal(0, 50, 32)
    sig = rng.uniform(1, 5, 32)
    for s in range(5):
        P = par[s, 0]
        a = oracle_mod.chi2(par[s:s + 1], t, v, sig, 1)
        b = oracle_mod.chi2(par[s:s + 1], t + P, v, sig, 1)
        assert abs(a[0] - b[0]) <= 1e-10 * a[0]


def test_chi2_zero_amplitude_planet_drops_out(oracle_mod):
    rng = np.random.default_rng(11)
    par = _random_systems(rng, 4, 3)
    par[:, 5 + 1] = 0.0                               # K of planet 1
    t = np.sort(rng.uniform(2450000, 2452000, 64))
    v = rng.normal(0, 50, 64)
    sig = rng.uniform(1, 5, 64)
    red = np.concatenate([par[:, :5], par[:, 10:]], axis=1)
    assert np.allclose(oracle_mod.chi2(par, t, v, sig, 3),
                       oracle_mod.chi2(red, t, v, sig, 2), rtol=1e-14)


def test_chi2_invalid_inputs_give_nan(oracle_mod):
    rng = np.random.default_rng(12)
    par = _random_systems(rng, 4, 2)
    par[1, 2] = 1.0          # e = 1
    par[2, 5] = 0.0          # P = 0
    t = np.sort(rng.uniform(0, 100, 16))
    v = rng.normal(0, 5, 16)
    sig = np.ones(16)
    out = oracle_mod.chi2(par, t, v, sig, 2)
    assert np.isfinite(out[0]) and np.isfinite(out[3])
    assert np.isnan(out[1]) and np.isnan(out[2])
    sig[3] = 0.0
    assert np.all(np.isnan(oracle_mod.chi2(par, t, v, sig, 2)))


def test_ragged_matches_uniform(oracle_mod):
    rng = np.random.default_rng(13)
    par = _random_systems(rng, 6, 2)
    t = np.sort(rng.uniform(2450000, 2452000, 50))
    v = rng.normal(0, 50, 50)
    sig = rng.uniform(1, 5, 50)
    ref = oracle_mod.chi2(par, t, v, sig, 2)
    n_pl = np.full(6, 2, np.int32)
    par_off = np.arange(7) * 11
    obs_off = np.arange(7) * 50
    got = oracle_mod.chi2_ragged(par.ravel(), par_off, n_pl, np.tile(t, 6),
                                 np.tile(v, 6), np.tile(sig, 6), obs_off)
    assert np.array_equal(got, ref)


# ------------------------------------------------------------- gradient

@pytest.mark.parametrize("t0", [2450000.0, 0.0])
def test_gradient_matches_central_differences(oracle_mod, t0):
    rng = np.random.default_rng(14)
    n_pl, n_obs = 3, 60
    par = _random_systems(rng, 3, n_pl, e_max=0.8)
    t = np.sort(rng.uniform(2450000, 2454000, n_obs))
    v = rng.normal(0, 50, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    chi, g = oracle_mod.chi2(par, t, v, sig, n_pl, t0=t0, grad=True)
    for s in range(par.shape[0]):
        fd = np.empty(par.shape[1])
        for q in range(par.shape[1]):
            # 1e-6 relative step; a period step moves the phase by
            # 2 pi |t - t0| h / P^2, so it is sized to move it by 3e-4 rad
            # (truncation ~1e-8, rounding of a 1e6-cycle phase ~1e-6)
            h = 1e-6 * max(abs(par[s, q]), 1e-3)
            if q % 5 == 0 and q < 5 * n_pl:
                P = par[s, q]
                h = 3e-4 * P * P / (2 * np.pi * np.max(np.abs(t - t0)))
            p1, p2 = par[s].copy(), par[s].copy()
            p1[q] += h
            p2[q] -= h
            c1 = oracle_mod.chi2(p1[None], t, v, sig, n_pl, t0=t0)[0]
            c2 = oracle_mod.chi2(p2[None], t, v, sig, n_pl, t0=t0)[0]
            fd[q] = (c1 - c2) / (2 * h)
        scale = np.maximum(np.abs(g[s]), 1e-3 * np.linalg.norm(g[s]))
        assert np.max(np.abs(fd - g[s]) / scale) < 1e-5, (s, fd, g[s])


def test_gradient_circular_closed_form(oracle_mod):
    """e = 0: dv/dM0 = -K sin(w + M) and dv/dK = cos(w + M)."""
    rng = np.random.default_rng(15)
    P, K, w, M0, gam = 37.0, 20.0, 1.1, 0.4, 1.5
    par = np.array([[P, K, 0.0, w, M0, gam]])
    t = np.sort(rng.uniform(0, 500, 30))
    v = rng.normal(0, 20, 30)
    sig = rng.uniform(1, 5, 30)
    _, g = oracle_mod.chi2(par, t, v, sig, 1, grad=True)
    ph = w + TWO_PI * t / P + M0
    r = gam + K * np.cos(ph) - v
    wk = 1 / sig ** 2
    assert np.isclose(g[0, 1], np.sum(2 * wk * r * np.cos(ph)), rtol=1e-12)
    assert np.isclose(g[0, 4], np.sum(2 * wk * r * -K * np.sin(ph)), rtol=1e-12)
    assert np.isclose(g[0, 3], np.sum(2 * wk * r * -K * np.sin(ph)), rtol=1e-12)
    assert np.isclose(g[0, 5], np.sum(2 * wk * r), rtol=1e-12)
    assert np.isclose(g[0, 0], np.sum(2 * wk * r * -K * np.sin(ph) * (-TWO_PI * t / P ** 2)),
                      rtol=1e-11)


def test_ragged_predict_matches_uniform(oracle_mod):
    rng = np.random.default_rng(16)
    rows = [_random_systems(rng, 1, J)[0] for J in (1, 3, 2)]
    n_obs = [5, 0, 9]
    t = np.sort(rng.uniform(2450000, 2452000, sum(n_obs)))
    par = np.concatenate(rows)
    par_off = np.concatenate([[0], np.cumsum([r.size for r in rows])])
    obs_off = np.concatenate([[0], np.cumsum(n_obs)])
    got = oracle_mod.predict_ragged(par, par_off, [1, 3, 2], t, obs_off)
    for s, (r, J) in enumerate(zip(rows, (1, 3, 2))):
        ts = t[obs_off[s]:obs_off[s + 1]]
        if ts.size:
            assert np.array_equal(got[obs_off[s]:obs_off[s + 1]], oracle_mod.predict(r, ts, J)[0])


def test_infinite_uncertainty_is_zero_weight(oracle_mod):
    rng = np.random.default_rng(17)
    par = _random_systems(rng, 3, 2)
    t = np.sort(rng.uniform(0, 500, 20))
    v = rng.normal(0, 20, 20)
    sig = rng.uniform(1, 5, 20)
    base = oracle_mod.chi2(par, t, v, sig, 2)
    t2 = np.append(t, 600.0)
    out = oracle_mod.chi2(par, t2, np.append(v, 1e3), np.append(sig, np.inf), 2)
    assert np.array_equal(out, base)


# ------------------------------------------------ free jitter, log-likelihood

def _with_jitter(par, sj):
    return np.concatenate([par, np.full((par.shape[0], 1), sj)], axis=1)


def test_nll_at_zero_jitter_is_half_chi2_plus_normalisation(oracle_mod):
    rng = np.random.default_rng(18)
    par = _random_systems(rng, 5, 3)
    t = np.sort(rng.uniform(2450000, 2454000, 80))
    v = rng.normal(0, 30, 80)
    sig = rng.uniform(1, 5, 80)
    chi = oracle_mod.chi2(par, t, v, sig, 3)
    nll = oracle_mod.nll(_with_jitter(par, 0.0), t, v, sig, 3)
    const = 0.5 * np.sum(np.log(2 * np.pi * sig ** 2))
    assert np.allclose(nll, 0.5 * chi + const, rtol=1e-13)
    # a jitter in the likelihood is the same as Eq. 5's sigma_j for the chi2 part
    sj = 2.2
    nll_j = oracle_mod.nll(_with_jitter(par, sj), t, v, sig, 3)
    chi_j = oracle_mod.chi2(par, t, v, sig, 3, jitter=sj)
    assert np.allclose(nll_j, 0.5 * chi_j + 0.5 * np.sum(np.log(2 * np.pi * (sig ** 2 + sj ** 2))),
                       rtol=1e-13)
    assert np.array_equal(oracle_mod.nll(_with_jitter(par, -sj), t, v, sig, 3), nll_j)


def test_nll_jitter_derivative_vanishes_at_closed_form_optimum(oracle_mod):
    """With equal uncertainties sigma, d nll/d sigma_j = 0 at
    sigma_j^2 = mean(r^2) - sigma^2 (the Gaussian variance estimate)."""
    rng = np.random.default_rng(19)
    par = _random_systems(rng, 1, 2)
    t = np.sort(rng.uniform(2450000, 2452000, 60))
    r_true = rng.normal(0, 6, 60)
    model = oracle_mod.predict(par, t, 2)[0]
    v = model - r_true                         # residual V - v = r_true
    sig = np.full(60, 2.0)
    sj = np.sqrt(np.mean(r_true ** 2) - 4.0)
    _, g = oracle_mod.nll(_with_jitter(par, sj), t, v, sig, 2, grad=True)
    assert abs(g[0, -1]) < 1e-10 * np.sqrt(60)
    _, g2 = oracle_mod.nll(_with_jitter(par, 1.5 * sj), t, v, sig, 2, grad=True)
    assert g2[0, -1] > 0


def test_nll_gradient_matches_central_differences(oracle_mod):
    rng = np.random.default_rng(20)
    n_pl = 2
    par = _with_jitter(_random_systems(rng, 3, n_pl, e_max=0.8), 3.0)
    t = np.sort(rng.uniform(2450000, 2454000, 50))
    v = rng.normal(0, 40, 50)
    sig = rng.uniform(1, 5, 50)
    t0 = 2450000.0
    _, g = oracle_mod.nll(par, t, v, sig, n_pl, t0=t0, grad=True)
    for s in range(3):
        fd = np.empty(par.shape[1])
        for q in range(par.shape[1]):
            h = 1e-6 * max(abs(par[s, q]), 1e-3)
            if q % 5 == 0 and q < 5 * n_pl:
                P = par[s, q]
                h = 3e-4 * P * P / (2 * np.pi * np.max(np.abs(t - t0)))
            p1, p2 = par[s].copy(), par[s].copy()
            p1[q] += h
            p2[q] -= h
            fd[q] = (oracle_mod.nll(p1[None], t, v, sig, n_pl, t0=t0)[0]
                     - oracle_mod.nll(p2[None], t, v, sig, n_pl, t0=t0)[0]) / (2 * h)
        scale = np.maximum(np.abs(g[s]), 1e-3 * np.linalg.norm(g[s]))
        assert np.max(np.abs(fd - g[s]) / scale) < 1e-5


# ------------------------------------------------ DE-MC step

def test_demcmc_zero_move_always_accepted(oracle_mod):
    """gamma = 0, eps_scale = 0: the proposal is the state itself, Delta
    chi2 = 0, and ln u < 0 for u < 1 accepts it (states unchanged)."""
    rng = np.random.default_rng(22)
    states = _random_systems(rng, 8, 2)
    t = np.sort(rng.uniform(2450000, 2452000, 30))
    v = rng.normal(0, 30, 30)
    sig = rng.uniform(1, 5, 30)
    chi = oracle_mod.chi2(states, t, v, sig, 2)
    u = rng.uniform(0.0, 1.0, (4, 3))
    u[:, 0] = rng.uniform(0.01, 0.99, 4)
    st, c2, acc, prop, cp = oracle_mod.demcmc_step(states, chi, t, v, sig, 2, 0, 4, 4, 4, 0.0,
                                                   np.zeros(11), rng.standard_normal((4, 11)), u)
    assert np.array_equal(prop, states[:4]) and np.array_equal(cp, chi[:4])
    assert np.all(acc == 1) and np.array_equal(st, states)


def test_demcmc_partners_and_perturbation(oracle_mod):
    """The partner pair, read back from the proposals (gamma = 1 and chain j
    holding P = j, K = j^2, so P* - P_i = r1 - r2 and K* - K_i = r1^2 - r2^2):
    two distinct chains of the partner range, uniform over the ordered
    pairs (chi-square over 2000 draws), also at the edge draws 0, 1 - 2^-53
    and NaN (which counts as 0); and with gamma = 0 the perturbation is
    (eps_scale |x|) z, and only that."""
    rng = np.random.default_rng(27)
    n_pl, m = 1, 10
    n = 2 * m
    states = np.zeros((n, 6))
    states[:, 0] = np.arange(n, dtype=float)
    states[:, 1] = np.arange(n, dtype=float) ** 2
    states[:, 2] = 0.1
    t = np.linspace(2450000, 2450100, 5)
    v, sig = np.zeros(5), np.ones(5)
    chi = np.full(n, 1e300)
    pairs = []
    for rep_ in range(200):
        u = rng.uniform(0.0, 1.0, (m, 3))
        if rep_ == 0:
            u[0, 1:] = 0.0
            u[1, 1:] = 1.0 - 2.0 ** -53
            u[2, 1:] = np.nan
        _, _, _, prop, _ = oracle_mod.demcmc_step(states, chi, t, v, sig, n_pl, 0, m, m, m, 1.0,
                                                  np.zeros(6), np.zeros((m, 6)), u)
        d1 = prop[:, 0] - states[:m, 0]
        d2 = prop[:, 1] - states[:m, 1]
        s = d2 / d1
        r1, r2 = np.rint((s + d1) / 2).astype(int), np.rint((s - d1) / 2).astype(int)
        assert np.all(r1 != r2) and np.all((r1 >= m) & (r1 < n)) and np.all((r2 >= m) & (r2 < n))
        if rep_ == 0:
            assert (r1[0], r2[0]) == (m, m + 1) and (r1[1], r2[1]) == (n - 1, n - 2)
            assert (r1[2], r2[2]) == (m, m + 1)
            r1, r2 = r1[3:], r2[3:]
        pairs.append((r1 - m) * m + (r2 - m))
    counts = np.bincount(np.concatenate(pairs), minlength=m * m).reshape(m, m)
    assert np.all(np.diag(counts) == 0)
    expect = counts.sum() / (m * (m - 1))
    stat = ((counts - expect) ** 2 / expect)[~np.eye(m, dtype=bool)].sum()
    assert stat < 160            # chi-square, 89 degrees of freedom: p ~ 1e-5
    # perturbation with gamma = 0
    x = _random_systems(rng, n, n_pl)
    scale = rng.uniform(0.0, 1e-3, 6)
    z = rng.standard_normal((m, 6))
    _, _, _, prop, _ = oracle_mod.demcmc_step(x, np.full(n, 1e300), t, v, sig, n_pl, 0, m, m, m,
                                              0.0, scale, z, rng.uniform(0, 1, (m, 3)))
    assert np.array_equal(prop, x[:m] + (scale * np.abs(x[:m])) * z)


def test_demcmc_metropolis_rule(oracle_mod):
    """Accept iff u < exp(-(chi2* - chi2)/2), checked against chi2 computed
    separately; rejected chains keep state and chi2; partner ranges that
    overlap the updated chains or leave the population are refused."""
    rng = np.random.default_rng(23)
    n, n_pl = 40, 1
    states = _random_systems(rng, n, n_pl, e_max=0.5)
    t = np.sort(rng.uniform(2450000, 2451000, 25))
    v = oracle_mod.predict(states[0], t, n_pl)[0] + rng.normal(0, 2, 25)
    sig = np.full(25, 2.0)
    chi = oracle_mod.chi2(states, t, v, sig, n_pl)
    z = rng.standard_normal((20, 6))
    u = rng.uniform(0, 1, (20, 3))
    st, c2, acc, prop, cp = oracle_mod.demcmc_step(states, chi, t, v, sig, n_pl, 0, 20, 20, 20,
                                                   0.7, np.full(6, 1e-3), z, u)
    ref_cp = oracle_mod.chi2(prop, t, v, sig, n_pl)
    finite = np.isfinite(ref_cp)
    assert np.array_equal(cp[finite], ref_cp[finite])
    with np.errstate(over="ignore"):
        expect = np.where(np.isfinite(cp), u[:, 0] < np.exp(-0.5 * (cp - chi[:20])), False)
    assert np.array_equal(acc.astype(bool), expect)
    assert np.array_equal(st[:20][~expect], states[:20][~expect])
    assert np.array_equal(st[:20][expect], prop[expect])
    assert np.array_equal(st[20:], states[20:])
    for pfirst, pcount in ((10, 20), (30, 20), (20, 1), (-1, 5)):
        with pytest.raises(ValueError):
            oracle_mod.demcmc_step(states, chi, t, v, sig, n_pl, 0, 20, pfirst, pcount, 0.7,
                                   np.full(6, 1e-3), z, u)


def test_demcmc_samples_the_linear_gaussian_posterior(oracle_mod):
    """A circular planet with P, w, M0 fixed (identical in every chain, so
    DE never moves them) makes v linear in (K, gamma): the posterior is
    Gaussian with the least-squares mean and covariance.  Two-half DE-MC
    with the oracle's steps must reproduce them."""
    rng = np.random.default_rng(24)
    P, w, M0 = 37.0, 0.4, 1.3
    t = np.sort(rng.uniform(0, 200, 40))
    sig = rng.uniform(1, 3, 40)
    phase = w + 2 * np.pi * t / P + M0
    A = np.stack([np.cos(phase), np.ones_like(t)], axis=1)      # v = K cos + gamma
    truth = np.array([12.0, -3.0])
    v = A @ truth + rng.normal(0, sig)
    Wm = np.diag(1 / sig ** 2)
    cov = np.linalg.inv(A.T @ Wm @ A)
    mean = cov @ A.T @ Wm @ v
    n = 64
    states = np.tile([P, 0.0, 0.0, w, M0, 0.0], (n, 1))
    states[:, 1] = mean[0] + 3 * np.sqrt(cov[0, 0]) * rng.standard_normal(n)
    states[:, 5] = mean[1] + 3 * np.sqrt(cov[1, 1]) * rng.standard_normal(n)
    chi = oracle_mod.chi2(states, t, v, sig, 1)
    gamma = 2.38 / np.sqrt(2 * 2)
    half = n // 2
    samples = []
    scale = np.array([0.0, 1e-5, 0.0, 0.0, 0.0, 1e-5])
    for gen in range(1500):
        for first, other in ((0, half), (half, 0)):
            states, chi, _, _, _ = oracle_mod.demcmc_step(
                states, chi, t, v, sig, 1, first, half, other, half, gamma, scale,
                rng.standard_normal((half, 6)), rng.uniform(0, 1, (half, 3)))
        if gen >= 300:
            samples.append(states[:, [1, 5]].copy())
    s = np.concatenate(samples)
    assert np.all(np.abs(s.mean(axis=0) - mean) < 0.1 * np.sqrt(np.diag(cov)))
    assert np.allclose(np.cov(s.T), cov, rtol=0.15, atol=0.1 * np.sqrt(cov[0, 0] * cov[1, 1]))


# ------------------------------------------------ Gauss-Newton matrix

def test_gauss_newton_is_half_the_hessian_at_zero_residual(oracle_mod):
    """With noise-free data from the same parameters every residual is zero,
    so the Hessian of chi2 is exactly 2 sum_k w_k J_k J_k^T: its central
    differences of the (separately pinned) analytic gradient must give 2H."""
    rng = np.random.default_rng(31)
    n_pl, n_obs, t0 = 2, 50, 2450000.0
    par = _random_systems(rng, 3, n_pl, e_max=0.7)
    t = np.sort(rng.uniform(2450000, 2451500, n_obs))
    sig = rng.uniform(1, 5, n_obs)
    H = oracle_mod.gauss_newton(par, t, sig, n_pl, t0=t0, packed=False)
    for s in range(par.shape[0]):
        v = oracle_mod.predict(par[s], t, n_pl, t0)[0]          # r_k = 0
        n = par.shape[1]
        hess = np.empty((n, n))
        for q in range(n):
            h = 1e-5 * max(abs(par[s, q]), 1e-2)
            if q % 5 == 0 and q < 5 * n_pl:
                P = par[s, q]
                h = 1e-3 * P * P / (2 * np.pi * np.max(np.abs(t - t0)))
            p1, p2 = par[s].copy(), par[s].copy()
            p1[q] += h
            p2[q] -= h
            g1 = oracle_mod.chi2(p1[None], t, v, sig, n_pl, t0=t0, grad=True)[1][0]
            g2 = oracle_mod.chi2(p2[None], t, v, sig, n_pl, t0=t0, grad=True)[1][0]
            hess[:, q] = (g1 - g2) / (2 * h)
        d = np.sqrt(np.abs(np.diag(2 * H[s])))
        scale = np.maximum(np.outer(d, d), 1e-12)
        assert np.max(np.abs(hess - 2 * H[s]) / scale) < 1e-5


def test_gauss_newton_circular_closed_form(oracle_mod):
    """e = 0: v = K cos(w + M) + gamma with M = 2 pi (t - t0)/P + M0, so the
    (P, K, w, M0, gamma) block of H has a closed form."""
    rng = np.random.default_rng(32)
    P, K, w, M0, gam, t0 = 23.0, 17.0, 0.7, 2.1, 1.5, 2450100.0
    t = np.sort(rng.uniform(2450000, 2451000, 45))
    sig = rng.uniform(1, 4, 45)
    H = oracle_mod.gauss_newton([P, K, 0.0, w, M0, gam], t, sig, 1, t0=t0, packed=False)[0]
    ph = w + TWO_PI * (t - t0) / P + M0
    J = np.stack([K * np.sin(ph) * TWO_PI * (t - t0) / P ** 2,   # dv/dP
                  np.cos(ph),                                   # dv/dK
                  -K * np.sin(ph),                              # dv/dw
                  -K * np.sin(ph),                              # dv/dM0
                  np.ones_like(t)], axis=1)                     # dv/dgamma
    ref = J.T @ (J / sig[:, None] ** 2)
    idx = [0, 1, 3, 4, 5]
    sub = H[np.ix_(idx, idx)]
    d = np.sqrt(np.diag(ref))
    assert np.max(np.abs(sub - ref) / np.outer(d, d)) < 1e-12


def test_gauss_newton_structure(oracle_mod):
    """Symmetric positive semi-definite; a zero-weight (infinite sigma)
    observation changes nothing; doubling every sigma divides H by 4; the
    jitter adds in quadrature; invalid parameters give NaN."""
    rng = np.random.default_rng(33)
    par = _random_systems(rng, 4, 3)
    t = np.sort(rng.uniform(2450000, 2452000, 30))
    sig = rng.uniform(1, 5, 30)
    H = oracle_mod.gauss_newton(par, t, sig, 3, packed=False)
    for s in range(4):
        ev = np.linalg.eigvalsh(H[s])
        assert ev.min() > -1e-9 * ev.max()
    t2, s2 = np.append(t, 2452500.0), np.append(sig, np.inf)
    assert np.array_equal(oracle_mod.gauss_newton(par, t2, s2, 3), oracle_mod.gauss_newton(par, t, sig, 3))
    Hp = oracle_mod.gauss_newton(par, t, sig, 3)
    assert np.allclose(oracle_mod.gauss_newton(par, t, 2 * sig, 3), Hp / 4, rtol=1e-13, atol=0)
    sig_j = np.sqrt(sig ** 2 - 0.5)
    assert np.allclose(oracle_mod.gauss_newton(par, t, sig_j, 3, jitter=np.sqrt(0.5)), Hp,
                       rtol=1e-12, atol=0)
    bad = par.copy()
    bad[1, 2] = 1.2
    Hb = oracle_mod.gauss_newton(bad, t, sig, 3)
    assert np.all(np.isnan(Hb[1])) and np.all(np.isfinite(Hb[[0, 2, 3]]))


def test_velocity_equals_the_eccentric_anomaly_form(oracle_mod):
    """The kernels evaluate Eq. 3 in its eccentric-anomaly form
    [K cos w (cos E - e) - K sqrt(1 - e^2) sin w sin E]/(1 - e cos E)
    + K e cos w (mixed path) or, with the e cos w term folded in,
    [K cos w (1 - e^2) cos E - K sqrt(1 - e^2) sin w sin E]/(1 - e cos E)
    (FP64 path); the oracle uses the true anomaly f explicitly.  They are
    algebraically identical (cos f = (cos E - e)/D, sin f = sqrt(1-e^2)
    sin E / D, (cos E - e) + e D = (1 - e^2) cos E), so they must agree to
    rounding."""
    rng = np.random.default_rng(41)
    for _ in range(20):
        P, K = np.exp(rng.uniform(0, np.log(3000))), rng.uniform(1, 100)
        e, w, M0 = rng.uniform(0, 0.97), rng.uniform(0, TWO_PI), rng.uniform(0, TWO_PI)
        t = np.sort(rng.uniform(0, 5000, 25))
        v = oracle_mod.planet_velocity([P, K, e, w, M0], t)
        M = oracle_mod.mean_anomaly(t, 0.0, P, M0)
        E = oracle_mod.kepler_E(M, e)
        D = 1 - e * np.cos(E)
        b2 = (1 - e) * (1 + e)
        v_E = (K * np.cos(w) * (np.cos(E) - e)
               - K * np.sqrt(b2) * np.sin(w) * np.sin(E)) / D + K * e * np.cos(w)
        v_folded = (K * np.cos(w) * b2 * np.cos(E) - K * np.sqrt(b2) * np.sin(w) * np.sin(E)) / D
        assert np.max(np.abs(v_E - v)) <= 1e-13 * K / (1 - e)
        assert np.max(np.abs(v_folded - v)) <= 1e-13 * K / (1 - e)


# ------------------------------------------------------------ gradient magnitudes

def test_gabs_bounds_and_additivity(oracle_mod):
    """gabs = sum_k |term_k of the gradient| (the cancellation scale used by
    the gradient parity bound): at least |g| componentwise, equal to |g| for
    one observation, and additive over disjoint sets of observations; the
    same for the free-jitter likelihood and a ragged batch."""
    rng = np.random.default_rng(91)
    n_pl, n_obs = 2, 60
    par = np.array([[40.0, 30.0, 0.4, 1.0, 2.0, 300.0, 12.0, 0.1, 4.0, 0.5, 3.0],
                    [7.0, 60.0, 0.7, 5.0, 1.0, 1500.0, 5.0, 0.2, 2.0, 6.0, -2.0]])
    t = np.sort(rng.uniform(2450000.0, 2452000.0, n_obs))
    v = rng.normal(0.0, 30.0, n_obs)
    sig = rng.uniform(1.0, 4.0, n_obs)
    c, g, ga = oracle_mod.chi2(par, t, v, sig, n_pl, t0=2450000.0, jitter=0.5, gabs=True)
    assert np.all(ga >= np.abs(g) * (1 - 1e-14))
    assert np.any(ga > 10 * np.abs(g))                      # cancellation is present
    _, g1, ga1 = oracle_mod.chi2(par, t[7:8], v[7:8], sig[7:8], n_pl, t0=2450000.0,
                                 jitter=0.5, gabs=True)
    np.testing.assert_allclose(ga1, np.abs(g1), rtol=1e-15)
    _, _, gaA = oracle_mod.chi2(par, t[:25], v[:25], sig[:25], n_pl, t0=2450000.0,
                                jitter=0.5, gabs=True)
    _, _, gaB = oracle_mod.chi2(par, t[25:], v[25:], sig[25:], n_pl, t0=2450000.0,
                                jitter=0.5, gabs=True)
    np.testing.assert_allclose(gaA + gaB, ga, rtol=1e-13)
    pj = np.concatenate([par, [[0.8], [2.5]]], axis=1)
    _, gn, gan = oracle_mod.nll(pj, t, v, sig, n_pl, t0=2450000.0, gabs=True)
    assert np.all(gan >= np.abs(gn) * (1 - 1e-14))
    _, gn1, gan1 = oracle_mod.nll(pj, t[3:4], v[3:4], sig[3:4], n_pl, t0=2450000.0, gabs=True)
    np.testing.assert_allclose(gan1, np.abs(gn1), rtol=1e-15)
    # ragged: the two systems on their own halves of the observations
    par_off = np.array([0, 11, 22])
    obs_off = np.array([0, 30, 60])
    cr, gr, gar = oracle_mod.chi2_ragged(par.ravel(), par_off, np.array([2, 2], np.int32),
                                         t, v, sig, obs_off, t0=2450000.0, jitter=0.5,
                                         gabs=True)
    for s in range(2):
        o = slice(obs_off[s], obs_off[s + 1])
        _, _, gu = oracle_mod.chi2(par[s:s + 1], t[o], v[o], sig[o], n_pl, t0=2450000.0,
                                   jitter=0.5, gabs=True)
        np.testing.assert_allclose(gar[par_off[s]:par_off[s + 1]], gu[0], rtol=1e-13)
