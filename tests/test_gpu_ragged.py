"""Ragged batches (kc_plan_*) vs the FP64 CPU oracle, through the C ABI.

Systems with their own planet count and observations; one persistent,
graph-replayed launch.  Same tolerances as the uniform path."""
import numpy as np
import pytest
import torch
from tolerance import U32, U64, chi2_rounding_term, grad_bound, grad_excess_ragged, ragged_ariths

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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref) / np.maximum(np.abs(ref), 1.0)


def grad_err_ragged(got, ref, gabs, par_off, mode="mixed", ariths=None):
    """Largest error of a gradient component over its bound (<= 1 passes);
    ariths: per system, how the kernel formed and summed it
    (tests/tolerance.py)."""
    rel, u = (GRAD_MIXED_TOL, U32) if mode == "mixed" else (GRAD_F64_TOL, U64)
    return grad_excess_ragged(got, ref, gabs, par_off, rel, u, ariths)


def observed(oracle_mod, w):
    return oracle_mod.predict_ragged(w.truth, w.par_off, w.n_pl, w.t, w.obs_off) + w.noise


@pytest.fixture(scope="module")
def small(oracle_mod):
    """600 systems of the config-4 distribution, with shorter series."""
    from paper_0812_2976_gb300 import synth
    w = synth.ragged(600, seed=77, obs_range=(0, 300), pl_range=(1, 8))
    return w, observed(oracle_mod, w)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_ragged_chi2_and_gradient(kc, oracle_mod, small, mode):
    w, v = small
    ref, gref, gabs = oracle_mod.chi2_ragged(w.params, w.par_off, w.n_pl, w.t, v, w.sigma,
                                             w.obs_off, t0=2450000.0, jitter=0.7, gabs=True)
    T, V, S, P = dev(w.t), dev(v), dev(w.sigma), dev(w.params)
    tol = MIXED_TOL if mode == "mixed" else FP64_TOL
    plan = kc.RaggedPlan(w.obs_off, w.n_pl, t0=2450000.0, jitter=0.7, mode=mode)
    plan.set_observations(T, V, S)
    chi = plan.run(P).cpu().numpy()
    assert rel_err(chi, ref).max() <= tol
    gplan = kc.RaggedPlan(w.obs_off, w.n_pl, t0=2450000.0, jitter=0.7, mode=mode,
                          want_grad=True)
    gplan.set_observations(T, V, S)
    chi_g, g = gplan.run(P)
    assert rel_err(chi_g.cpu().numpy(), ref).max() <= tol
    ar = ragged_ariths(oracle_mod, w.params, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off,
                       2450000.0, 0.7, mode)
    assert grad_err_ragged(g.cpu().numpy(), gref, gabs, w.par_off, mode, ar) <= 1.0


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_ragged_high_eccentricity(kc, oracle_mod, small, mode):
    """Every fifth system with its first planet at 0.96 <= e <= 0.99 (in the
    FP64 kernel those warps take the second double-precision step).  Mixed
    chi2 is held to 1e-5 plus the
    single-precision conditioning bound of the velocity near pericentre,
    |dv| <= 4e-7 K / (1 - e), carried through 2 sum_k w_k |r_k| |dv|."""
    w, v = small
    par = w.params.copy()
    rng = np.random.default_rng(5)
    hi = np.arange(0, w.n_sys, 5)
    par[w.par_off[hi] + 2] = rng.uniform(0.96, 0.99, hi.size)
    ref, gref, gabs = oracle_mod.chi2_ragged(par, w.par_off, w.n_pl, w.t, v, w.sigma,
                                             w.obs_off, t0=2450000.0, jitter=0.7, gabs=True)
    T, V, S, P = dev(w.t), dev(v), dev(w.sigma), dev(par)
    gplan = kc.RaggedPlan(w.obs_off, w.n_pl, t0=2450000.0, jitter=0.7, mode=mode,
                          want_grad=True)
    gplan.set_observations(T, V, S)
    chi_g, g = gplan.run(P)
    chi = chi_g.cpu().numpy().astype(np.float64)
    g = g.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(chi)) and np.all(np.isfinite(g))
    if mode == "fp64":
        assert rel_err(chi, ref).max() <= FP64_TOL
        ar = ragged_ariths(oracle_mod, par, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off,
                           2450000.0, 0.7, "fp64")
        assert grad_err_ragged(g, gref, gabs, w.par_off, "fp64", ar) <= 1.0
        return
    model = oracle_mod.predict_ragged(par, w.par_off, w.n_pl, w.t, w.obs_off, t0=2450000.0)
    ar = ragged_ariths(oracle_mod, par, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off,
                       2450000.0, 0.7, "mixed")
    var = w.sigma ** 2 + 0.7 ** 2
    wr = np.abs(model - v) / var
    for s in range(w.n_sys):
        o0, o1 = w.obs_off[s], w.obs_off[s + 1]
        a, b = w.par_off[s], w.par_off[s + 1]
        p = par[a:b]
        J = int(w.n_pl[s])
        dv = sum(p[5 * j + 1] * 4e-7 / (1 - p[5 * j + 2]) for j in range(J))
        bound = 1e-5 * max(ref[s], 1.0) + 2 * wr[o0:o1].sum() * dv
        assert abs(chi[s] - ref[s]) <= bound, (s, chi[s], ref[s], bound)
        # gradient: the same velocity error dv reaches every component
        # through the residual, sum_k 2 w_k |dV_k/dtheta_i| dv, which
        # Cauchy-Schwarz bounds by 2 sqrt(H_ii sum_k w_k) dv with H the
        # oracle's Gauss-Newton matrix; the partials' own single-precision
        # error near pericentre grows like u / (1 - e cos E)^2, at most
        # 8 u / (1 - e_max)^2 of each term (|term| summed in gabs)
        if o1 == o0:
            assert np.all(g[a:b] == 0.0), s
            continue
        H = oracle_mod.gauss_newton(p[None, :], w.t[o0:o1], w.sigma[o0:o1], J,
                                    t0=2450000.0, jitter=0.7, packed=False)[0]
        e_max = max(p[5 * j + 2] for j in range(J))
        extra = (2 * np.sqrt(np.diagonal(H) * np.sum(1.0 / var[o0:o1])) * dv
                 + 8 * U32 * gabs[a:b] / (1 - e_max) ** 2)
        gb = grad_bound(gref[a:b][None, :], gabs[a:b][None, :], GRAD_MIXED_TOL, U32,
                        ar[s])[0] + extra
        assert np.all(np.abs(g[a:b] - gref[a:b]) <= gb), (s, np.max(np.abs(g[a:b] - gref[a:b]) / gb))


def test_graph_replay_new_pointers_and_streams(kc, oracle_mod, small):
    w, v = small
    T, V, S = dev(w.t), dev(v), dev(w.sigma)
    plan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed")
    plan.set_observations(T, V, S)
    P1 = dev(w.params)
    P2 = dev(w.truth)
    a = plan.run(P1).clone()                     # captures the graph
    b = plan.run(P2)                             # replays with new pointers
    c = plan.run(P1, chi2_out=torch.empty_like(a))
    ref1 = oracle_mod.chi2_ragged(w.params, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off)
    ref2 = oracle_mod.chi2_ragged(w.truth, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off)
    # 1e-5 relative plus the residuals' rounding carried into chi2 (at the
    # truth, chi2 ~ n_obs: a 2-observation system with K ~ 50 m/s moves by
    # ~1e-5 of its chi2 per 1e-7 rad of M)
    for got, ref, par in ((a, ref1, w.params), (b, ref2, w.truth)):
        got = got.cpu().numpy().astype(np.float64)
        for s in range(w.n_sys):
            o0, o1 = w.obs_off[s], w.obs_off[s + 1]
            p0, p1 = w.par_off[s], w.par_off[s + 1]
            extra = chi2_rounding_term(oracle_mod, par[p0:p1], w.t[o0:o1], v[o0:o1],
                                       w.sigma[o0:o1], int(w.n_pl[s]), 0.0, 0.0, U32)[0] \
                if o1 > o0 else 0.0
            assert abs(got[s] - ref[s]) <= MIXED_TOL * max(ref[s], 1.0) + extra, (s, got[s], ref[s])
    assert torch.equal(a, c)
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        d = plan.run(P1)                         # another stream: new capture
    s2.synchronize()
    assert torch.equal(a, d)


def test_autotune_keeps_results(kc, small):
    w, v = small
    T, V, S, P = dev(w.t), dev(v), dev(w.sigma), dev(w.params)
    plan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed")
    plan.set_observations(T, V, S)
    before = plan.run(P).clone()
    block, k = plan.autotune(P)
    assert block in (64, 128, 256) and k >= 1
    after = plan.run(P)
    assert torch.equal(before, after)           # one warp per system: order-free


def test_padded_uniform_plan_agrees(kc, oracle_mod, small):
    """Padding every system to the largest size (K = 0 planets, zero-weight
    observations) leaves chi2 unchanged: the padded baseline of the bench
    computes the same numbers."""
    from paper_0812_2976_gb300 import synth
    w, v = small
    pw, pv = synth.pad_ragged(w, v)
    plan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed")
    plan.set_observations(dev(w.t), dev(v), dev(w.sigma))
    a = plan.run(dev(w.params)).cpu().numpy()
    pplan = kc.RaggedPlan(pw.obs_off, pw.n_pl, mode="mixed")
    pplan.set_observations(dev(pw.t), dev(pv), dev(pw.sigma))
    b = pplan.run(dev(pw.params)).cpu().numpy()
    assert rel_err(b, a.astype(np.float64)).max() <= MIXED_TOL


def test_invalid_and_empty_systems(kc):
    obs_off = np.array([0, 10, 10, 25], dtype=np.int64)      # system 1 has no data
    n_pl = np.array([2, 1, 3], dtype=np.int32)
    rng = np.random.default_rng(3)
    params = []
    for J in n_pl:
        for _ in range(J):
            params += [rng.uniform(2, 50), rng.uniform(1, 50), rng.uniform(0, 0.5),
                       rng.uniform(0, 6), rng.uniform(0, 6)]
        params.append(1.0)
    params = np.array(params)
    t = np.sort(rng.uniform(2450000, 2450100, 25))
    v = rng.normal(0, 5, 25)
    sig = np.ones(25)
    for mode in ("mixed", "fp64"):
        plan = kc.RaggedPlan(obs_off, n_pl, mode=mode)
        plan.set_observations(dev(t), dev(v), dev(sig))
        out = plan.run(dev(params)).cpu().numpy()
        assert np.all(np.isfinite(out)) and out[1] == 0.0
        bad = params.copy()
        bad[11 + 2] = 1.5                                     # e of system 1
        out = plan.run(dev(bad)).cpu().numpy()
        assert np.isfinite(out[0]) and np.isnan(out[1]) and np.isfinite(out[2])


def test_bad_plan_arguments(kc):
    with pytest.raises(kc.KcError):
        kc.RaggedPlan([0, 5, 3], [1, 1])                      # decreasing offsets
    with pytest.raises(kc.KcError):
        kc.RaggedPlan([0, 5], [9])                            # n_pl > 8
    plan = kc.RaggedPlan([0, 4], [1])
    with pytest.raises(kc.KcError):
        plan.run(dev(np.ones(6)))                             # no observations yet


def test_config4_full_size_sampled(kc, oracle_mod):
    """200000 systems, n_obs ~ U[16,1024], n_pl ~ U{1..6}: the full plan on
    the GPU, the oracle on a sample of systems (forward and gradient)."""
    from paper_0812_2976_gb300 import synth
    w = synth.ragged()
    v = observed(oracle_mod, w)
    T, V, S, P = dev(w.t), dev(v), dev(w.sigma), dev(w.params)
    plan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed", want_grad=True)
    plan.set_observations(T, V, S)
    chi, g = plan.run(P)
    chi, g = chi.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.isfinite(chi))
    assert np.all(np.isfinite(g))
    rng = np.random.default_rng(5)
    work = w.n_pl.astype(np.int64) * np.diff(w.obs_off)
    idx = np.unique(np.concatenate([rng.choice(w.n_sys, 300, replace=False),
                                    np.argsort(work)[-20:], np.argsort(work)[:20]]))
    sub = synth.subset_ragged(w, idx)
    vsub = np.concatenate([v[w.obs_off[s]:w.obs_off[s + 1]] for s in idx])
    ref, gref, gabs = oracle_mod.chi2_ragged(sub.params, sub.par_off, sub.n_pl, sub.t, vsub,
                                             sub.sigma, sub.obs_off, gabs=True)
    assert rel_err(chi[idx], ref).max() <= MIXED_TOL
    gsub = np.concatenate([g[w.par_off[s]:w.par_off[s + 1]] for s in idx])
    ar = ragged_ariths(oracle_mod, sub.params, sub.par_off, sub.n_pl, sub.t, vsub, sub.sigma,
                       sub.obs_off, 0.0, 0.0, "mixed")
    assert grad_err_ragged(gsub, gref, gabs, sub.par_off, "mixed", ar) <= 1.0


def test_rv_predict_ragged_vs_oracle(kc, oracle_mod, small):
    w, _ = small
    ref = oracle_mod.predict_ragged(w.params, w.par_off, w.n_pl, w.t, w.obs_off, 2450000.0)
    got = kc.kc_rv_predict_ragged(dev(w.params), torch.tensor(w.par_off),
                                  torch.tensor(w.n_pl), dev(w.t), torch.tensor(w.obs_off),
                                  t0=2450000.0).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-9


def test_runs_on_two_streams_may_overlap(kc, oracle_mod):
    """One plan run on two streams with nothing ordering the runs: each
    stream has its own work queue, so both streams' results are the
    oracle's (a queue shared by the two kernels would split the systems
    between them)."""
    from paper_0812_2976_gb300 import synth
    w = synth.ragged(20000, seed=91)
    v = observed(oracle_mod, w)
    ref1 = oracle_mod.chi2_ragged(w.params, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off)
    ref2 = oracle_mod.chi2_ragged(w.truth, w.par_off, w.n_pl, w.t, v, w.sigma, w.obs_off)
    plan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed")
    plan.set_observations(dev(w.t), dev(v), dev(w.sigma))
    P1, P2 = dev(w.params), dev(w.truth)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for _ in range(3):
        with torch.cuda.stream(s1):
            a = plan.run(P1)
        with torch.cuda.stream(s2):
            b = plan.run(P2)
        outs.append((a, b))
    torch.cuda.synchronize()
    for a, b in outs:
        assert rel_err(a.cpu().numpy(), ref1).max() <= MIXED_TOL
        assert rel_err(b.cpu().numpy(), ref2).max() <= MIXED_TOL
