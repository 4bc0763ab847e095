"""DE-MC step (kc_demcmc_step) and driver on the GPU vs the FP64 oracle.

The random draws (standard normal z, uniform u) and the current chi2 are the
same inputs on both sides; each side maps them to partners and perturbations.  Proposals are exact arithmetic of the inputs and must
match bit for bit; accept decisions must match wherever the Metropolis
margin |ln u + (chi2* - chi2)/2| is above what the chi2 tolerance of the mode
can move (1e-12 relative in FP64, 1e-5 mixed); the states then follow."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kc():
    import paper_0812_2976_gb300 as kc
    from paper_0812_2976_gb300 import build
    build.build()
    kc._lib.load()
    return kc


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("mode,tol,tile", [
    ("fp64", 1e-12, None), ("mixed", 1e-5, None),
    ("mixed", 1e-5, (16, 256, 0)),      # fused tile kernel: proposals and accept inside
    ("mixed", 1e-5, (16, 128, 1)),      # prepared two-pass: accept in the main kernel
    ("mixed", 1e-5, (64, 64, 2)),       # chunked two-pass: accept as its own kernel
    ("mixed", 1e-5, (8, 96, 3)),        # warp-per-system kernel, four systems per warp
])
def test_step_matches_oracle(kc, oracle_mod, mode, tol, tile):
    """The Metropolis step runs in the chi2 kernel's epilogue, or after the
    chunked two-pass variant as its own kernel; every launch shape gives
    the oracle's step (with no tile pinned, mixed takes the warp-per-system
    kernel)."""
    if tile is not None:
        kc.kc_set_tile("chi2", mode, 256, 4, 256, tile)
        assert kc.kc_get_tile("chi2", mode, 256, 4, 256) == tile
    try:
        _step_matches_oracle(kc, oracle_mod, mode, tol)
    finally:
        if tile is not None:
            kc.kc_set_tile("chi2", mode, 256, 4, 256, None)


def _step_matches_oracle(kc, oracle_mod, mode, tol):
    from paper_0812_2976_gb300 import synth
    w = synth.uniform(1, n_sys=512)
    v = oracle_mod.predict(w.truth, w.t, w.n_pl)[0] + w.noise
    states = w.params
    chi = oracle_mod.chi2(states, w.t, v, w.sigma, w.n_pl)
    rng = np.random.default_rng(40)
    first, count, other = 256, 256, 0
    npar = states.shape[1]
    scale = np.full(npar, 1e-4)
    z = rng.standard_normal((count, npar))
    u = rng.uniform(0, 1, (count, 3))
    u[5, 1:] = [0.0, 1.0 - 2.0 ** -53]                          # edge draws
    u[7, 1:] = np.nan                                          # counts as 0
    gamma = 2.38 / np.sqrt(2 * npar)
    ref = oracle_mod.demcmc_step(states, chi, w.t, v, w.sigma, w.n_pl, first, count, other,
                                 256, gamma, scale, z, u)
    ref_states, ref_chi, ref_acc, ref_prop, ref_cp = ref
    S = dev(states)
    C = dev(chi, torch.float64 if mode == "fp64" else torch.float32)
    prop = torch.empty((count, states.shape[1]), dtype=torch.float64, device="cuda")
    cp = torch.empty(count, dtype=C.dtype, device="cuda")
    acc = kc.kc_demcmc_step(S, C, dev(w.t), dev(v), dev(w.sigma), first, count, other, 256,
                            gamma, dev(scale), dev(z), dev(u), proposals=prop, chi2_prop=cp,
                            mode=mode).cpu().numpy()
    prop = prop.cpu().numpy()
    assert np.array_equal(prop, ref_prop)                       # bit for bit
    cp = cp.cpu().numpy().astype(np.float64)
    ok = np.isfinite(ref_cp)
    assert np.max(np.abs(cp[ok] - ref_cp[ok]) / np.maximum(ref_cp[ok], 1.0)) <= tol
    # decisions away from the Metropolis boundary are identical
    chi_cur = C.cpu().numpy().astype(np.float64)[first:] if mode == "mixed" else chi[first:]
    margin = np.abs(np.log(u[:, 0]) + 0.5 * (ref_cp - chi[first:]))
    slack = 4 * tol * np.maximum(ref_cp, 1.0) + 4 * tol * np.maximum(chi_cur, 1.0)
    sure = ok & (margin > slack)
    assert sure.sum() > count // 2
    assert np.array_equal(acc[sure], ref_acc[sure])
    new_states = S.cpu().numpy()
    for c in np.nonzero(sure)[0]:
        expect = ref_prop[c] if ref_acc[c] else states[first + c]
        assert np.array_equal(new_states[first + c], expect)
    assert np.array_equal(new_states[:first], states[:first])
    # partner ranges that overlap the updated chains or leave the population
    for pf, pc in ((128, 256), (0, 1), (400, 200)):
        with pytest.raises(Exception):
            kc.kc_demcmc_step(S, C, dev(w.t), dev(v), dev(w.sigma), first, count, pf, pc, gamma,
                              dev(scale), dev(z), dev(u), mode=mode)


def test_driver_samples_the_linear_gaussian_posterior(kc):
    """The DEMCMC driver on a circular planet with only K and gamma free:
    the posterior is Gaussian with the least-squares mean and covariance."""
    rng = np.random.default_rng(41)
    P, w, M0 = 37.0, 0.4, 1.3
    t = np.sort(rng.uniform(2450000, 2450200, 40))
    sig = rng.uniform(1, 3, 40)
    phase = w + 2 * np.pi * np.fmod(t, P) / P + M0
    A = np.stack([np.cos(phase), np.ones_like(t)], axis=1)
    v = A @ np.array([12.0, -3.0]) + rng.normal(0, sig)
    Wm = np.diag(1 / sig ** 2)
    cov = np.linalg.inv(A.T @ Wm @ A)
    mean = cov @ A.T @ Wm @ v
    n = 256
    states = np.tile([P, 0.0, 0.0, w, M0, 0.0], (n, 1))
    states[:, 1] = mean[0] + 3 * np.sqrt(cov[0, 0]) * rng.standard_normal(n)
    states[:, 5] = mean[1] + 3 * np.sqrt(cov[1, 1]) * rng.standard_normal(n)
    mc = kc.DEMCMC(dev(states), dev(t), dev(v), dev(sig), mode="mixed",
                   eps_scale=[0.0, 1e-5, 0.0, 0.0, 0.0, 1e-5], seed=3)
    samples = []
    for gen in range(1200):
        mc.step()
        if gen >= 200 and gen % 2 == 0:
            samples.append(mc.states[:, [1, 5]].clone())
    s = torch.cat(samples).cpu().numpy()
    assert 0.1 < mc.acceptance < 0.9
    assert np.all(np.abs(s.mean(axis=0) - mean) < 0.1 * np.sqrt(np.diag(cov)))
    assert np.allclose(np.cov(s.T), cov, rtol=0.15, atol=0.1 * np.sqrt(cov[0, 0] * cov[1, 1]))
    # P, w, M0 never move: every chain holds the same value
    st = mc.states.cpu().numpy()
    assert np.all(st[:, 0] == P) and np.all(st[:, 3] == w) and np.all(st[:, 4] == M0)


@pytest.mark.parametrize("generations,hop_every,batch",
                         [(12, 0, 2), (13, 4, 2), (13, 5, 2), (40, 0, 8), (7, 0, 1)])
def test_graph_replay_equals_eager(kc, generations, hop_every, batch):
    """The same seed gives the same chain eagerly and with graph replay
    (replayed spans of two draw batches, eager generations around them and
    for spans holding a gamma = 1 generation, counts that cut a batch),
    and the same acceptance tally."""
    from paper_0812_2976_gb300 import synth
    import oracle
    w = synth.uniform(1, n_sys=256)
    v = oracle.predict(w.truth, w.t, w.n_pl)[0] + w.noise
    runs = []
    for use_graph in (False, True):
        mc = kc.DEMCMC(dev(w.params), dev(w.t), dev(v), dev(w.sigma), mode="mixed",
                       eps_scale=1e-6, hop_every=hop_every, seed=11, draw_batch=batch)
        mc.run(generations - 5, use_graph=use_graph)
        mc.run(5, use_graph=use_graph)
        assert mc.generation == generations
        runs.append((mc.states.cpu().numpy(), mc.chi2.cpu().numpy(), mc.acceptance))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert np.median(runs[0][1]) < np.median(oracle.chi2(w.params, w.t, v, w.sigma, w.n_pl))
