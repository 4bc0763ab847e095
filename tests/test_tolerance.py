"""The gradient parity helpers must fail a row that is wrong, NaN on one
side, or nonzero where the oracle's bound is zero (no GPU needed)."""
import numpy as np
from tolerance import U32, grad_excess, grad_excess_ragged, grad_ratios


def rows():
    rng = np.random.default_rng(0)
    ref = rng.normal(0, 10, (4, 6))
    gabs = np.abs(ref) * 3 + 1.0
    return ref, gabs


def test_exact_copy_passes():
    ref, gabs = rows()
    assert grad_excess(ref.copy(), ref, gabs, 1e-3, U32) == 0.0
    assert grad_excess_ragged(ref.ravel(), ref.ravel(), gabs.ravel(), [0, 6, 12, 18, 24],
                              1e-3, U32) == 0.0


def test_planted_nan_fails_both_helpers():
    ref, gabs = rows()
    got = ref.copy()
    got[2, 3] = np.nan
    assert grad_excess(got, ref, gabs, 1e-3, U32) > 1.0
    assert grad_excess_ragged(got.ravel(), ref.ravel(), gabs.ravel(), [0, 6, 12, 18, 24],
                              1e-3, U32) > 1.0
    # NaN in the oracle only fails too; NaN on both sides (an invalid system) matches
    ref2 = ref.copy()
    ref2[1, 0] = np.nan
    assert grad_excess(ref, ref2, gabs, 1e-3, U32) > 1.0
    assert grad_excess(ref2, ref2, gabs, 1e-3, U32) == 0.0


def test_planted_wrong_value_fails_both_helpers():
    ref, gabs = rows()
    got = ref.copy()
    got[0, 5] *= 1.01
    assert grad_excess(got, ref, gabs, 1e-3, U32) > 1.0
    assert grad_excess_ragged(got.ravel(), ref.ravel(), gabs.ravel(), [0, 6, 12, 18, 24],
                              1e-3, U32) > 1.0


def test_zero_bound_row_must_match_exactly():
    """A system without observations: oracle gradient and gabs are 0, so the
    bound is 0 (0/0 before); zero passes, anything else fails."""
    ref, gabs = rows()
    ref[3] = 0.0
    gabs[3] = 0.0
    got = ref.copy()
    assert grad_excess(got, ref, gabs, 1e-3, U32) == 0.0
    got[3, 1] = 1e-30
    assert np.isinf(grad_ratios(got, ref, gabs, 1e-3, U32)[3, 1])
    assert grad_excess_ragged(got.ravel(), ref.ravel(), gabs.ravel(), [0, 6, 12, 18, 24],
                              1e-3, U32) > 1.0


def test_ragged_rows_of_different_lengths():
    ref = np.arange(1.0, 12.0)
    gabs = np.abs(ref)
    off = [0, 6, 6, 11]                     # the middle system has no parameters
    assert grad_excess_ragged(ref, ref, gabs, off, 1e-3, U32) == 0.0
    got = ref.copy()
    got[-1] = np.inf
    assert grad_excess_ragged(got, ref, gabs, off, 1e-3, U32) > 1.0


def test_derived_terms_only_where_the_terms_cancel():
    """Non-cancelling components keep the base bound; cancelling ones add
    (KAPPA_FORM + accumulation) u sum|c| and the residual term."""
    from tolerance import KAPPA_FORM, Arith, grad_bound
    ref = np.array([[1.0, 1e-4, 1e-4, 2.0]])
    gabs = np.array([[5.0, 100.0, 100.0, 2.0]])       # columns 1, 2 cancel
    comp = np.array([False, True, False, False])       # column 1 compensated
    resid = np.array([[7.0, 3e-9, 5e-9, 11.0]])
    ar = Arith(lanes=32, n_obs=512, compensated=comp, resid=resid)
    core = grad_bound(ref, gabs, 1e-3, U32)
    b = grad_bound(ref, gabs, 1e-3, U32, ar)
    assert b[0, 0] == core[0, 0] and b[0, 3] == core[0, 3]
    assert np.isclose(b[0, 1], core[0, 1] + (KAPPA_FORM + 2) * U32 * 100.0 + 3e-9)
    assert np.isclose(b[0, 2], core[0, 2] + (KAPPA_FORM + 16 + 5) * U32 * 100.0 + 5e-9)
    # a planted error just above a cancelling component's bound fails
    got = ref.copy()
    got[0, 2] += 1.01 * b[0, 2]
    assert grad_excess(got, ref, gabs, 1e-3, U32, ar) > 1.0
    got[0, 2] = ref[0, 2] + 0.99 * b[0, 2]
    assert grad_excess(got, ref, gabs, 1e-3, U32, ar) <= 1.0


def test_residual_error_grows_towards_pericentre(oracle_mod):
    """eps_k of the residual bound: circular orbits give the constant part;
    an eccentric orbit's largest value sits at pericentre (D = 1 - e)."""
    from tolerance import KAPPA_M, residual_error
    t = np.linspace(0.0, 10.0, 2001)
    circ = np.array([[10.0, 5.0, 0.0, 0.3, 0.0, 0.0]])
    ecc = np.array([[10.0, 5.0, 0.9, 0.3, 0.0, 0.0]])
    v = np.zeros_like(t)
    e0 = residual_error(oracle_mod, circ, t, v, 1, 0.0, U32)[0]
    e9 = residual_error(oracle_mod, ecc, t, v, 1, 0.0, U32)[0]
    assert np.allclose(e0, U32 * (5.0 * (KAPPA_M + 3 + 18) + 3 * np.abs(
        oracle_mod.predict(circ, t, 1)[0])), rtol=1e-12)
    k = int(np.argmax(e9))
    M = oracle_mod.mean_anomaly(t[k], 0.0, 10.0, 0.0)
    assert abs(np.remainder(M + np.pi, 2 * np.pi) - np.pi) < 0.05     # at pericentre
    # K ((KAPPA_M + 3) / D^2 + 18 / D) at D = 1 - e = 0.1, plus 3 |V| (< 1 % here)
    assert np.isclose(e9.max(), U32 * 5.0 * ((KAPPA_M + 3) / 0.1 ** 2 + 18 / 0.1), rtol=0.01)


def test_mean_anomaly_float_error_bound():
    """KAPPA_M: the mixed path's mean anomaly (phase frac(tau/P) + c from
    float pairs, its low part formed already times 2 pi, one final FMA with
    the float 2 pi) emulated in float32 on 10^6 random phases stays within
    KAPPA_M u of the exact value, and the bound is not loose by more than
    a factor of two (a dropped term would show)."""
    from tolerance import KAPPA_M
    rng = np.random.default_rng(3)
    n = 1_000_000
    f32 = np.float32

    def fma(x, y, z):      # float32 FMA: the exact product of two floats fits a double
        return (np.float64(1) * x * y + z).astype(f32)

    magic = f32(1.5 * 2 ** 23)

    def rnd(x):
        return ((x + magic) - magic).astype(f32)

    P = np.exp(rng.uniform(0, np.log(4000), n))
    tau = rng.uniform(0, 6000, n)
    c = rng.uniform(-0.5, 0.5, n)
    inv = 1.0 / P
    n_hi = inv.astype(f32)
    n_lo = (inv - n_hi).astype(f32)
    c_hi = c.astype(f32)
    c_lo = (c - c_hi).astype(f32)
    th = tau.astype(f32)
    tl = (tau - th).astype(f32)
    two_pi = np.full(n, f32(2 * np.pi))
    p = (th * n_hi).astype(f32)
    pe = fma(th, n_hi, -p)
    lo = fma(fma(tl, n_hi, pe), two_pi, fma(th, (n_lo * two_pi).astype(f32),
                                             (c_lo * two_pi).astype(f32)))
    u = ((p - rnd(p)).astype(f32) + c_hi).astype(f32)
    u = (u - rnd(u)).astype(f32)
    M = fma(u, two_pi, lo).astype(np.float64)
    exact = tau / P + c
    exact = (exact - np.round(exact)) * 2 * np.pi
    err = np.abs(M - exact)
    err = np.minimum(err, np.abs(err - 2 * np.pi))
    assert err.max() <= KAPPA_M * U32
    assert err.max() > 0.5 * KAPPA_M * U32
