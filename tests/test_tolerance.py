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
