"""The benchmark's roofline numerators: FLOPs per planet-observation
evaluation of each path, as derived from the kernels' algorithms (no GPU
needed).  A change to a count that the kernels did not make fails here."""
import bench


def test_mixed_chi2_flops():
    # mean anomaly 18, start 18, sin/cos 27, Halley 11, update 10, velocity 8,
    # planet Kahan 4, the per-observation residual and Kahan 10 over n_pl
    assert bench.mixed_flops_per_eval(4, warp=True) == 98.5
    assert bench.mixed_flops_per_eval(4) == bench.mixed_flops_per_eval(4, warp=True)
    assert bench.mixed_flops_per_eval(1) == 96 + 10


def test_adjoint_and_gauss_newton_flops():
    # the adjoint: the forward's 96 + 44 per planet-observation, 12 (not 10)
    # per observation
    assert bench.grad_flops_per_eval(3) == 96 + 44 + 12 / 3
    # Gauss-Newton: + the row of U, 5 per planet and 1 per observation
    assert abs(bench.gn_flops_per_eval(3) - (144 + 5 + 1 / 3)) < 1e-12


def test_gauss_newton_tensor_flops_per_variant():
    # mma.sync at n_pl = 3 (16 parameters): two 16 x 8 tiles on or above the
    # diagonal, three TF32 products, 2 FLOP per MAC, per observation
    assert bench.gn_tensor_flops_per_obs(3, 0) == 2 * 3 * 16 * 8 * 2
    # tcgen05: 64 x 64 tiles of four systems, two products (hi hi, lo hi)
    assert bench.gn_tensor_flops_per_obs(3, 4) == 64 * 64 * 2 * 2 / 4
    # n_pl = 4 (21 parameters, mma.sync only): m-tile 0 with n-tiles 0-2 and
    # m-tile 1 with n-tile 2 reach the upper triangle
    assert bench.gn_tensor_flops_per_obs(4, 0) == 4 * 3 * 16 * 8 * 2


def test_fp64_flops():
    # mean anomaly 6, table sin/cos 20, Halley 13, update 8, velocity and sum 11
    assert bench.F64_FLOPS_PER_EVAL == 58
