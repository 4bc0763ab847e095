"""kc_chi2_eval_mixed_noalloc: the mixed chi-square for callers that must not
allocate device memory while they evaluate (its intermediate data live in a
fixed array inside libkc.so).  Checked through the C ABI against the regular
kc_chi2_eval_mixed on two calls in a row, with the tolerance of the other
mixed-precision tests.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import paper_0812_2976_gb300 as kc
    from paper_0812_2976_gb300 import build
    build.build()
    return kc._lib.load()


def scratch_limit():
    """KC_NOALLOC_SCRATCH_BYTES as include/kc.h defines it."""
    import os
    import re
    from conftest import ROOT
    text = open(os.path.join(ROOT, "include", "kc.h")).read()
    m = re.search(r"#define KC_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    return int(m.group(1)) << int(m.group(2))


def batch(seed, n_sys, n_pl, n_obs):
    rng = np.random.default_rng(seed)
    cols = []
    for _ in range(n_pl):
        cols += [np.exp(rng.uniform(0, np.log(4000), n_sys)), rng.uniform(1, 100, n_sys),
                 rng.uniform(0, 0.9, n_sys), rng.uniform(0, 2 * np.pi, n_sys),
                 rng.uniform(0, 2 * np.pi, n_sys)]
    params = np.stack(cols + [rng.uniform(-10, 10, n_sys)], axis=1)
    t = np.sort(rng.uniform(2450000, 2454000, n_obs))
    v = rng.normal(0, 40, n_obs)
    sig = rng.uniform(1, 5, n_obs)
    return [torch.tensor(a, dtype=torch.float64, device="cuda") for a in (params, t, v, sig)]


def call_noalloc(lib, P, T, V, S, n_pl, out, resid):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.kc_chi2_eval_mixed_noalloc(P.data_ptr(), T.data_ptr(), V.data_ptr(),
                                          S.data_ptr(), P.shape[0], n_pl, T.numel(), 0.0, 0.0,
                                          out.data_ptr(), resid.data_ptr(), stream)


def call_regular(lib, P, T, V, S, n_pl, out, resid):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.kc_chi2_eval_mixed(P.data_ptr(), T.data_ptr(), V.data_ptr(), S.data_ptr(),
                                  P.shape[0], n_pl, T.numel(), out.data_ptr(), resid.data_ptr(),
                                  stream)


def test_noalloc_matches_regular_entry_point_twice(lib):
    # two different problems in a row: the second call must not see the
    # first call's leftovers in the shared array
    for seed, (n_sys, n_pl, n_obs) in ((1, (4096, 4, 256)), (2, (777, 3, 301))):
        P, T, V, S = batch(seed, n_sys, n_pl, n_obs)
        out = torch.empty(n_sys, dtype=torch.float32, device="cuda")
        resid = torch.empty_like(out)
        ref = torch.empty_like(out)
        ref_resid = torch.empty_like(out)
        assert call_noalloc(lib, P, T, V, S, n_pl, out, resid) == 0, lib.kc_last_error()
        assert call_regular(lib, P, T, V, S, n_pl, ref, ref_resid) == 0, lib.kc_last_error()
        torch.cuda.synchronize()
        a = out.cpu().numpy().astype(np.float64)
        b = ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)) <= MIXED_TOL
        assert float(resid.max()) <= 4e-6


def test_noalloc_rejects_problems_beyond_its_array(lib):
    P, T, V, S = batch(3, 64, 8, 16)
    out = torch.empty(64, dtype=torch.float32, device="cuda")
    limit = scratch_limit()
    n_sys_too_many = limit // 32 + 1          # 32 B per planet alone exceeds the array
    st = lib.kc_chi2_eval_mixed_noalloc(P.data_ptr(), T.data_ptr(), V.data_ptr(), S.data_ptr(),
                                        n_sys_too_many, 8, T.numel(), 0.0, 0.0, out.data_ptr(),
                                        None, None)
    assert st == 1
    assert b"scratch" in lib.kc_last_error()
