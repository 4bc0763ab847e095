"""kc_chi2_eval_mixed_noalloc: the mixed chi-square for callers that must not
allocate device memory while they evaluate (its intermediate data live in a
fixed array inside libkc.so).  Checked through the C ABI against the regular
kc_chi2_eval_mixed and against the FP64 oracle on two calls in a row, with
the tolerance of the other mixed-precision tests; a second call in a fresh
process must leave the device's free memory unchanged.  This file is
collected last on purpose."""
import os
import subprocess
import sys

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
    import re
    from conftest import ROOT
    text = open(os.path.join(ROOT, "include", "kc.h")).read()
    m = re.search(r"#define KC_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    return int(m.group(1)) << int(m.group(2))


def batch_host(seed, n_sys, n_pl, n_obs):
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
    return params, t, v, sig


def batch(seed, n_sys, n_pl, n_obs):
    return [torch.tensor(a, dtype=torch.float64, device="cuda")
            for a in batch_host(seed, n_sys, n_pl, n_obs)]


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


def test_noalloc_matches_regular_entry_point_and_oracle_twice(lib, oracle_mod):
    # two different problems in a row: the second call must not see the
    # first call's leftovers in the shared array
    for seed, (n_sys, n_pl, n_obs) in ((1, (4096, 4, 256)), (2, (777, 3, 301))):
        host = batch_host(seed, n_sys, n_pl, n_obs)
        P, T, V, S = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in host]
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
        exact = oracle_mod.chi2(host[0], host[1], host[2], host[3], n_pl)
        assert np.max(np.abs(a - exact) / np.maximum(np.abs(exact), 1.0)) <= MIXED_TOL


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


def test_binding_checks_outputs_and_refuses_copies(lib):
    import paper_0812_2976_gb300 as kc
    P, T, V, S = batch(4, 100, 2, 40)
    good = torch.empty(100, dtype=torch.float32, device="cuda")
    for bad in (torch.empty(100, dtype=torch.float64, device="cuda"),     # wrong type
                torch.empty(100, dtype=torch.float32),                     # host memory
                torch.empty(99, dtype=torch.float32, device="cuda"),       # too short
                torch.empty(200, dtype=torch.float32, device="cuda")[::2]):  # strided
        with pytest.raises((TypeError, ValueError)):
            kc.kc_chi2_eval_mixed_noalloc(P, T, V, S, bad)
        with pytest.raises((TypeError, ValueError)):
            kc.kc_chi2_eval_mixed_noalloc(P, T, V, S, good, max_kepler_resid=bad)
    Pn = torch.empty((P.shape[1], P.shape[0]), dtype=torch.float64, device="cuda").t()
    Pn.copy_(P)
    with pytest.raises(ValueError, match="contiguous"):
        kc.kc_chi2_eval_mixed_noalloc(Pn, T, V, S, good)
    kc.kc_chi2_eval_mixed_noalloc(P, T, V, S, good)
    assert torch.isfinite(good).all()


FRESH_PROCESS = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
import paper_0812_2976_gb300 as kc
from paper_0812_2976_gb300 import build
build.build()
lib = kc._lib.load()
sys.path.insert(0, sys.argv[2])
from test_zz_no_alloc import batch, call_noalloc, call_regular
n_pl = 4
P, T, V, S = batch(5, 4096, n_pl, 256)
out = torch.empty(4096, dtype=torch.float32, device="cuda")
resid = torch.empty_like(out)
assert call_noalloc(lib, P, T, V, S, n_pl, out, resid) == 0    # set-up, kernels loaded
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for _ in range(3):
    assert call_noalloc(lib, P, T, V, S, n_pl, out, resid) == 0
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
# positive control: the regular call's two-pass tile takes its scratch from
# the library's memory pool, which the same measurement must see
P2, T2, V2, S2 = batch(6, 65536, n_pl, 256)
kc.kc_set_tile("chi2", "mixed", 65536, n_pl, 256, (16, 256, 1))
out2 = torch.empty(65536, dtype=torch.float32, device="cuda")
resid2 = torch.empty_like(out2)
torch.cuda.synchronize()
free2 = torch.cuda.mem_get_info()[0]
assert call_regular(lib, P2, T2, V2, S2, n_pl, out2, resid2) == 0
torch.cuda.synchronize()
free3 = torch.cuda.mem_get_info()[0]
print(free0, free1, free2, free3)
"""


def test_noalloc_allocates_no_device_memory_in_a_fresh_process():
    """The defining property, measured at the driver: in a process whose only
    library calls so far were no-alloc calls, more of them leave the free
    device memory unchanged, while a regular two-pass call (scratch from the
    library's memory pool) visibly takes some."""
    from conftest import ROOT
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, "-c", FRESH_PROCESS, ROOT, here], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    free0, free1, free2, free3 = (int(x) for x in r.stdout.split()[-4:])
    assert free1 == free0, (free0, free1)
    assert free3 < free2, (free2, free3)
