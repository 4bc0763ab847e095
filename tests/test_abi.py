"""Host-side checks of the C ABI: the library loads, exports every function
include/kc.h declares, and rejects bad arguments before launching anything.
No call here reaches a kernel, so these run without a GPU."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "kc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_0812_2976_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for want in ("kc_chi2_eval", "kc_chi2_eval_mixed", "kc_chi2_eval_ex", "kc_chi2_grad",
                 "kc_rv_predict", "kc_kepler_solve", "kc_status_string", "kc_last_error",
                 "kc_last_device_error", "kc_plan_create_ragged", "kc_plan_run",
                 "kc_plan_destroy", "kc_version"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    from paper_0812_2976_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_status_strings(lib):
    assert lib.kc_status_string(0) == b"ok"
    assert lib.kc_status_string(1) == b"invalid argument"
    assert lib.kc_version() >= 100


def test_bad_arguments_rejected_on_host(lib):
    p = ctypes.c_void_p(64)        # never dereferenced: checks fail first
    # n_pl out of range
    assert lib.kc_chi2_eval(p, p, p, p, 4, 0, 8, p, None) == 1
    assert b"n_pl" in lib.kc_last_error()
    assert lib.kc_chi2_eval(p, p, p, p, 4, 9, 8, p, None) == 1
    # negative sizes
    assert lib.kc_chi2_eval(p, p, p, p, -1, 2, 8, p, None) == 1
    assert lib.kc_chi2_eval(p, p, p, p, 4, 2, -3, p, None) == 1
    # NULL inputs / outputs
    assert lib.kc_chi2_eval(None, p, p, p, 4, 2, 8, p, None) == 1
    assert lib.kc_chi2_eval_mixed(p, p, p, p, 4, 2, 8, None, None, None) == 1
    assert lib.kc_chi2_grad(p, p, p, p, 4, 2, 8, 0.0, 0.0, 1, None, None, None) == 1
    # misaligned double pointer
    assert lib.kc_chi2_eval(ctypes.c_void_p(68), p, p, p, 4, 2, 8, p, None) == 1
    assert b"aligned" in lib.kc_last_error()
    # bad mode, non-finite epoch
    assert lib.kc_chi2_eval_ex(p, p, p, p, 4, 2, 8, 0.0, 0.0, 7, p, None, None) == 1
    assert lib.kc_chi2_eval_ex(p, p, p, p, 4, 2, 8, float("nan"), 0.0, 1, p, None, None) == 1
    assert lib.kc_kepler_solve(p, p, -1, 0, p, None) == 1
    assert lib.kc_rv_predict(p, p, 2, 0, 4, 0.0, p, None) == 1
    assert lib.kc_last_device_error(None) == 1
    # Gauss-Newton: bad mode, n_pl, non-finite t0, misaligned output, NULL matrix
    assert lib.kc_chi2_gauss_newton(p, p, p, p, 4, 2, 8, 0.0, 0.0, 2, None, None, p, None) == 1
    assert lib.kc_chi2_gauss_newton(p, p, p, p, 4, 9, 8, 0.0, 0.0, 1, None, None, p, None) == 1
    assert lib.kc_chi2_gauss_newton(p, p, p, p, 4, 2, 8, float("inf"), 0.0, 1, None, None, p,
                                    None) == 1
    assert lib.kc_chi2_gauss_newton(p, p, p, p, 4, 2, 8, 0.0, 0.0, 0, ctypes.c_void_p(68), None,
                                    p, None) == 1
    assert lib.kc_chi2_gauss_newton(p, p, p, p, 4, 2, 8, 0.0, 0.0, 1, None, None, None, None) == 1
    assert lib.kc_measure_pipe_rate(0, None, None) == 1
    # KC_DEBUG index word: a normal build has none
    w = ctypes.c_uint64(7)
    assert lib.kc_debug_word(ctypes.byref(w)) == 4 and w.value == 0
    assert lib.kc_debug_word(None) == 1
    # the allocation-free call refuses sizes whose scratch size would wrap
    assert lib.kc_chi2_eval_mixed_noalloc(p, p, p, p, (1 << 62) + 1, 8, 16, 0.0, 0.0, p, None,
                                          None) == 1
    assert b"too large" in lib.kc_last_error()
    # DE-MC step: the partner range must be inside the population, hold two
    # chains and not overlap the updated chains (states, n_chains = 16,
    # n_pl = 1, ..., first = 0, count = 8, partner_first, partner_count)
    for pf, pc, msg in ((4, 8, b"overlaps"), (8, 1, b"partner_count"), (10, 8, b"partner_count")):
        assert lib.kc_demcmc_step(p, p, 16, 1, p, p, p, 8, 0.0, 0.0, 1, 0, 8, pf, pc, 0.5,
                                  p, p, p, p, p, None, None) == 1
        assert msg in lib.kc_last_error()
    # ... and gamma, the epoch and the jitter finite
    for t0, jit, g, msg in ((0.0, 0.0, float("inf"), b"gamma"), (float("nan"), 0.0, 0.5, b"t0"),
                            (0.0, float("inf"), 0.5, b"jitter")):
        assert lib.kc_demcmc_step(p, p, 16, 1, p, p, p, 8, t0, jit, 1, 0, 8, 8, 8, g,
                                  p, p, p, p, p, None, None) == 1
        assert msg in lib.kc_last_error()


def test_ragged_plan_offsets_checked_on_host(lib):
    """Offsets that decrease, overflow or exceed the observation limits are
    refused before any device memory is touched; so are bad planet counts."""
    plan = ctypes.c_void_p()

    def create(off, npl):
        off = (ctypes.c_int64 * len(off))(*off)
        npl = (ctypes.c_int32 * len(npl))(*npl)
        return lib.kc_plan_create_ragged(ctypes.byref(plan), off, npl, len(npl), 0.0, 0.0, 1, 0)
    i64max, i64min = 2 ** 63 - 1, -2 ** 63
    for off, npl, msg in (([1, 5], [1], b"obs_off[0]"),
                          ([0, 5, 3], [1, 1], b"decreases"),
                          ([0, 16, i64min], [1, 1], b"decreases"),        # would wrap
                          ([0, 16, i64max], [1, 1], b"observations"),
                          ([0, (1 << 24) + 1], [1], b"observations"),
                          ([0, 4], [0], b"n_pl"), ([0, 4], [9], b"n_pl")):
        assert create(off, npl) == 1, (off, npl)
        assert msg in lib.kc_last_error(), (msg, lib.kc_last_error())
        assert not plan.value
    assert lib.kc_plan_create_ragged(ctypes.byref(plan), ctypes.c_void_p(64), ctypes.c_void_p(64),
                                     (1 << 40) + 1, 0.0, 0.0, 1, 0) == 1
    assert b"too large" in lib.kc_last_error()


def test_empty_batches_are_no_ops(lib):
    p = ctypes.c_void_p(64)
    assert lib.kc_chi2_eval(p, p, p, p, 0, 2, 8, p, None) == 0
    assert lib.kc_chi2_grad(p, p, p, p, 0, 3, 8, 0.0, 0.0, 0, None, p, None) == 0
    assert lib.kc_kepler_solve(p, p, 0, 1, p, None) == 0
    assert lib.kc_rv_predict(p, p, 0, 2, 8, 0.0, p, None) == 0
    assert lib.kc_last_error() == b""


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_0812_2976_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libkc.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_tile_table_host_logic(lib):
    from paper_0812_2976_gb300 import _lib
    t = _lib.KcTile()
    # default heuristic for the paper-shaped batch
    assert lib.kc_get_tile(0, 1, 4096, 4, 256, ctypes.byref(t)) == 0
    # mixed chi2: the persistent kernel, lanes per system 8/16/32 and whole warps
    assert t.split == 3 and t.threads_per_system == 32
    assert t.block % 32 == 0 and 32 <= t.block <= 1024
    default = (t.threads_per_system, t.block, t.split)
    assert lib.kc_get_tile(0, 1, 4096, 4, 32, ctypes.byref(t)) == 0
    assert (t.threads_per_system, t.split) == (8, 3)             # 4 observations per lane
    assert lib.kc_get_tile(0, 0, 4096, 4, 256, ctypes.byref(t)) == 0
    assert t.block in (64, 128, 256) and t.split == 0           # FP64 kernel
    # pin, read back, same size class (power-of-two bucket), then remove
    pin = _lib.KcTile(16, 128, 1)
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, ctypes.byref(pin)) == 0
    assert lib.kc_get_tile(0, 1, 5000, 4, 300, ctypes.byref(t)) == 0
    assert (t.threads_per_system, t.block, t.split) == (16, 128, 1)
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, None) == 0
    assert lib.kc_get_tile(0, 1, 4096, 4, 256, ctypes.byref(t)) == 0
    assert (t.threads_per_system, t.block, t.split) == default
    # inadmissible tiles are refused
    for bad in ((3, 128, 0), (64, 32, 0), (256, 128, 0), (64, 256, 0), (8, 16, 0), (8, 64, 2)):
        kern = 1 if bad[:2] == (64, 256) else 0
        assert lib.kc_set_tile(kern, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(*bad))) == 1
    # split = 2: threads_per_system = 32 x chunks, may exceed the block
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(512, 64, 2))) == 0
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(16, 64, 2))) == 1
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(2048, 64, 2))) == 1
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, None) == 0
    # split = 3 (warp kernel): 8 to 128 lanes (64, 128: a system over two or
    # four warps), whole warps up to 1024 threads, whole systems per CTA
    for good in ((32, 288, 3), (8, 1024, 3), (16, 32, 3), (64, 128, 3), (128, 1024, 3)):
        assert lib.kc_set_tile(0, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(*good))) == 0
    for bad in ((4, 128, 3), (32, 100, 3), (32, 2048, 3), (64, 96, 3), (128, 64, 3),
                (256, 256, 3), (48, 96, 3)):
        assert lib.kc_set_tile(0, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(*bad))) == 1
    assert lib.kc_set_tile(1, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(32, 288, 3))) == 1
    assert lib.kc_set_tile(0, 0, 4096, 4, 256, ctypes.byref(_lib.KcTile(32, 288, 3))) == 1
    assert lib.kc_set_tile(0, 1, 4096, 4, 256, None) == 0
    # the split variants exist for the mixed chi2 kernel only
    assert lib.kc_set_tile(0, 0, 4096, 4, 256, ctypes.byref(_lib.KcTile(8, 64, 1))) == 1
    assert lib.kc_set_tile(1, 1, 4096, 4, 256, ctypes.byref(_lib.KcTile(8, 64, 1))) == 1
    assert lib.kc_get_tile(0, 1, 4096, 0, 256, ctypes.byref(t)) == 1
    # Gauss-Newton (kernel 2, mixed only): split 0 = mma.sync, 4 = tcgen05
    # (n_pl <= 3); one warp per system, 128 threads
    assert lib.kc_get_tile(2, 1, 65536, 3, 512, ctypes.byref(t)) == 0
    assert (t.threads_per_system, t.block, t.split) == (32, 128, 4)     # default: tcgen05
    assert lib.kc_get_tile(2, 1, 65536, 4, 512, ctypes.byref(t)) == 0
    assert (t.threads_per_system, t.block, t.split) == (32, 128, 0)
    assert lib.kc_get_tile(2, 0, 65536, 3, 512, ctypes.byref(t)) == 1
    for split in (4, 0):
        assert lib.kc_set_tile(2, 1, 65536, 3, 512, ctypes.byref(_lib.KcTile(32, 128, split))) == 0
        assert lib.kc_get_tile(2, 1, 65536, 3, 512, ctypes.byref(t)) == 0
        assert (t.threads_per_system, t.block, t.split) == (32, 128, split)
    assert lib.kc_set_tile(2, 1, 65536, 4, 512, ctypes.byref(_lib.KcTile(32, 128, 4))) == 1
    assert lib.kc_set_tile(2, 1, 65536, 4, 512, ctypes.byref(_lib.KcTile(32, 128, 0))) == 0
    for bad in ((16, 128, 4), (32, 256, 4), (32, 128, 3), (32, 128, 1), (32, 128, 5)):
        assert lib.kc_set_tile(2, 1, 65536, 3, 512, ctypes.byref(_lib.KcTile(*bad))) == 1
    assert lib.kc_set_tile(2, 0, 65536, 3, 512, ctypes.byref(_lib.KcTile(32, 128, 0))) == 1
    assert lib.kc_set_tile(3, 1, 65536, 3, 512, ctypes.byref(_lib.KcTile(32, 128, 0))) == 1
    for n_pl in (3, 4):
        assert lib.kc_set_tile(2, 1, 65536, n_pl, 512, None) == 0
