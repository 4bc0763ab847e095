"""ctypes loader for libkc.so (the C ABI declared in include/kc.h).

The library must have been built (``paper_0812_2976_gb300.build.build()``);
there is no fallback: every computation runs in the CUDA kernels, and a
missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os
import threading

# KC_LIBRARY selects another build of the same library (the KC_DEBUG build,
# libkc_debug.so, in its test); by default the in-tree libkc.so.  Either
# way a missing file raises.
LIB_PATH = (os.environ.get("KC_LIBRARY") or
            os.path.join(os.path.dirname(os.path.abspath(__file__)), "libkc.so"))

KC_OK, KC_ERR_ARG, KC_ERR_CUDA, KC_ERR_NOMEM, KC_ERR_UNSUPPORTED = range(5)
KC_FP64, KC_MIXED, KC_FP32 = 0, 1, 2
KC_MAX_PLANETS = 8

_lock = threading.Lock()
_lib = None

_d = ctypes.c_void_p          # device pointers are passed as raw addresses
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f64 = ctypes.c_double
_st = ctypes.c_void_p         # kc_stream (cudaStream_t)

KC_KERNEL_CHI2, KC_KERNEL_GRAD, KC_KERNEL_GN = 0, 1, 2


class KcTile(ctypes.Structure):
    """struct kc_tile of include/kc.h."""
    _fields_ = [("threads_per_system", ctypes.c_int32), ("block", ctypes.c_int32),
                ("split", ctypes.c_int32)]


_tile_p = ctypes.POINTER(KcTile)

# name -> (restype, argtypes); the same order as include/kc.h
SIGNATURES = {
    "kc_chi2_eval": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _d, _st]),
    "kc_chi2_eval_mixed": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _d, _d, _st]),
    "kc_chi2_eval_ex": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _f64, _f64, _i32,
                               _d, _d, _st]),
    "kc_chi2_eval_mixed_noalloc": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _f64, _f64, _d,
                                          _d, _st]),
    "kc_chi2_grad": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _f64, _f64, _i32, _d,
                            _d, _st]),
    "kc_chi2_gauss_newton": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _f64, _f64, _i32, _d, _d,
                                     _d, _st]),
    "kc_nll_eval": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _f64, _i32, _d, _st]),
    "kc_nll_grad": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _f64, _i32, _d, _d, _st]),
    "kc_demcmc_step": (_i32, [_d, _d, _i64, _i32, _d, _d, _d, _i32, _f64, _f64, _i32, _i64,
                              _i64, _i64, _i64, _f64, _d, _d, _d, _d, _d, _d, _st]),
    "kc_rv_predict": (_i32, [_d, _d, _i64, _i32, _i32, _f64, _d, _st]),
    "kc_rv_predict_ragged": (_i32, [_d, _d, _d, _d, _d, _i64, _f64, _d, _st]),
    "kc_kepler_solve": (_i32, [_d, _d, _i64, _i32, _d, _st]),
    "kc_plan_create_ragged": (_i32, [ctypes.POINTER(ctypes.c_void_p), _d, _d, _i64, _f64,
                                     _f64, _i32, _i32]),
    "kc_plan_sizes": (_i32, [ctypes.c_void_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "kc_plan_set_observations": (_i32, [ctypes.c_void_p, _d, _d, _d, _st]),
    "kc_plan_run": (_i32, [ctypes.c_void_p, _d, _d, _d, _st]),
    "kc_plan_autotune": (_i32, [ctypes.c_void_p, _d, _d, _d, ctypes.POINTER(_i32),
                                ctypes.POINTER(_i32), _st]),
    "kc_plan_destroy": (None, [ctypes.c_void_p]),
    "kc_set_tile": (_i32, [_i32, _i32, _i64, _i32, _i32, _tile_p]),
    "kc_get_tile": (_i32, [_i32, _i32, _i64, _i32, _i32, _tile_p]),
    "kc_autotune": (_i32, [_d, _d, _d, _d, _i64, _i32, _i32, _i32, _i32, _tile_p,
                           ctypes.POINTER(ctypes.c_float), _st]),
    "kc_status_string": (ctypes.c_char_p, [_i32]),
    "kc_last_device_error": (_i32, [ctypes.POINTER(_i64)]),
    "kc_measure_pipe_rate": (_i32, [_i32, ctypes.POINTER(ctypes.c_double), _st]),
    "kc_last_error": (ctypes.c_char_p, []),
    "kc_debug_word": (_i32, [ctypes.POINTER(ctypes.c_uint64)]),
    "kc_version": (_i32, []),
}


class KcError(RuntimeError):
    def __init__(self, status: int, fn: str, detail: str):
        self.status = status
        super().__init__(f"{fn} failed with status {status}: {detail}")


def load() -> ctypes.CDLL:
    """Load libkc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, fn: str) -> None:
    if status != KC_OK:
        lib = load()
        detail = lib.kc_last_error().decode() or lib.kc_status_string(status).decode()
        raise KcError(status, fn, detail)
