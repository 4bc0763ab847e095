import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built libkc.so")


@pytest.fixture(autouse=True)
def _kc_debug_word(request):
    """In a run against the KC_DEBUG build of the library (KC_DEBUG_WORD=1,
    set by tests/test_gpu_debug_build.py for its child run), every GPU test
    must leave the device index-check word at zero."""
    yield
    if os.environ.get("KC_DEBUG_WORD") == "1" and request.node.get_closest_marker("gpu"):
        import ctypes
        from paper_0812_2976_gb300 import _lib
        word = ctypes.c_uint64(0)
        status = _lib.load().kc_debug_word(ctypes.byref(word))
        assert status == 0, "the loaded library is not a KC_DEBUG build"
        assert word.value == 0, f"failed device index check: {word.value:#x}"


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
