"""The FMA-pipe probe behind the roofline denominators (kc_measure_pipe_rate)
returns rates consistent with GB300's unit counts: 128 FP32 lanes per SM,
and an FP64 rate 1/64 of that."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kc():
    import paper_0812_2976_gb300 as kc
    from paper_0812_2976_gb300 import build
    build.build()
    kc._lib.load()
    return kc


def test_fma_pipe_rates(kc):
    f32 = kc.kc_measure_pipe_rate("fp32")
    f64 = kc.kc_measure_pipe_rate("fp64")
    assert 100.0 <= f32 <= 129.0, f32
    assert 0.5 <= f64 <= 4.0, f64
    assert f32 / f64 > 20.0


def test_probe_rejects_bad_pipe(kc):
    import ctypes
    lib = kc._lib.load()
    r = ctypes.c_double(0.0)
    assert lib.kc_measure_pipe_rate(7, ctypes.byref(r), None) == kc._lib.KC_ERR_ARG
