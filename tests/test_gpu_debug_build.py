"""The KC_DEBUG build of the library (device index checks that record the
first failure in a word and skip the access, never trapping): the GPU parity
suites run against it in a child process, and after every test the word
must still be zero.  Only valid inputs reach the GPU here; invalid offsets
and sizes are refused on the host (tests/test_abi.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_ragged.py", "tests/test_gpu_nll.py",
          "tests/test_gpu_demcmc.py", "tests/test_gpu_gauss_newton.py"]


def test_parity_suites_leave_the_index_word_zero():
    from conftest import ROOT
    from paper_0812_2976_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, KC_LIBRARY=lib, KC_DEBUG_WORD="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *SUITES, "-m", "gpu", "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
