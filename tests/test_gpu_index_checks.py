"""The debug build, libne_debug.so: every kernel compiled with
NE_INDEX_CHECKS, whose key accesses (copy windows, gathers, tap-table
blocks, output rows and tiles, batch jobs and units) test their indices and
record a violation in a status word instead of making the access.

In a normal run, one test builds it and runs the parity suites of the
convolution kernels through it in a child process (NE_INDEX_CHECKS=1 makes
the binding load it).  There, every GPU test must leave the status word
clear (the check is in tests/conftest.py), and the self-test below shows
that a failing check is recorded with its site and index and that the
access under it is skipped."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CHECKED = os.environ.get("NE_INDEX_CHECKS") == "1"
SUITES = ["test_gpu_index_checks.py", "test_gpu_parity.py", "test_gpu_tcr.py",
          "test_gpu_batch.py", "test_gpu_small.py"]


@pytest.fixture(scope="module")
def ne():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_03838_gb300 import ne as nemod
    return nemod


@pytest.mark.skipif(CHECKED, reason="runs the child, not in it")
def test_parity_suites_through_the_debug_build(ne):
    from paper_1509_03838_gb300 import build
    build.build()
    build.build(debug=True)
    env = dict(os.environ, NE_INDEX_CHECKS="1")
    out = subprocess.run(
        [sys.executable, "-m", "pytest", *[os.path.join(HERE, f) for f in SUITES],
         "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
         "-k", "not earlier_tensor_core_kernels"],
        env=env, capture_output=True, text=True, timeout=1500)
    assert out.returncode == 0, out.stdout[-4000:] + out.stderr[-2000:]
    assert " passed" in out.stdout and " failed" not in out.stdout


@pytest.mark.skipif(not CHECKED, reason="needs libne_debug.so (NE_INDEX_CHECKS=1)")
def test_index_check_records_and_skips(ne):
    assert ne.LIB_PATH.endswith("libne_debug.so")
    ne.ne_debug_index_status(clear=True)
    assert ne.ne_debug_index_selftest(5, 10) == 1       # in range: access made
    assert ne.ne_debug_index_status(clear=False) == (0, 0)
    assert ne.ne_debug_index_selftest(10, 10) == 0      # one past the end
    assert ne.ne_debug_index_status(clear=False) == (1, (1 << 48) | 10)
    assert ne.ne_debug_index_selftest(-1, 10) == 0      # negative: first kept
    assert ne.ne_debug_index_status(clear=True) == (2, (1 << 48) | 10)
    assert ne.ne_debug_index_status(clear=True) == (0, 0)
    assert ne.ne_debug_index_selftest(-1, 10) == 0
    assert ne.ne_debug_index_status(clear=True) == (1, (1 << 48) | ((1 << 48) - 1))
