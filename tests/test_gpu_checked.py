"""The bounds-checked build (-DAIRGA_CHECKED, libairga_checked.so).

Its kernels test every instrumented index (window and band rows, row
pointers, column indices, transposition maps, factor positions) against the
buffer it addresses and count the misses instead of accessing out of range.

  * test_gpu_suite_under_checked_library runs the whole `-m gpu` suite in a
    child process with AIRGA_LIB=checked: the conftest hook reads the record
    after every test, so each parity case of the band, general-sparse,
    batched, mixed-precision and allocation-free paths doubles as a bounds
    check, and any recorded index fails the run;
  * test_check_records_out_of_range_index (inside that run only) shows that
    the check itself records: one thread tests an index outside [0, bound)
    without touching memory there.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INSIDE = os.environ.get("AIRGA_LIB") == "checked"


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_01216_gb300 import build
    build.build()
    from paper_1606_01216_gb300 import airga
    airga.lib()
    return airga


def test_gpu_suite_under_checked_library(G):
    if INSIDE:
        pytest.skip("this is the checked run")
    from paper_1606_01216_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, AIRGA_LIB="checked")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider",
         "-k", "not test_gpu_suite_under_checked_library"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-6000:] + r.stderr[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " error" not in r.stdout, tail


def test_normal_build_has_no_record(G):
    if INSIDE:
        pytest.skip("the normal library only")
    with pytest.raises(G.AirgaError) as e:
        G.debug_checked()
    assert e.value.code == G.E_UNSUPPORTED
    with pytest.raises(G.AirgaError):
        G.debug_check_selftest(5, 3, 900)


def test_check_records_out_of_range_index(G):
    if not INSIDE:
        pytest.skip("runs inside the checked-library run")
    assert G.lib_path().endswith("libairga_checked.so")
    G.debug_checked()                                  # start from a clear record
    G.debug_check_selftest(2, 3, 901)                  # inside: nothing recorded
    assert G.debug_checked() == (0, 0, 0)
    G.debug_check_selftest(5, 3, 902)                  # past the end
    assert G.debug_checked() == (1, 902, 5)
    G.debug_check_selftest(-1, 3, 903)                 # before the start
    assert G.debug_checked() == (1, 903, -1)
    for k in range(4):                                 # counts accumulate; the first site stays
        G.debug_check_selftest(3 + k, 3, 910 + k)
    assert G.debug_checked() == (4, 910, 3)
    assert G.debug_checked() == (0, 0, 0)              # reading clears
