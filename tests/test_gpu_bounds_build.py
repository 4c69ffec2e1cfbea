"""The index-checking debug build (libic_bounds.so, -DIC_BOUNDS_CHECK): every
grid, noise, neighbour-bin and particle index the kernels form is checked
against its array, and any index outside it becomes IC_ERR_ARG at the next
status check.  It stands in for a memory checker.

The parity tests (GPU against the oracle, ragged grids, every tiling and
staging mode, particles on the periodic seam), the rebuilt neighbour lists,
the whole-row kernel's tests, the adjoint's oracle comparisons and seeded
random configurations, and the check's own self-test run once more against
that build in a child process; none may raise a flag.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_selftest_and_variant_flag():
    from paper_1307_0702_gb300 import _lib

    lib = _lib.load()
    if os.environ.get("IC_LIBRARY") == "bounds":
        assert lib.ic_bounds_check_build() == 1
        assert lib.ic_bounds_selftest() == _lib.IC_OK
    else:
        assert lib.ic_bounds_check_build() == 0
        assert lib.ic_bounds_selftest() == _lib.IC_ERR_STATE   # the probe kernel checks nothing here


@pytest.mark.skipif(os.environ.get("IC_LIBRARY") == "bounds", reason="runs the checked build from the plain one")
def test_parity_suite_under_index_checks():
    from paper_1307_0702_gb300 import build

    build.build(bounds_check=True)
    env = dict(os.environ, IC_LIBRARY="bounds")
    files = ["tests/test_gpu_bounds_build.py", "tests/test_gpu_parity.py", "tests/test_gpu_neighbours.py",
             "tests/test_gpu_rows.py", "tests/test_gpu_adjoint.py"]
    # the adjoint's seeded random configurations and its oracle comparison (short runs)
    select = "not adjoint or random_configurations or matches_the_oracle_adjoint"
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-m", "gpu", "-k", select, "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
