"""The GPU suites once more, on the bounds-checking build of the library.

libfpgb300_check.so is compiled with -DFPK_BOUNDS_CHECK: before every global access of the
sweep, the halo packing and the speed and time-step reductions, the element is checked against
the array it belongs to, and every shared-ring offset against the ring.  A violation would be
redirected to the array's first element and recorded in the block's status word, which
fp_get_device_status reports as FP_ERR_BOUNDS (nothing faults).  The parity, slab and
allocation-free suites run in a child process against that build (FPGB300_LIBRARY), with the
audit of tests/conftest.py reading every block's status word when the block is closed: all of
their cases (every scheme, metric order, precision, boundary rule, block link, halo, tile shape
and batch layout they cover) must pass without one out-of-range index.  The three full-size
cases are left out for time; their launch shapes are those of the smaller batch cases."""
import os
import re
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_suites_meet_no_out_of_range_index_in_the_bounds_checking_build():
    from paper_2101_05886_gb300 import build
    lib = build.build(check=True)
    env = dict(os.environ, FPGB300_LIBRARY=lib, FPGB300_BOUNDS_AUDIT="1")
    cmd = [sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "tests/test_gpu_slab.py",
           "tests/test_zz_no_alloc.py", "-m", "gpu", "-q", "-p", "no:cacheprovider", "-k", "not full_size"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=2400)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    passed = re.search(r"(\d+) passed", r.stdout)
    assert passed and int(passed.group(1)) >= 100, tail
