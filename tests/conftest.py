import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


# Bounds audit: with FPGB300_BOUNDS_AUDIT=1 (and FPGB300_LIBRARY naming the bounds-checking build,
# see tests/test_gpu_bounds_check.py) every block reads its device status word when it is closed,
# and a test fails if any kernel met an index outside its array (FP_ERR_BOUNDS).
if os.environ.get("FPGB300_BOUNDS_AUDIT") == "1":
    @pytest.fixture(autouse=True)
    def _bounds_audit():
        import gc

        import torch

        from paper_2101_05886_gb300 import binding as B
        from paper_2101_05886_gb300 import solver

        assert B.fp_bounds_checking() == 1, "the audit needs the bounds-checking build"
        seen = []
        close = solver.Block.close

        def audited_close(self):
            if self.ctx:
                seen.append(B.lib().fp_get_device_status(self.ctx, torch.cuda.current_stream().cuda_stream))
            close(self)

        solver.Block.close = audited_close
        try:
            yield
            gc.collect()                    # blocks the test left open are closed (and read) here
        finally:
            solver.Block.close = close
        assert seen, "no block was closed"
        assert B.FP_ERR_BOUNDS not in seen, f"a kernel met an out-of-range index ({seen.count(B.FP_ERR_BOUNDS)} blocks)"
