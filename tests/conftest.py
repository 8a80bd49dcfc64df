import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libbbx.so")
    config.addinivalue_line("markers", "slow: longer CPU test")
    # Build the oracle (gcc) and, where nvcc exists, the CUDA library, so a
    # fresh checkout can run the suite directly.
    import oracle
    oracle.build()
    if shutil.which(os.environ.get("NVCC", "nvcc")):
        from paper_1605_06015_gb300 import build as libbuild
        libbuild.build()
