import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")
    try:  # the oracle's OpenMP CSR product (gcc, a second at most); the oracle uses scipy's product without it
        from oracle import build_oracle
        build_oracle.build()
    except Exception:
        pass
