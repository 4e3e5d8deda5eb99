import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def pytest_sessionstart(session):
    """Build the CUDA library (by path: the package import needs it built) and the oracle."""
    import importlib.util
    for name, rel in (("_tvlbm_build", ("paper_1004_5059_gb300", "build.py")), ("_oracle_build", ("oracle", "build.py"))):
        spec = importlib.util.spec_from_file_location(name, os.path.join(ROOT, *rel))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
