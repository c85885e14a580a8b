import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _has_hypothesis() -> bool:
    try:
        import hypothesis  # noqa: F401
        return True
    except ImportError:
        return False


# The two randomised property modules are CPU-only and need hypothesis. Where
# it is not installed they are left out of collection rather than reported as
# skipped modules (a module-level skip shows up even in a `-m gpu` run, where
# these modules would be deselected anyway).
collect_ignore = [] if _has_hypothesis() else ["test_oracle_properties.py",
                                               "test_shard_properties.py"]


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def _cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
