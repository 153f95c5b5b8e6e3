import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.lib()
    return O


def pytest_sessionfinish(session, exitstatus):
    """Write the GPU parity margins (achieved per-field errors and bounds of
    every comparison) to the JSON file DGFV_PARITY_MARGINS names, if any."""
    out = os.environ.get("DGFV_PARITY_MARGINS")
    if not out:
        return
    try:
        from tests import gpu_helpers
    except ImportError:
        return
    import json
    with open(out, "w") as f:
        json.dump(gpu_helpers.MARGINS, f, indent=1)
