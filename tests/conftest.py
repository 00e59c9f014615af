import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line(
        "markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def ed_lib():
    """The built C-ABI library through its Python binding (GPU tests only)."""
    from paper_2005_13498_gb300 import ed
    return ed


@pytest.fixture(scope="session")
def parity_log():
    """Records measured errors of the parity tests as JSON lines in the file
    named by ED_PARITY_LOG (nothing is written when it is unset)."""
    import json
    path = os.environ.get("ED_PARITY_LOG")

    def record(test, **values):
        if path:
            with open(path, "a") as f:
                f.write(json.dumps({"test": test, **{k: float(v) for k, v in values.items()}})
                        + "\n")
    return record
