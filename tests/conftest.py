import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build_c()
    return oracle


class ErrorLog:
    """Measured errors against the oracle, one record per (test, quantity):
    written as JSON at the end of the session when PSPS_ERROR_LOG names a
    file (the table of errors per result and configuration is made from it)."""

    def __init__(self):
        self.rows = []
        self.current = ""

    def note(self, error: float):
        """A relative L2 error computed by the current test (every parity
        comparison goes through _helpers.rel_l2)."""
        self.rows.append({"test": self.current, "quantity": "rel_l2", "error": float(error)})

    def add(self, test: str, quantity: str, error: float, bound: float, **extra):
        self.rows.append({"test": test or self.current, "quantity": quantity, "error": float(error), "bound": float(bound),
                          **{k: (float(v) if isinstance(v, (int, float)) else v) for k, v in extra.items()}})


_ERRORS = ErrorLog()


@pytest.fixture(scope="session")
def error_log():
    return _ERRORS


@pytest.fixture(autouse=True)
def _error_log_context(request):
    _ERRORS.current = request.node.nodeid
    yield


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("PSPS_ERROR_LOG")
    if path and _ERRORS.rows:
        import json
        with open(path, "w") as f:
            json.dump(_ERRORS.rows, f, indent=1)
