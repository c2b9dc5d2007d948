import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU runs of the oracle")


def pytest_sessionfinish(session, exitstatus):
    """With LESBGK_PARITY_REPORT set, write every recorded GPU-vs-oracle
    comparison (per field: abs, e, e_own, e_pert, bound, tol) to that file."""
    path = os.environ.get("LESBGK_PARITY_REPORT")
    if not path:
        return
    from tests.common import REPORT
    with open(path, "w") as fh:
        json.dump(REPORT, fh, indent=1)
