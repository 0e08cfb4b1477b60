import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test (oracle physics runs)")


def pytest_terminal_summary(terminalreporter):
    """Print the achieved parity figures of the session (and write them as
    JSON to $TLB_PARITY_RECORD when it is set)."""
    try:
        import helpers
    except ImportError:
        return
    if not helpers.RECORDS:
        return
    import json

    terminalreporter.write_sep("-", "achieved parity figures")
    for r in helpers.RECORDS:
        terminalreporter.write_line(json.dumps(r))
    path = os.environ.get("TLB_PARITY_RECORD")
    if path:
        with open(path, "w") as fh:
            json.dump(helpers.RECORDS, fh, indent=1)
