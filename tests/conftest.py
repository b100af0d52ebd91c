import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size workload (minutes on the CPU)")


def pytest_terminal_summary(terminalreporter):
    """Per-field parity errors in each field's own norm (recorded by tests._util next to the
    shared velocity-scale bar): the largest per (test, field), printed, and written as JSON to
    the file SWENSE_FIELD_REPORT names, if any."""
    try:
        from tests._util import FIELD_RECORDS
    except ImportError:
        return
    if not FIELD_RECORDS:
        return
    import json
    worst = {}
    for r in FIELD_RECORDS:
        key = (r["test"], r["field"])
        if key not in worst or r["own_norm"] > worst[key]["own_norm"]:
            worst[key] = r
    rows = sorted(worst.values(), key=lambda r: -r["own_norm"])
    terminalreporter.write_line(f"per-field errors (own norm), {len(rows)} (test, field) pairs; "
                                f"largest: " + ", ".join(f"{r['field']} {r['own_norm']:.2e} "
                                                          f"[{r['test'].split('::')[-1]}]" for r in rows[:5]))
    path = os.environ.get("SWENSE_FIELD_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(rows, fh, indent=1)
