import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")


def golden_path(name: str) -> str:
    return os.path.join(GOLDEN, name)


def read_golden(name: str):
    """Non-comment lines of a golden fixture, split on '|'."""
    rows = []
    with open(golden_path(name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([f.strip() for f in line.rstrip("\n").split("|")])
    return rows


@pytest.fixture
def golden():
    return read_golden


def pytest_terminal_summary(terminalreporter):
    """Shares of the bounded semantic comparisons of the session: cases that
    passed only because they lie within twice the oracle's float32 running
    error bound, and cases whose bound is infinite (excused)."""
    mod = sys.modules.get("gpu_util")
    shares = getattr(mod, "SHARES", None) if mod is not None else None
    if not shares:
        return
    terminalreporter.write_line("")
    terminalreporter.write_line("bounded semantic comparisons (outside 1e-4 (1 + |v|) of float64):")
    for label, n, b, a in shares:
        terminalreporter.write_line(
            f"  {label}: {n} cases, within 2x the float32 bound {b:.2e}, infinite bound {a:.2e}")
