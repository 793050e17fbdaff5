import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


_REPORTS = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


@pytest.fixture(scope="session")
def cuda_device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture
def parity_report():
    """report(name, **figures): errors against the oracle measured by a
    parity test, printed together in the terminal summary at the end of the
    run (one line per entry)."""
    def report(name, **figures):
        _REPORTS.append((name, figures))
    return report


def pytest_terminal_summary(terminalreporter):
    if not _REPORTS:
        return
    terminalreporter.section("errors against the oracle (measured by the parity tests)")
    for name, figs in _REPORTS:
        parts = []
        for k, v in figs.items():
            parts.append(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}")
        terminalreporter.write_line(f"{name}: " + ", ".join(parts))
