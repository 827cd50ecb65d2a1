import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Report how many gradients passed only through the bandflux-derived
    bound (tests/_helpers.assert_grad_close) in this session."""
    try:
        from tests import _helpers as H
    except Exception:
        return
    if not H.FALLBACK_LOG:
        return
    n = sum(r[1] for r in H.FALLBACK_LOG)
    f = sum(r[2] for r in H.FALLBACK_LOG)
    terminalreporter.write_line(f"gradient checks: {len(H.FALLBACK_LOG)} calls, {n} samples, "
                                f"{f} through the bandflux-derived bound only")
    for test, ns, nf in H.FALLBACK_LOG:
        if nf:
            terminalreporter.write_line(f"  {test}: {nf} of {ns}")
