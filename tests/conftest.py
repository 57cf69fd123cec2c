import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Print the worst GPU-vs-oracle errors the parity checks measured."""
    mod = sys.modules.get("tests.parity_util")
    worst = getattr(mod, "WORST", None) if mod else None
    if worst:
        terminalreporter.write_line("parity worst errors: " +
                                    ", ".join(f"{k} {v:.2e}" for k, v in sorted(worst.items())))
