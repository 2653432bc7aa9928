"""pytest configuration: the `gpu` marker, import paths, and an up-to-date
build of the CUDA library and the C oracle before any test imports them.

Tests marked ``gpu`` need a GB300 and the CUDA library built for sm_103a;
everything else runs on the CPU (``-m "not gpu"``)."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    import __graft_entry__

    __graft_entry__.build()   # no-op when the builds are current
