"""pytest configuration: the `gpu` marker and import paths.

Tests marked ``gpu`` need a GB300 and the CUDA library built for sm_103a;
everything else runs on the CPU (``-m "not gpu"``)."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
