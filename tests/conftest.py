import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_sessionstart(session):
    """Builds the library and the oracle in-tree when either is missing (a fresh checkout keeps
    no built files); nvcc cross-compiles for sm_103a without a GPU."""
    lib = os.path.join(ROOT, "paper_1403_7294_gb300", "libac.so")
    orc = os.path.join(ROOT, "oracle", "liboracle.so")
    if not (os.path.exists(lib) and os.path.exists(orc)):
        import __graft_entry__

        __graft_entry__.build()


def load_golden(name):
    """Parse a tests/golden/*.txt fixture into a dict of lists of token lists."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(":")
            out.setdefault(key.strip(), []).append(rest.split())
    return out
