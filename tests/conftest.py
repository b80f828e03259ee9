import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running full-size case")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


def with_dep_removed(arc, block):
    """The archive with one block's dependency intervals pointed at block 0:
    its real source blocks leave any seek closure (a corruption made on the
    host; the archive's bytes are otherwise unchanged)."""
    import numpy as np

    bad = arc.copy()
    hdr = arc[:64].view(np.uint64)
    nb, deps_off = int(hdr[3]), int(hdr[5])
    ptr = bad[deps_off:deps_off + 4 * (nb + 1)].view(np.uint32)
    ivs = bad[deps_off + 4 * (nb + 1):].view(np.uint32)
    for i in range(int(ptr[block]), int(ptr[block + 1])):
        ivs[2 * i] = 0
        ivs[2 * i + 1] = 0
    return bad
