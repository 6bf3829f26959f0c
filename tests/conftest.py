import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def load_exact_ln_dos(L: int) -> np.ndarray:
    """ln g(e) from the committed fixture written by tests/golden/make_exact_dos.py."""
    vals = []
    with open(os.path.join(GOLDEN, f"exact_dos_L{L}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = line.split()
            vals.append(float(parts[1]))
    return np.array(vals, dtype=np.float64)


def load_exact_dos_integers(L: int) -> list:
    vals = []
    with open(os.path.join(GOLDEN, f"exact_dos_L{L}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            vals.append(int(line.split()[2]))
    return vals


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.lib()
    return oracle
