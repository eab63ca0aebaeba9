import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture into a dict name -> numpy array."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name)
    out, lines = {}, [l.strip() for l in open(path) if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        name, r, c = lines[i].split()
        r, c = int(r), int(c)
        out[name] = np.array([[float(v) for v in lines[i + 1 + q].split()] for q in range(r)])
        assert out[name].shape == (r, c)
        i += 1 + r
    return out
