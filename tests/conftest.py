import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_golden(name):
    """Parse a tests/golden text fixture: '[KEY rows cols]' headers + rows."""
    import numpy as np
    out, key, rows = {}, None, []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                if key:
                    out[key] = np.array(rows, dtype=np.float64).reshape(shape)
                parts = line.strip("[]").split()
                key, shape, rows = parts[0], (int(parts[1]), int(parts[2])), []
                continue
            rows.append([float(x) for x in line.split()])
    if key:
        out[key] = np.array(rows, dtype=np.float64).reshape(shape)
    return out
