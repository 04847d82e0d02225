import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_solar_system():
    import numpy as np
    names, rows = [], []
    with open(os.path.join(GOLDEN, "solar_system.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            names.append(parts[0])
            rows.append([float(p) for p in parts[1:]])
    a = np.array(rows)
    k = 0.01720209895
    return names, a[:, 0].copy(), a[:, 1:4].copy(), a[:, 4:7].copy(), k * k
