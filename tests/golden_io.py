"""Reader for the golden fixtures in tests/golden (float.hex per line)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(float.fromhex(line))
    return np.array(vals, dtype=np.float64)
