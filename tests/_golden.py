"""Reader for the hand-derived fixtures under tests/golden/ (key followed by numbers)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            arr = np.array([float(v) for v in vals])
            out[key] = arr if len(arr) > 1 else arr[0]
    return out
