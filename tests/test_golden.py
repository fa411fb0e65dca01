"""The oracle against its stored regression fixtures (tests/golden/)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_stored_fixtures():
    stored = {}
    for line in open(os.path.join(HERE, "golden", "oracle_fbp_8cube.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        stored[name] = np.array([float(v) for v in vals])
    now = make_golden.compute()
    assert set(now) == set(stored)
    for k, v in now.items():
        v = np.asarray(v, dtype=np.float64)
        # FP64 with OpenMP reductions: agreement to ~1e-13 of the data scale
        scale = np.abs(stored[k]).max()
        assert np.allclose(v, stored[k], rtol=0, atol=1e-11 * scale), k
