"""The stored dense-pole hulls of the 64^2 square array (read by the benchmark's
64^2 lattice workload) are what the oracle computes, and the exact forward-difference
hull is a clean interval, about [0.172, 5.82]."""
import json
import os

import numpy as np

from oracle import exact as X
from synth import square_array_mask

HERE = os.path.dirname(os.path.abspath(__file__))


def test_dense_pole_hull_fixture_matches_oracle():
    data = json.load(open(os.path.join(HERE, "golden", "dense_pole_hulls_64.json")))["hulls"]
    mask = square_array_mask(64)
    e = np.array([1.0, 0.0])
    for green in ("trig", "fd"):
        m, w = X.poles(mask, e, green)
        for cutoff in (1e-10, 1e-3):
            a, b, _, _ = X.pole_hull(m, w, cutoff)
            ref = data[f"{green}|{cutoff:g}"]
            assert abs(a - ref["alpha"]) <= 1e-9 * abs(a) and abs(b - ref["beta"]) <= 1e-9 * abs(b)
    fd = data["fd|1e-10"]
    assert 0.17 < fd["alpha"] < 0.18 and 5.8 < fd["beta"] < 5.9
