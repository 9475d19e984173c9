"""Write dense_pole_hulls_64.json: the pole interval [alpha, beta] of the 64 x 64
square array of squares (f = 1/4, e = (1, 0)) from the FP64 oracle's dense
eigen-decomposition of chi Gamma_1 chi (section "Estimating the parameters alpha
and beta"; the poles of sigma_*(sigma_1) are 1 - 1/m_n with weights
|u_n^H chi e|^2), for both Green symbols and the weight cutoffs 1e-10 (the
numerically exact hull) and 1e-3 (an estimate).  Calls only the oracle:

    python tests/golden/make_dense_pole_hulls.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact as X  # noqa: E402
from synth import square_array_mask  # noqa: E402


def main():
    mask = square_array_mask(64)
    e = np.array([1.0, 0.0])
    out = {"workload": "64x64 square array of squares (f = 1/4), e = (1, 0)",
           "method": "oracle.exact.poles (dense eigen-decomposition of chi Gamma_1 chi) and oracle.exact.pole_hull",
           "hulls": {}}
    for green in ("trig", "fd"):
        m, w = X.poles(mask, e, green)
        for cutoff in (1e-10, 1e-3):
            a, b, mmin, mmax = X.pole_hull(m, w, cutoff)
            out["hulls"][f"{green}|{cutoff:g}"] = {"alpha": a, "beta": b, "m_min": mmin, "m_max": mmax,
                                                   "weighted_poles": int(np.sum(w > cutoff * np.sum(w)))}
    with open(os.path.join(HERE, "dense_pole_hulls_64.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
