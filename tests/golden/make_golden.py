"""Writes tests/golden/rational_amplitudes.json: exact rational amplitudes
A = eps_n . R_top of a few seeded rational points, computed ONLY by the
oracle (oracle.bg_oracle over fractions.Fraction).  The paper prints no
worked numerical example, so these fixtures are regression anchors whose
correctness rests on the oracle's pins (tests/test_oracle_pins.py).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bg_oracle as O                       # noqa: E402
from paper_2502_07060_gb300 import inputs as G         # noqa: E402

CASES = [(4, 4, 4, 0), (5, 4, 4, 0), (5, 4, 6, 0), (6, 6, 6, 0), (6, 4, 4, 1), (7, 6, 8, 1),
         (8, 6, 6, 0)]


def main():
    out = []
    for idx, (n, d, Ds, metric) in enumerate(CASES):
        rng = np.random.Generator(np.random.Philox(4242 + idx))
        k, eps = G.rational_point(rng, n, d, Ds, metric, lo=-5, hi=6)
        a, st = O.amplitude(k, eps, metric)
        assert st == O.OK
        out.append({
            "n": n, "d": d, "Ds": Ds, "metric": metric,
            "k": [[str(x) for x in v] for v in k],
            "eps": [[str(x) for x in v] for v in eps],
            "amplitude": str(a),
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rational_amplitudes.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.bg_oracle over Fraction (tests/golden/make_golden.py)",
                   "cases": out}, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
