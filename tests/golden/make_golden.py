"""Writes the stored fixtures of tests/golden/ using only the CPU oracle.

edt_departure_170.json -- a small binary image on which the wavefront
distance transform (Algorithm 3) assigns squared distance 170 to a pixel
whose exact squared distance is 169, the departure illustrated in Figure 3
(Section 2.2).  Found by a seeded search over sparse random feature sets.

recon_small.json -- small reconstruction inputs with their Algorithm 2
results (uint8, 4- and 8-connected) for regression of the oracle and as
fixed vectors for the GPU tests.

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def find_departure_170(seed=0, side=32, tries=200000):
    rng = np.random.default_rng(seed)
    for _ in range(tries):
        b = np.ones((side, side), np.uint8)
        k = int(rng.integers(2, 6))
        ys = rng.integers(0, side, k)
        xs = rng.integers(0, side, k)
        b[ys, xs] = 0
        sq, _ = oracle.edt(b)
        ex = oracle.edt_exact(b)
        hit = np.argwhere((ex == 169) & (sq == 170))
        if len(hit):
            y, x = hit[0]
            return b, (int(y), int(x))
    raise RuntimeError("no departure found")


def main():
    b, (y, x) = find_departure_170()
    with open(os.path.join(HERE, "edt_departure_170.json"), "w") as f:
        json.dump({
            "source": "Section 2.2, Figure 3: propagation gives sqrt(170) where the exact distance is 13",
            "note": "features are the 0-valued pixels; found by tests/golden/make_golden.py",
            "binary": b.tolist(), "pixel": [y, x], "alg3_sqdist": 170, "exact_sqdist": 169,
        }, f)
    rng = np.random.default_rng(1234)
    cases = []
    for (h, w, levels) in ((7, 9, 8), (16, 16, 256), (13, 21, 256), (1, 17, 256), (19, 1, 256)):
        I = rng.integers(0, levels, (h, w)).astype(np.uint8)
        J = np.minimum(I, rng.integers(0, levels, (h, w)).astype(np.uint8))
        cases.append({"mask": I.tolist(), "marker": J.tolist(),
                      "out8": oracle.fh(J, I, 8).tolist(), "out4": oracle.fh(J, I, 4).tolist()})
    with open(os.path.join(HERE, "recon_small.json"), "w") as f:
        json.dump({"source": "Algorithm 2 (Section 2.1) results from the CPU oracle", "cases": cases}, f)


if __name__ == "__main__":
    main()
