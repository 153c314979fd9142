"""Writes the regression fixtures of this directory from the FP64 oracle.

Run from the repository root: python tests/golden/make_fixtures.py
Only oracle/ and the seeded input generators are used."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1211_0540_gb300 import inputs  # noqa: E402

N, L, LAM, SEED = 8, 6.0, 1.0, 2024


def main():
    f = inputs.homogeneous_cells(N, L, 1, seed=SEED)
    Q = oracle.collide(N, L, LAM, f)
    Qm = oracle.collide(N, L, LAM, f, part=1, project=False)
    out = {
        "what": "projected collision operator Q = P_N Qt(f) (Sec. 3.2-3.3) of one cell, FP64 oracle",
        "N": N, "L": L, "lambda": LAM,
        "input": "paper_1211_0540_gb300.inputs.homogeneous_cells(N, L, 1, seed=%d)" % SEED,
        "Q": [repr(float(x)) for x in Q[0]],
        "loss_norm": repr(float(np.linalg.norm(Qm[0]))),
        "moments": [repr(float(x)) for x in oracle.moments(N, L, Q)[0]],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_n8_collide.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")


if __name__ == "__main__":
    main()
