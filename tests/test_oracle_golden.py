"""The oracle against its stored regression fixture, written by
tests/golden/make_fixtures.py from the oracle itself: the paper prints no
solution values (its figures are plots, its one table wall-clock times)."""
import json
import os

import numpy as np

import oracle
from paper_1211_0540_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_n8_collide.json")


def load_golden():
    with open(GOLDEN) as fh:
        d = json.load(fh)
    seed = int(d["input"].split("seed=")[1].rstrip(")"))
    f = inputs.homogeneous_cells(d["N"], d["L"], 1, seed=seed)
    Q = np.array([float(x) for x in d["Q"]])
    return d, f, Q


def test_oracle_reproduces_fixture():
    d, f, Qref = load_golden()
    Q = oracle.collide(d["N"], d["L"], d["lambda"], f)[0]
    # summation order may differ between machines (FMA contraction): not bit-exact
    assert np.abs(Q - Qref).max() <= 1e-12 * np.abs(Qref).max()
    m = oracle.moments(d["N"], d["L"], Qref[None])[0]
    assert np.abs(m).max() <= 1e-12 * np.abs(Qref).sum() * (2 * d["L"] / d["N"]) ** 3 * d["L"] ** 2
