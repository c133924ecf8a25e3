"""Writes tests/golden/*.txt from the FP64 oracle only (never from the CUDA path).

The paper prints no worked example, so these files are regression fixtures of the
oracle itself: they pin it against accidental change once the independent checks
(closed forms, finite differences, invariances) have passed.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2410_22867_gb300 import synth  # noqa: E402


def water64():
    w = synth.water_weights(1001)
    s = synth.water_box(64, 0)
    r = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box, method="brute")
    lines = ["# 64 H2O (192 atoms), L = %.12f A, water_box(64, seed 0), water_weights(seed 1001)" % s.box[0],
             "# brute-force neighbour list; FP64 oracle; units eV, eV/A",
             "energy %.17e" % r["energy"]]
    for i in range(0, 192, 17):
        lines.append("atom_energy %d %.17e" % (i, r["atom_energy"][i]))
        lines.append("force %d %.17e %.17e %.17e" % ((i,) + tuple(r["forces"][i])))
    lines.append("virial " + " ".join("%.17e" % v for v in r["virial"].ravel()))
    with open(os.path.join(HERE, "water64_oracle.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    water64()
