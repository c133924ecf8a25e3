"""Writes tests/golden/env_stats.json: the per-type input normalisation (davg, dstd)
of the smooth descriptor for the water and copper systems, from the FP64 oracle only.

Section II-A's environment matrix is normalised per centre type before it enters the
embedding net.  The statistics are those of one seeded configuration of each system,
taken over every neighbour slot of every atom of the centre type (S slots per atom;
a padded slot counts as the zero row):
    davg = (mean of s, 0, 0, 0)
    dstd = (std of s, rms of the three angular components, same, same)
with 1e-2 as the smallest dstd.  The angular components have mean zero by symmetry,
so only s is shifted.

Run:  python tests/golden/make_env_stats.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2410_22867_gb300 import synth  # noqa: E402

SOURCES = {
    "water": ("water_box(1024, seed 3): 1024 H2O, 3,072 atoms", lambda: synth.water_box(1024, 3),
              synth.water_weights),
    "copper": ("copper_fcc(10, seed 0): 4,000 atoms", lambda: synth.copper_fcc(10, 0), synth.copper_weights),
}
DSTD_FLOOR = 1e-2


def stats(kind):
    desc, make_sys, make_w = SOURCES[kind]
    s, w = make_sys(), make_w(1001)
    sums = oracle.Model(w.to_blob()).env_stats(s.coords, s.types, s.box)
    davg, dstd = [], []
    for t in range(w.ntypes):
        n, s1, s2, a2 = sums[t, 0], sums[t, 1], sums[t, 2], sums[t, 3]
        mean = s1 / n
        sr = math.sqrt(max(s2 / n - mean * mean, 0.0))
        sa = math.sqrt(a2 / (3.0 * n))
        davg.append([mean, 0.0, 0.0, 0.0])
        dstd.append([max(sr, DSTD_FLOOR)] + [max(sa, DSTD_FLOOR)] * 3)
    return {"source": desc, "type_names": list(w.type_names), "davg": davg, "dstd": dstd,
            "sums": sums.tolist()}


if __name__ == "__main__":
    out = {"_doc": "per centre type: davg[t][4], dstd[t][4]; sums[t] = [slots, sum s, sum s^2, "
                   "sum of squared angular components, atoms]; written by make_env_stats.py from the oracle"}
    for k in SOURCES:
        out[k] = stats(k)
    with open(os.path.join(HERE, "env_stats.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
