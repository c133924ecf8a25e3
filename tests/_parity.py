"""Error measures of a GPU result against the FP64 oracle, shared by the GPU parity tests.

Absolute bars alone can be larger than the whole signal of an untrained model, so every
comparison also reports measures relative to the signal:
  f_rel   force RMSE / force RMS of the oracle;
  dev_rel RMS error of the per-atom energy deviations E_i - <E>_type (the oracle's per-type
          mean is subtracted from both sides) over the RMS of those deviations.  A result
          with D = 0 or with the atom-to-atom variation lost scores about 1.
"""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def env_stats():
    with open(os.path.join(HERE, "golden", "env_stats.json")) as f:
        return json.load(f)


def errors(out, ref, types, sel=None):
    """out: GPU result (torch tensors), ref: oracle result (numpy); sel: boolean mask of the
    atoms compared (all if None)."""
    F = out["forces"].cpu().numpy()
    Ei = out["atom_energy"].cpu().numpy()
    Fr, Er = ref["forces"], ref["atom_energy"]
    t = np.asarray(types)
    if sel is not None:
        F, Ei, Fr, Er, t = F[sel], Ei[sel], Fr[sel], Er[sel], t[sel]
    rmse = float(np.sqrt(((F - Fr) ** 2).mean()))
    rms = float(np.sqrt((Fr ** 2).mean()))
    dg, dr = Ei.copy(), Er.copy()
    for ty in np.unique(t):
        mu = Er[t == ty].mean()
        dg[t == ty] -= mu
        dr[t == ty] -= mu
    spread = float(np.sqrt((dr ** 2).mean()))
    return {"f_rmse": rmse, "f_rms": rms, "f_rel": rmse / rms if rms > 0 else float("inf"),
            "e_atom": float(abs(Ei.sum() - Er.sum()) / len(Ei)),
            "ei_max": float(np.abs(Ei - Er).max()),
            "ei_rel": float((np.abs(Ei - Er) / np.maximum(np.abs(Er), np.abs(Er).mean())).max()),
            "spread": spread,
            "dev_rel": float(np.sqrt(((dg - dr) ** 2).mean())) / spread if spread > 0 else float("inf")}


def copper_subbox_masks(s, a, rcut):
    """Atoms of FCC cells [0,10)^3 (by lattice site) and all centres within r_c of them."""
    L = s.box[0]
    site = np.rint(s.coords / (a / 2)).astype(int)  # half-lattice index of the nearest site
    sub = np.all((site >= 0) & (site < 20), axis=1)
    assert sub.sum() == 4000
    lo, hi = -rcut - 0.5, 10 * a + rcut + 0.5
    w = s.coords.copy()
    w = w - L * np.floor(w / L)
    w[w > L - rcut - 1.0] -= L
    centre = np.all((w > lo) & (w < hi), axis=1)
    return sub, centre
