"""The optional features together, against the oracle (GPU only): the tabulated embedding and
the per-atom virial in a triclinic cell, the RDF of a sheared box, and nearest-first truncation
in a batch that mixes a cubic and a triclinic replica."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

from _parity import env_stats, errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


def _sheared(s, tilt=((0.3, 0.0), (-0.2, 0.25))):
    L = s.box[0]
    H = L * np.array([[1.0, 0.0, 0.0], [tilt[0][0], 1.0, 0.0], [tilt[1][0], tilt[1][1], 1.0]])
    return (s.coords / L) @ H, H.ravel()


def _cuda(x, t):
    return torch.tensor(x, dtype=torch.float64, device="cuda"), torch.tensor(t, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_tabulated_triclinic(dp, prec):
    s = synth.water_box(64, 2)
    x, H = _sheared(s)
    w = synth.normalised_weights("water", env_stats())
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x0, x1, n = m.tabulate(256)
    orc = oracle.Model(w.to_blob())
    orc.tabulate(x0, x1, n)
    ref = orc.compute(x, s.types, H)
    out = m.compute(*_cuda(x, s.types), H)
    e = errors(out, ref, s.types)
    if prec == "fp64":
        assert e["ei_rel"] <= 1e-10 and e["f_rel"] <= 1e-9, e
    else:
        assert e["f_rel"] <= 3e-3 and e["dev_rel"] <= 1e-2, e
    m.close()


def test_atom_virial_and_rdf_triclinic(dp):
    s = synth.water_box(256, 4)
    x, H = _sheared(s, ((0.25, 0.0), (0.15, -0.2)))
    w = synth.normalised_weights("water", env_stats())
    orc = oracle.Model(w.to_blob())
    ref = orc.compute(x, s.types, H, atom_virial=True)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    out = m.compute(*_cuda(x, s.types), H)
    W = m.atom_virial().cpu().numpy()
    Wr = ref["atom_virial"]
    assert np.sqrt(((W - Wr) ** 2).mean()) <= 1e-9 * np.sqrt((Wr ** 2).mean())
    np.testing.assert_allclose(W.sum(0), out["virial"].cpu().numpy(), rtol=1e-10, atol=1e-12)
    nbins, rmax = 200, 6.0
    c = m.rdf(nbins, rmax).astype(np.int64)
    cr = orc.rdf(x, s.types, H, nbins, rmax).astype(np.int64)
    np.testing.assert_array_equal(c, cr)
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_truncation_in_a_mixed_batch(dp, prec):
    # sel (20, 40) truncates every atom; one cubic and one sheared replica in one batch
    w = synth.xavier_weights(("O", "H"), 6.0, 0.5, (20, 40), 1001)
    a = synth.water_box(32, 1)
    b = synth.water_box(64, 0)
    xb, Hb = _sheared(b)
    orc = oracle.Model(w.to_blob())
    orc.set_truncation(True)
    refs = [orc.compute(a.coords, a.types, a.box), orc.compute(xb, b.types, Hb)]
    coords = np.concatenate([a.coords, xb])
    types = np.concatenate([a.types, b.types]).astype(np.int32)
    offs = np.array([0, a.natoms, a.natoms + b.natoms], dtype=np.int32)
    m = dp.DPModel(w, prec, max_atoms=len(types), max_replicas=2, skin=0.5)
    m.set_truncation(True)
    out = m.compute_batch(*_cuda(coords, types), offs, np.stack([a.box, Hb]))
    E = out["energy"].cpu().numpy()
    F = out["forces"].cpu().numpy()
    for r, ref in enumerate(refs):
        Fr = ref["forces"]
        f_rel = np.sqrt(((F[offs[r]:offs[r + 1]] - Fr) ** 2).mean()) / np.sqrt((Fr ** 2).mean())
        if prec == "fp64":
            assert E[r] == pytest.approx(ref["energy"], rel=1e-12)
            assert f_rel <= 1e-10, f_rel
        else:
            assert abs(E[r] - ref["energy"]) / (offs[r + 1] - offs[r]) <= 1e-4
            assert f_rel <= 1e-2, f_rel
    m.close()
