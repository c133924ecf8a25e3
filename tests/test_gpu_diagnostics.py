"""Per-atom virial and the pair-distance histogram (RDF) on the GPU against the oracle (GPU only)."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

from _parity import env_stats

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-4), ("mix_fp16", 1e-2), ("mix_bf16", 3e-2)])
def test_atom_virial_matches_oracle(dp, prec, tol):
    s = synth.water_box(64, 3)
    w = synth.normalised_weights("water", env_stats())
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box, atom_virial=True)
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    out = m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    W = m.atom_virial().cpu().numpy()
    Wr = ref["atom_virial"]
    rel = np.sqrt(((W - Wr) ** 2).mean()) / np.sqrt((Wr ** 2).mean())
    assert rel <= tol, rel
    # the per-atom virials sum to the box virial of the same evaluation
    np.testing.assert_allclose(W.sum(0), out["virial"].cpu().numpy(), rtol=1e-6 if prec != "fp64" else 1e-10,
                               atol=1e-6 * np.abs(Wr.sum(0)).max())
    # the mixed pass leaves the forces of the evaluation as they were
    F0 = out["forces"].clone()
    m.atom_virial()
    assert torch.equal(out["forces"], F0)
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_rdf_matches_oracle(dp, prec):
    s = synth.water_box(256, 4)
    w = synth.water_weights()
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    nbins, rmax = 240, 6.0
    c = m.rdf(nbins, rmax).astype(np.int64)
    ref = oracle.Model(w.to_blob()).rdf(s.coords, s.types, s.box, nbins, rmax).astype(np.int64)
    assert c.sum() == ref.sum()  # the same pairs within r_max
    moved = np.abs(c - ref).sum() // 2  # pairs that land in a neighbouring bin by rounding
    assert moved <= (0 if prec == "fp64" else 1e-4 * ref.sum() + 2), moved
    # g(r) of the O-O pairs peaks near the hydrogen-bond distance
    import paper_2410_22867_gb300 as dpm
    nat = [int((s.types == t).sum()) for t in range(2)]
    r, g = dpm.rdf_g(c, nat, s.box[0] ** 3, rmax)
    assert 2.3 < r[np.argmax(g[0, 0])] < 3.6
    m.close()
