"""Nearest-first sel truncation on the GPU against the oracle's (GPU only).

Every centre of these systems has more neighbours of some type within r_c than sel allows,
so its formatted segments go through the selection.  The neighbour lists must agree bit for
bit (the ranking uses the FP64 r^2 in every precision); energies and forces within the bars
of each precision.  The Verlet list still holds 1.3 sel ((r_c + skin) / r_c)^3 entries per type,
so these far-truncated models run with a skin of 0.5 A (every pair within r_c + skin fits)."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

from _parity import errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


def _system(case):
    if case == "water64":  # about 30 O and 60 H neighbours within 6 A against sel (20, 40)
        return synth.water_box(64, 0), synth.xavier_weights(("O", "H"), 6.0, 0.5, (20, 40), 1001)
    if case == "water8":  # a 6.2 A box: several periodic images of one j compete
        return synth.water_box(8, 3), synth.xavier_weights(("O", "H"), 6.0, 0.5, (20, 40), 1001)
    # a perfect FCC lattice: the cut at 40 falls inside the third shell (18 + 24 neighbours), so
    # equal distances are ranked by (j, image)
    return synth.copper_fcc(2, 0, sigma=0.0), synth.xavier_weights(("Cu",), 6.0, 2.0, (40,), 1001)


SKIN = 0.5


def _oracle(w):
    m = oracle.Model(w.to_blob())
    m.set_truncation(True)
    return m


def _cuda(s):
    return (torch.tensor(s.coords, dtype=torch.float64, device="cuda"),
            torch.tensor(s.types, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
@pytest.mark.parametrize("case", ["water64", "water8", "cu_perfect"])
def test_truncated_nlist_bit_exact(dp, prec, case):
    s, w = _system(case)
    ref_nl, ref_im, cnt, ovf = _oracle(w).nlist(s.coords, s.types, s.box, "brute")
    assert not ovf
    full = oracle.Model(w.to_blob()).nlist(s.coords, s.types, s.box, "brute", sel=[10 ** 4] * len(w.sel))[2]
    assert (full.max(0) > np.array(w.sel)).all()  # the selection is exercised for every type
    m = dp.DPModel(w, prec, max_atoms=s.natoms, skin=SKIN)
    m.set_truncation(True)
    x, t = _cuda(s)
    m.compute(x, t, s.box)
    nl, im = m.get_nlist()
    nl, im = nl.cpu().numpy(), im.cpu().numpy()
    np.testing.assert_array_equal(nl, ref_nl)
    np.testing.assert_array_equal(np.where(ref_nl >= 0, im, 0), np.where(ref_nl >= 0, ref_im, 0))
    m.close()


def test_overflow_without_truncation_is_an_error(dp):
    s, w = _system("water64")
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms, skin=SKIN)
    x, t = _cuda(s)
    with pytest.raises(dp.DPError) as e:
        m.compute(x, t, s.box)
    assert e.value.status == 5
    m.close()


# fp64: per-atom energies and forces to 1e-10 relative; fp32 and mixed: the parity bars of the
# untruncated model
BARS = {"fp64": {"f_rel": 1e-10, "dev_rel": 1e-9}, "fp32": {"f_rel": 1e-4, "dev_rel": 1e-3},
        "mix_fp16": {"f_rel": 1e-2, "dev_rel": 0.3}}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
def test_truncated_energy_and_forces(dp, prec):
    s, w = _system("water64")
    ref = _oracle(w).compute(s.coords, s.types, s.box)
    m = dp.DPModel(w, prec, max_atoms=s.natoms, skin=SKIN)
    m.set_truncation(True)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    e = errors(out, ref, s.types)
    assert e["f_rel"] <= BARS[prec]["f_rel"], e
    assert e["dev_rel"] <= BARS[prec]["dev_rel"], e
    if prec == "fp64":
        assert e["ei_rel"] <= 1e-10, e
    m.close()


def test_truncated_md_matches_oracle(dp):
    # the per-step filter re-ranks the Verlet entries with the moved positions on both sides
    s, w = _system("water64")
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    ref = _oracle(w).md(s.coords, v0, s.types, s.box, s.masses(), 0.5, 20, rebuild_every=10, skin=SKIN)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms, skin=SKIN)
    m.set_truncation(True)
    x = torch.tensor(s.coords, device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(s.types, device="cuda")
    st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=10)
    out = m.verlet(st, 0.5, 20, capture_graph=True)
    np.testing.assert_allclose(x.cpu().numpy(), ref["x"], atol=1e-10)
    np.testing.assert_allclose(v.cpu().numpy(), ref["v"], atol=1e-10)
    assert out["potential"].item() == pytest.approx(ref["pe"][-1], rel=1e-10)
    m.close()
