"""Triclinic cells on the GPU against the oracle (GPU only).

Neighbour lists bit-exact in every precision (the image shift n H is summed in the same fixed
order on both sides); energies, forces and virials within each precision's bars; a sheared
trajectory; and the cube's lattice given in a skewed basis, which must reproduce the cubic
result."""
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


def _rotated(x, H, seed=11):
    R = synth._rand_rotation(np.random.default_rng(seed))
    return x @ R.T, (H.reshape(3, 3) @ R.T).ravel()


def _case(name):
    if name == "water8":      # a 6.2 A cell: several images of one j within r_c
        s = synth.water_box(8, 3)
        x, H = _sheared(s)
        return s, x, H, synth.xavier_weights(("O", "H"), 6.0, 0.5, (200, 400), 1001)
    if name == "water64":
        s = synth.water_box(64, 0)
        x, H = _sheared(s, ((0.45, 0.0), (-0.3, 0.35)))
        return s, x, H, synth.water_weights()
    if name == "water64_rot":  # a general cell: no row along an axis
        s = synth.water_box(64, 0)
        x, H = _rotated(*_sheared(s))
        return s, x, H, synth.water_weights()
    s = synth.copper_fcc(3, 0)
    x, H = _sheared(s, ((0.2, 0.0), (0.1, -0.15)))
    return s, x, H, synth.copper_weights()


def _cuda(x, types):
    return (torch.tensor(x, dtype=torch.float64, device="cuda"),
            torch.tensor(types, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
@pytest.mark.parametrize("name", ["water8", "water64", "water64_rot", "cu3"])
def test_triclinic_nlist_bit_exact(dp, prec, name):
    s, x, H, w = _case(name)
    ref_nl, ref_im, _, ovf = oracle.Model(w.to_blob()).nlist(x, s.types, H, "brute")
    assert not ovf
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    xc, t = _cuda(x, s.types)
    m.compute(xc, t, H)
    nl, im = m.get_nlist()
    nl, im = nl.cpu().numpy(), im.cpu().numpy()
    np.testing.assert_array_equal(nl, ref_nl)
    np.testing.assert_array_equal(np.where(ref_nl >= 0, im, 0), np.where(ref_nl >= 0, ref_im, 0))
    m.close()


# the normalised water model (per-atom energies spread by ~0.1 eV, forces ~0.5 eV/A) and the
# bars of its cubic parity test
BARS = {"fp64": {"f_rel": 1e-9, "dev_rel": 1e-9}, "fp32": {"f_rel": 1e-4, "dev_rel": 1e-3},
        "mix_fp16": {"f_rel": 3e-3, "dev_rel": 1e-2}}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
@pytest.mark.parametrize("name", ["water64", "water64_rot"])
def test_triclinic_energy_forces_virial(dp, prec, name):
    s, x, H, _ = _case(name)
    w = synth.normalised_weights("water", env_stats())
    ref = oracle.Model(w.to_blob()).compute(x, s.types, H)
    assert np.sqrt((ref["forces"] ** 2).mean()) > 0.3
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    xc, t = _cuda(x, s.types)
    out = m.compute(xc, t, H)
    e = errors(out, ref, s.types)
    assert e["f_rel"] <= BARS[prec]["f_rel"], e
    assert e["dev_rel"] <= BARS[prec]["dev_rel"], e
    V = out["virial"].cpu().numpy().reshape(3, 3)
    np.testing.assert_allclose(V, ref["virial"], rtol=0,
                               atol=max(3 * BARS[prec]["f_rel"], 1e-12) * np.abs(ref["virial"]).max())
    if prec == "fp64":
        assert e["ei_rel"] <= 1e-10, e
    m.close()


def test_cube_lattice_in_a_skewed_basis(dp):
    s = synth.water_box(64, 0)
    L = s.box[0]
    H = np.array([[L, 0, 0], [L, L, 0], [0, L, L]], dtype=np.float64).ravel()
    w = synth.water_weights()
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    xc, t = _cuda(s.coords, s.types)
    cube = m.compute(xc, t, s.box)
    e_cube, f_cube = cube["energy"].item(), cube["forces"].cpu().numpy()
    skew = m.compute(xc, t, H)
    assert skew["energy"].item() == pytest.approx(e_cube, rel=1e-12)
    np.testing.assert_allclose(skew["forces"].cpu().numpy(), f_cube, rtol=0, atol=1e-11)
    m.close()


def test_triclinic_md_matches_oracle(dp):
    s, x, H, w = _case("water64")
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    ref = oracle.Model(w.to_blob()).md(x, v0, s.types, H, s.masses(), 0.5, 20, rebuild_every=10)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    xc = torch.tensor(x, device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(s.types, device="cuda")
    st = m.md_state(xc, v, t, H, s.masses(), rebuild_every=10)
    out = m.verlet(st, 0.5, 20, capture_graph=True)
    np.testing.assert_allclose(xc.cpu().numpy(), ref["x"], atol=1e-10)
    np.testing.assert_allclose(v.cpu().numpy(), ref["v"], atol=1e-10)
    assert out["potential"].item() == pytest.approx(ref["pe"][-1], rel=1e-10)
    m.close()


def test_batch_mixes_cubic_and_triclinic_replicas(dp):
    a = synth.water_box(32, 1)
    b = synth.water_box(64, 0)
    xb, Hb = _sheared(b)
    w = synth.water_weights()
    orc = oracle.Model(w.to_blob())
    refs = [orc.compute(a.coords, a.types, a.box), orc.compute(xb, b.types, Hb)]
    coords = np.concatenate([a.coords, xb])
    types = np.concatenate([a.types, b.types]).astype(np.int32)
    offs = np.array([0, a.natoms, a.natoms + b.natoms], dtype=np.int32)
    boxes = np.stack([a.box, Hb])
    m = dp.DPModel(w, "fp64", max_atoms=len(types), max_replicas=2)
    xc, t = _cuda(coords, types)
    out = m.compute_batch(xc, t, offs, boxes)
    E = out["energy"].cpu().numpy()
    F = out["forces"].cpu().numpy()
    for r, ref in enumerate(refs):
        assert E[r] == pytest.approx(ref["energy"], rel=1e-12)
        np.testing.assert_allclose(F[offs[r]:offs[r + 1]], ref["forces"], rtol=0, atol=1e-10)
    m.close()


def test_left_handed_cell_is_an_argument_error(dp):
    s = synth.water_box(8, 3)
    L = s.box[0]
    m = dp.DPModel(synth.water_weights(), "fp64", max_atoms=s.natoms)
    xc, t = _cuda(s.coords, s.types)
    with pytest.raises(dp.DPError) as e:
        m.compute(xc, t, np.diag([L, L, -L]).ravel())
    assert e.value.status == 1
    m.close()
