"""CUDA path against the FP64 oracle on the same seeded inputs (GPU only).

Bars: neighbour list bit-exact; FP64 per-atom energy within 1e-10 relative;
FP32 force RMSE <= 1e-5 eV/A; every error is stated against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

from _parity import copper_subbox_masks, errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


def _cuda(s):
    return (torch.tensor(s.coords, dtype=torch.float64, device="cuda"),
            torch.tensor(s.types, dtype=torch.int32, device="cuda"))


def _nl_rows_equal(gpu_nl, gpu_im, ref_nl, ref_im):
    np.testing.assert_array_equal(gpu_nl, ref_nl)
    np.testing.assert_array_equal(np.where(ref_nl >= 0, gpu_im, 0), np.where(ref_nl >= 0, ref_im, 0))


# ------------------------------------------------------------------ neighbour list
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["water64", "water8", "water32", "water4096", "cu3"])
def test_nlist_bit_exact(dp, prec, case):
    if case.startswith("water"):
        s = synth.water_box(int(case[5:]), 0)
        w = synth.water_weights()
        method = "brute" if s.natoms <= 200 else "cell"
    else:
        s = synth.copper_fcc(int(case[2:]), 0)
        w = synth.copper_weights()
        method = "brute"
    if case == "water8":
        # 8 molecules: a 6.2 A box, several periodic images of every atom are in reach
        w = synth.xavier_weights(("O", "H"), 6.0, 0.5, (200, 400), 1001)
    ref_nl, ref_im, _, ovf = oracle.Model(w.to_blob()).nlist(s.coords, s.types, s.box, method)
    assert not ovf
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x, t = _cuda(s)
    m.compute(x, t, s.box)
    nl, im = m.get_nlist()
    _nl_rows_equal(nl.cpu().numpy(), im.cpu().numpy(), ref_nl, ref_im)


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_nlist_bit_exact_sparse_box(dp, prec):
    # A 108-atom copper cluster in a 70 A box, straddling the periodic corner.  A single
    # evaluation sizes its cells by r_c: half-size cells would need 17^3 = 4913 cells, more than
    # the cell list holds for 108 atoms (1196), so the library falls back to cells of edge >= r_c
    # (8^3).
    c = synth.copper_fcc(3, 5)
    L = 70.0
    coords = np.mod(c.coords - 4.0, L)
    s = synth.System(coords, c.types, np.array([L, 0, 0, 0, L, 0, 0, 0, L], dtype=np.float64), c.type_names)
    w = synth.copper_weights()
    ref_nl, ref_im, _, ovf = oracle.Model(w.to_blob()).nlist(s.coords, s.types, s.box, "brute")
    assert not ovf
    assert (ref_nl >= 0).sum() > 50 * s.natoms  # a dense cluster: most pairs are real neighbours
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x, t = _cuda(s)
    m.compute(x, t, s.box)
    nl, im = m.get_nlist()
    _nl_rows_equal(nl.cpu().numpy(), im.cpu().numpy(), ref_nl, ref_im)
    m.close()


def _stencil_candidates(coords, L, nc, m):
    """Atoms in the (2m+1)^3 periodic stencil of every non-empty cell of an nc^3 grid."""
    idx = np.minimum((np.mod(coords, L) / (L / nc)).astype(int), nc - 1)
    cnt = np.zeros((nc, nc, nc), dtype=np.int64)
    np.add.at(cnt, (idx[:, 0], idx[:, 1], idx[:, 2]), 1)
    tot = np.zeros_like(cnt)
    for o in np.ndindex(2 * m + 1, 2 * m + 1, 2 * m + 1):
        tot += np.roll(cnt, shift=tuple(m - np.array(o)), axis=(0, 1, 2))
    return tot[cnt > 0]


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_nlist_bit_exact_dense_cluster(dp, prec):
    # A compressed 4,000-atom FCC cluster (a = 2.4 A) in a 42 A box, r_c 6 + skin 2.  The r_c + skin
    # list an MD run starts from uses 10^3 cells (edge 4.2 A, 5^3 stencil): those inside the
    # cluster see more candidates than one CTA of the cell-staged Verlet build holds, those at its
    # surface fewer, so both Verlet kernels write parts of that list.  The r_c list of a single
    # evaluation (cells of edge >= r_c / 2) is checked as well.
    c = synth.copper_fcc(10, 7, a=2.4, sigma=0.05)
    L = 42.0
    s = synth.System(c.coords + 9.0, c.types, np.array([L, 0, 0, 0, L, 0, 0, 0, L], dtype=np.float64), c.type_names)
    cand = _stencil_candidates(s.coords, L, 10, 2)
    assert cand.max() > 2048 and cand.min() <= 2048
    w = synth.xavier_weights(("Cu",), 6.0, 0.5, (320,), 1001)
    ref_nl, ref_im, _, ovf = oracle.Model(w.to_blob()).nlist(s.coords, s.types, s.box, "cell")
    assert not ovf
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x, t = _cuda(s)
    m.compute(x, t, s.box)
    nl, im = m.get_nlist()
    _nl_rows_equal(nl.cpu().numpy(), im.cpu().numpy(), ref_nl, ref_im)
    st = m.md_state(x.clone(), torch.zeros_like(x), t, s.box, s.masses(), rebuild_every=10)
    m.verlet(st, 0.5, 0, capture_graph=False)
    nl, im = m.get_nlist()
    _nl_rows_equal(nl.cpu().numpy(), im.cpu().numpy(), ref_nl, ref_im)
    m.close()


def test_nlist_bit_exact_copper_full(dp):
    s = synth.copper_fcc(32, 0)
    w = synth.copper_weights()
    ref_nl, ref_im, _, ovf = oracle.Model(w.to_blob()).nlist(s.coords, s.types, s.box, "cell")
    m = dp.DPModel(w, "fp32", max_atoms=s.natoms)
    x, t = _cuda(s)
    m.compute(x, t, s.box)
    nl, im = m.get_nlist()
    _nl_rows_equal(nl.cpu().numpy(), im.cpu().numpy(), ref_nl, ref_im)


# ------------------------------------------------------------------ energies / forces
def _rel_energy_err(Ei, ref):
    scale = np.maximum(np.abs(ref), np.abs(ref).mean())
    return np.abs(Ei - ref) / scale


@pytest.mark.parametrize("n_mol,seed", [(64, 0), (1024, 3), (37, 9)])
def test_fp64_matches_oracle(dp, n_mol, seed):
    s = synth.water_box(n_mol, seed)
    w = synth.water_weights()
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    Ei = out["atom_energy"].cpu().numpy()
    assert _rel_energy_err(Ei, ref["atom_energy"]).max() <= 1e-10
    assert out["energy"].item() == pytest.approx(ref["energy"], rel=1e-12)
    F = out["forces"].cpu().numpy()
    Fs = np.abs(ref["forces"]).max()
    assert np.abs(F - ref["forces"]).max() <= 1e-9 * Fs
    np.testing.assert_allclose(out["virial"].cpu().numpy(), ref["virial"], rtol=1e-9, atol=1e-12 * Fs)


def test_fp64_energy_over_reduction_chunks(dp):
    # 12,288 atoms: the per-replica sums of energy and virial run over two chunks of 8,192
    # atoms and a second pass that adds the chunk partials
    s = synth.water_box(4096, 5)
    w = synth.water_weights()
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    assert out["energy"].item() == pytest.approx(ref["energy"], rel=1e-11)
    assert out["energy"].item() == pytest.approx(out["atom_energy"].sum().item(), rel=1e-13)
    Fs = np.abs(ref["forces"]).max()
    np.testing.assert_allclose(out["virial"].cpu().numpy(), ref["virial"], rtol=1e-9, atol=1e-12 * Fs)


def test_fp64_copper_small(dp):
    s = synth.copper_fcc(4, 2)
    w = synth.copper_weights()
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    assert _rel_energy_err(out["atom_energy"].cpu().numpy(), ref["atom_energy"]).max() <= 1e-10
    Fs = np.abs(ref["forces"]).max()
    assert np.abs(out["forces"].cpu().numpy() - ref["forces"]).max() <= 1e-9 * Fs


@pytest.mark.parametrize("n_mol", [64, 1024])
def test_fp32_matches_oracle(dp, n_mol):
    s = synth.water_box(n_mol, 1)
    w = synth.water_weights()
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box)
    m = dp.DPModel(w, "fp32", max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    F = out["forces"].cpu().numpy()
    rmse = np.sqrt(((F - ref["forces"]) ** 2).mean())
    rms = np.sqrt((ref["forces"] ** 2).mean())
    assert rmse <= 1e-5
    assert rmse / rms <= 1e-4
    Ei = out["atom_energy"].cpu().numpy()
    assert np.abs(Ei - ref["atom_energy"]).max() <= 1e-5
    assert abs(out["energy"].item() - ref["energy"]) / s.natoms <= 1e-6


def test_fp32_copper_subbox(dp):
    """Cu 32^3 (131,072 atoms) in FP32; errors on the 4,000 atoms of FCC cells [0,10)^3,
    with the oracle evaluating only centres within r_c of that sub-box.  The untrained
    model's forces are ~1e-5 eV/A, so the bars are relative to the signal."""
    s = synth.copper_fcc(32, 0)
    w = synth.copper_weights()
    sub, centre = copper_subbox_masks(s, 3.634, w.rcut)
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box, centre_mask=centre)
    m = dp.DPModel(w, "fp32", max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    e = errors(out, ref, s.types, sub)
    assert e["f_rmse"] <= 1e-5, e
    assert e["f_rel"] <= 1e-4, e
    assert e["dev_rel"] <= 0.3, e  # E_i spread 7e-6 eV, FP32 rounding of E_i ~ 1e-7 eV
    assert e["ei_max"] <= 1e-5, e


# ------------------------------------------------------------------ batch / edge cases
def test_batch_equals_single(dp):
    reps = [synth.water_box(n, 10 + n) for n in (32, 40, 64, 7)]
    w = synth.water_weights()
    coords, types, offs, boxes = synth.concat(reps)
    m = dp.DPModel(w, "fp64", max_atoms=len(types), max_replicas=len(reps))
    x = torch.tensor(coords, device="cuda")
    t = torch.tensor(types, device="cuda")
    out = m.compute_batch(x, t, offs, boxes)
    orc = oracle.Model(w.to_blob())
    for r, s in enumerate(reps):
        ref = orc.compute(s.coords, s.types, s.box)
        assert out["energy"][r].item() == pytest.approx(ref["energy"], rel=1e-12)
        F = out["forces"][offs[r]:offs[r + 1]].cpu().numpy()
        assert np.abs(F - ref["forces"]).max() <= 1e-9 * np.abs(ref["forces"]).max()
        np.testing.assert_allclose(out["virial"][r].cpu().numpy(), ref["virial"], rtol=1e-9, atol=1e-13)


def test_isolated_atoms_and_single_atom(dp):
    w = synth.water_weights()
    orc = oracle.Model(w.to_blob())
    L = 40.0
    box = np.diag([L, L, L]).ravel()
    for coords, types in ((np.array([[1.0, 2.0, 3.0]]), np.array([1], np.int32)),
                          (np.array([[1.0, 2, 3], [20.0, 20, 20], [5.0, 30, 12]]), np.array([0, 1, 0], np.int32))):
        m = dp.DPModel(w, "fp64", max_atoms=8)
        out = m.compute(torch.tensor(coords, device="cuda"), torch.tensor(types, device="cuda"), box)
        ref = orc.compute(coords, types, box)
        np.testing.assert_allclose(out["atom_energy"].cpu().numpy(), ref["atom_energy"], rtol=1e-12)
        assert np.abs(out["forces"].cpu().numpy()).max() == 0.0


def test_sel_overflow_is_reported(dp):
    w = synth.xavier_weights(("O", "H"), 6.0, 0.5, (10, 20), 1001)
    s = synth.water_box(64, 0)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x, t = _cuda(s)
    with pytest.raises(dp.DPError) as e:
        m.compute(x, t, s.box)
    assert e.value.status == 5
    # the model stays usable
    w2 = synth.water_weights()
    m2 = dp.DPModel(w2, "fp64", max_atoms=s.natoms)
    m2.compute(x, t, s.box)


def test_bad_arguments(dp):
    w = synth.water_weights()
    s = synth.water_box(8, 0)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x, t = _cuda(s)
    flat = s.box.copy()
    flat[3:6] = flat[0:3]  # two equal cell vectors: zero volume
    with pytest.raises(dp.DPError) as e:
        m.compute(x, t, flat)
    assert e.value.status == 1
    big = synth.water_box(16, 0)
    xb, tb = _cuda(big)
    with pytest.raises(dp.DPError) as e:
        m.compute(xb, tb, big.box)
    assert e.value.status == 8
    bad_t = t.clone()
    bad_t[3] = 7
    with pytest.raises(dp.DPError) as e:
        m.compute(x, bad_t, s.box)
    assert e.value.status == 1


# ------------------------------------------------------------------ MD
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_md_matches_oracle_trajectory(dp, prec):
    s = synth.water_box(64, 0)
    w = synth.water_weights()
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    nsteps = 20
    ref = oracle.Model(w.to_blob()).md(s.coords, v0, s.types, s.box, s.masses(), 0.5, nsteps, rebuild_every=10)
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x = torch.tensor(s.coords, device="cuda")
    v = torch.tensor(v0, device="cuda")
    t = torch.tensor(s.types, device="cuda")
    st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=10)
    out = m.verlet(st, 0.5, nsteps, capture_graph=True)
    tol_x = 1e-10 if prec == "fp64" else 1e-6
    np.testing.assert_allclose(x.cpu().numpy(), ref["x"], atol=tol_x)
    np.testing.assert_allclose(v.cpu().numpy(), ref["v"], atol=tol_x)
    assert out["potential"].item() == pytest.approx(ref["pe"][-1], rel=1e-10 if prec == "fp64" else 1e-6)
    assert out["kinetic"].item() == pytest.approx(ref["ke"][-1], rel=1e-9 if prec == "fp64" else 1e-5)


def test_md_graph_equals_eager(dp):
    s = synth.water_box(64, 2)
    w = synth.water_weights()
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 5)
    res = []
    for cap in (False, True):
        m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
        x = torch.tensor(s.coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=5)
        m.verlet(st, 0.5, 12, capture_graph=cap)
        res.append((x.cpu().numpy(), v.cpu().numpy()))
    np.testing.assert_allclose(res[0][0], res[1][0], atol=1e-12)
    np.testing.assert_allclose(res[0][1], res[1][1], atol=1e-12)


def test_md_skin_exceeded_is_reported(dp):
    s = synth.water_box(8, 0)
    w = synth.water_weights()
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x = torch.tensor(s.coords, device="cuda")
    v = torch.zeros_like(x)
    v[0, 0] = 0.5  # 0.5 A/fs: 1.25 A after 5 steps of 0.5 fs, beyond skin/2
    t = torch.tensor(s.types, device="cuda")
    st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=100)
    with pytest.raises(dp.DPError) as e:
        m.verlet(st, 0.5, 6, capture_graph=False)
    assert e.value.status == 6


# ------------------------------------------------------------------ mixed precision (tensor cores)
@pytest.mark.parametrize("which", [0, 1, 2, 3, 4, 5, 6, 7])
def test_tensor_core_layout_selftest(dp, which):
    # 0-4: K-major operands of several shapes; 5-7: MN-major B, MN-major A, both MN-major
    err, vmax = dp.selftest(which)
    assert vmax > 1.0
    assert err == 0.0


# measured relative error x margin on the untrained models (force RMSE / force RMS,
# per-atom energy deviations; see _parity.py)
MIX_BARS = {"mix_bf16": {"f_rel": 3e-2, "dev_rel": 0.5}, "mix_fp16": {"f_rel": 1e-2, "dev_rel": 0.3}}


@pytest.mark.parametrize("prec", ["mix_bf16", "mix_fp16"])
@pytest.mark.parametrize("n_mol", [64, 1024])
def test_mixed_matches_oracle_water(dp, prec, n_mol):
    s = synth.water_box(n_mol, 2)
    w = synth.water_weights()
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box)
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    e = errors(out, ref, s.types)
    assert e["f_rmse"] <= 2e-3, e
    assert e["f_rel"] <= MIX_BARS[prec]["f_rel"], e
    assert e["dev_rel"] <= MIX_BARS[prec]["dev_rel"], e
    assert e["e_atom"] <= 1e-4, e
    np.testing.assert_allclose(out["virial"].cpu().numpy(), ref["virial"], rtol=0.05,
                               atol=3 * MIX_BARS[prec]["f_rel"] * np.abs(ref["virial"]).max())


@pytest.mark.parametrize("prec", ["mix_bf16", "mix_fp16"])
def test_mixed_copper_subbox(dp, prec):
    s = synth.copper_fcc(32, 0)
    w = synth.copper_weights()
    sub, centre = copper_subbox_masks(s, 3.634, w.rcut)
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box, centre_mask=centre)
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x, t = _cuda(s)
    out = m.compute(x, t, s.box)
    e = errors(out, ref, s.types, sub)
    assert e["f_rmse"] <= 2e-3, e
    assert e["f_rel"] <= MIX_BARS[prec]["f_rel"], e
    assert e["e_atom"] <= 1e-4, e
    # the untrained copper E_i spread (7e-6 eV) is below the 16-bit rounding of E_i itself;
    # the deviation measure is checked on the normalised model (test_gpu_normalised.py)
    assert e["ei_max"] <= 1e-4, e


def test_md_water12k_fp32_tracks_fp64(dp):
    # 4096 H2O (12,288 atoms), 300 K, dt 0.5 fs, rebuild every 10 steps.  With random weights
    # two atoms of this box collapse together between steps 31 and 41 in every precision (an
    # untrained model has no short-range repulsion), so the run stops at 30 steps.
    s = synth.water_box(4096, 0)
    w = synth.water_weights()
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 1)
    res = {}
    for prec in ("fp64", "fp32"):
        m = dp.DPModel(w, prec, max_atoms=s.natoms)
        x = torch.tensor(s.coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=10)
        out = m.verlet(st, 0.5, 1)
        e1 = out["potential"].item() + out["kinetic"].item()
        st.resume = 1
        out = m.verlet(st, 0.5, 29)
        e30 = out["potential"].item() + out["kinetic"].item()
        res[prec] = (x.cpu().numpy(), out["potential"].item(), abs(e30 - e1) / s.natoms)
        m.close()
    assert res["fp64"][2] <= 1e-6 and res["fp32"][2] <= 1e-6
    assert np.abs(res["fp32"][0] - res["fp64"][0]).max() <= 1e-4
    assert res["fp32"][1] == pytest.approx(res["fp64"][1], rel=1e-6)
