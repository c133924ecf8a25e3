"""Tabulated (compressed) embedding on the GPU against the oracle's tabulated model (GPU only).

Both sides build their own tables from the same weights (the oracle with second-order jets
through its net, the library with explicit forward-mode formulas in an FP64 kernel) on the same
intervals, so the tabulated results agree at each precision's bar; the tables themselves differ
from the nets by the quintic interpolation error (about 1e-10 at 256 intervals)."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

from _parity import copper_subbox_masks, env_stats, errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NINT = 256
# precision bars as for the networks (test_gpu_normalised.py), relative to the signal; measured
# with the tables: fp32 f_rel 1e-6, mix_fp16 f_rel 8e-4 (water) / 3.3e-3 (Cu), dev_rel 2e-3 / 3.1e-2
BARS = {"water": {"fp32": {"f_rel": 1e-4, "dev_rel": 1e-3},
                  "mix_bf16": {"f_rel": 2e-2, "dev_rel": 0.1},
                  "mix_fp16": {"f_rel": 3e-3, "dev_rel": 1e-2}},
        "copper": {"mix_fp16": {"f_rel": 1e-2, "dev_rel": 0.1}}}


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


def _tabulated_pair(dp, w, prec, natoms):
    m = dp.DPModel(w, prec, max_atoms=natoms)
    x0, x1, n = m.tabulate(NINT)
    orc = oracle.Model(w.to_blob())
    orc.tabulate(x0, x1, n)
    return m, orc


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_bf16", "mix_fp16"])
def test_tabulated_water_matches_oracle_table(dp, prec):
    s = synth.water_box(64, 2)
    w = synth.normalised_weights("water", env_stats())
    m, orc = _tabulated_pair(dp, w, prec, s.natoms)
    ref = orc.compute(s.coords, s.types, s.box)
    out = m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    e = errors(out, ref, s.types)
    if prec == "fp64":
        assert e["ei_rel"] <= 1e-10, e
        assert e["f_rel"] <= 1e-9, e
        np.testing.assert_allclose(out["virial"].cpu().numpy(), ref["virial"], rtol=1e-9, atol=1e-12)
    else:
        assert e["f_rel"] <= BARS["water"][prec]["f_rel"], e
        assert e["dev_rel"] <= BARS["water"][prec]["dev_rel"], e
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_tabulated_copper_subbox(dp, prec):
    s = synth.copper_fcc(32, 0)
    w = synth.normalised_weights("copper", env_stats())
    sub, centre = copper_subbox_masks(s, 3.634, w.rcut)
    m, orc = _tabulated_pair(dp, w, prec, s.natoms)
    ref = orc.compute(s.coords, s.types, s.box, centre_mask=centre)
    out = m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    e = errors(out, ref, s.types, sub)
    if prec == "fp64":
        assert e["ei_rel"] <= 1e-10, e
        assert e["f_rel"] <= 1e-9, e
    else:
        assert e["f_rel"] <= BARS["copper"][prec]["f_rel"], e
        assert e["dev_rel"] <= BARS["copper"][prec]["dev_rel"], e
        assert e["e_atom"] <= 1e-4 and e["f_rmse"] <= 2e-3, e
    m.close()


def test_table_close_to_network_and_switch_back(dp):
    # the GPU tables against the GPU nets (FP64): the interpolation error only; n = 0 restores
    s = synth.water_box(64, 3)
    w = synth.normalised_weights("water", env_stats())
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    x = torch.tensor(s.coords, device="cuda")
    t = torch.tensor(s.types, device="cuda")
    net = m.compute(x, t, s.box)
    m.tabulate(NINT)
    tab = m.compute(x, t, s.box)
    dE = abs(tab["energy"].item() - net["energy"].item()) / s.natoms
    dF = (tab["forces"] - net["forces"]).abs().max().item()
    assert 0 < dE < 1e-8 and dF < 1e-7, (dE, dF)
    m.tabulate(0)
    back = m.compute(x, t, s.box)
    assert back["energy"].item() == pytest.approx(net["energy"].item(), rel=1e-14)
    m.close()


def test_tabulated_md_fp64_follows_oracle(dp):
    s = synth.water_box(64, 0)
    w = synth.water_weights()
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    m, orc = _tabulated_pair(dp, w, "fp64", s.natoms)
    ref = orc.md(s.coords, v0, s.types, s.box, s.masses(), 0.5, 20, rebuild_every=10)
    x = torch.tensor(s.coords, device="cuda")
    v = torch.tensor(v0, device="cuda")
    st = m.md_state(x, v, torch.tensor(s.types, device="cuda"), s.box, s.masses(), rebuild_every=10)
    out = m.verlet(st, 0.5, 20, capture_graph=True)
    np.testing.assert_allclose(x.cpu().numpy(), ref["x"], atol=1e-10)
    assert out["potential"].item() == pytest.approx(ref["pe"][-1], rel=1e-10)
    m.close()


def test_param_grad_refused_on_tables(dp):
    s = synth.water_box(8, 0)
    w = synth.water_weights()
    m = dp.DPModel(w, "fp64", max_atoms=s.natoms)
    m.tabulate(64)
    x = torch.tensor(s.coords, device="cuda")
    with pytest.raises(dp.DPError) as e:
        m.param_grad(x, torch.tensor(s.types, device="cuda"), s.box, 0.0, torch.zeros_like(x))
    assert e.value.status == 4
    m.close()
