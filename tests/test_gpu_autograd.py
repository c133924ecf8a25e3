"""Force backward behind torch.autograd.Function, and the measurement / error-path hooks
(GPU only).

Potential: E(x) of one box, with the coordinate gradient -F from the library's force
backward (prod_force), against central differences of E and the FP64 oracle on the
1024-H2O box."""
import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


def test_potential_gradient_is_minus_force(dp, water_weights):
    s = synth.water_box(1024, 3)
    m = dp.DPModel(water_weights, "fp64", max_atoms=s.natoms)
    x = torch.tensor(s.coords, device="cuda", requires_grad=True)
    t = torch.tensor(s.types, device="cuda")
    E, V = dp.Potential.apply(x, m, t, s.box)
    assert E.requires_grad and not V.requires_grad
    (2.5 * E).backward()
    ref = oracle.Model(water_weights.to_blob()).compute(s.coords, s.types, s.box)
    assert E.item() == pytest.approx(ref["energy"], rel=1e-12)
    g = x.grad.cpu().numpy()
    np.testing.assert_allclose(g, -2.5 * ref["forces"], rtol=1e-8, atol=1e-9 * np.abs(ref["forces"]).max())
    np.testing.assert_allclose(V.cpu().numpy(), ref["virial"], rtol=1e-9, atol=1e-12)
    # central differences of E through the same function (h = 1e-5 A) on 20 random atoms.
    # E ~ 4.2e3 eV is summed with FP64 atomics (order-dependent at ~1e-12 eV), so a difference
    # over 2h carries ~1e-7 eV/A of rounding; the forces are ~1e-3 eV/A.
    rng = np.random.default_rng(5)
    h = 1e-5
    with torch.no_grad():
        for i in rng.choice(s.natoms, 20, replace=False):
            a = int(rng.integers(0, 3))
            xp = x.detach().clone(); xp[i, a] += h
            xm = x.detach().clone(); xm[i, a] -= h
            ep, _ = dp.Potential.apply(xp, m, t, s.box)
            em, _ = dp.Potential.apply(xm, m, t, s.box)
            fd = (ep.item() - em.item()) / (2 * h)
            assert fd == pytest.approx(g[i, a] / 2.5, rel=1e-5, abs=2e-7)
    m.close()


def test_potential_in_a_torch_loss(dp, water_weights):
    # a loss mixing the energy with other torch terms: autograd routes grad_E through -F
    s = synth.water_box(64, 1)
    m = dp.DPModel(water_weights, "fp32", max_atoms=s.natoms)
    x = torch.tensor(s.coords, device="cuda", requires_grad=True)
    t = torch.tensor(s.types, device="cuda")
    E, _ = dp.Potential.apply(x, m, t, s.box)
    loss = (E - 400.0) ** 2 + 0.1 * (x ** 2).sum()
    loss.backward()
    F = m.compute(x.detach(), t, s.box)["forces"]
    expect = -2.0 * (E.item() - 400.0) * F + 0.2 * x.detach()
    torch.testing.assert_close(x.grad, expect, rtol=1e-6, atol=1e-9)
    m.close()


def test_bounded_wait_gives_up_and_device_stays_usable(dp):
    # a wait on an mbarrier phase that nothing completes returns DP_ERR_WAIT_TIMEOUT
    assert dp.wait_selftest(4096) == 7
    assert dp.wait_selftest(64) == 7
    # the context is intact: a tensor-core self check and a small evaluation still work
    err, vmax = dp.selftest(0)
    assert err == 0.0 and vmax > 1.0
    s = synth.water_box(8, 0)
    m = dp.DPModel(synth.water_weights(), "mix_fp16", max_atoms=s.natoms)
    out = m.compute(torch.tensor(s.coords, device="cuda"), torch.tensor(s.types, device="cuda"), s.box)
    assert np.isfinite(out["energy"].item())
    m.close()


def test_measured_peaks_are_plausible(dp):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = {k: dp.measure_peak(k) for k in ("tanh", "ex2", "rcp", "ffma", "dfma")}
    # per SM per clock at <= 2.1 GHz: transcendental 4..32, FP32 FMA <= 128 (256 FLOP)
    for k in ("tanh", "ex2", "rcp"):
        per = r[k] / (sms * 2.1e9)
        assert 2.0 <= per <= 64.0, (k, r[k])
    assert 1e13 < r["ffma"] < sms * 256 * 2.2e9, r
    assert 1e11 < r["dfma"] < r["ffma"], r
