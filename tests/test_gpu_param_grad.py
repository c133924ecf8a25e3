"""Parameter gradient dp_param_grad (tangent-forward + reverse sweep) against the
FP64 oracle's dual-number gradient at sampled parameters, through the C-ABI (GPU only).

L = cE (E - E0)^2 + cF sum_k |F_k - F0_k|^2.  Indices are sampled from every
parameter block (each embedding pair's W1..b3, each fitting net's W1..b4, e_bias).
Bars: FP64 within 1e-9 of the sample's largest |dL/dtheta|; FP32 within 2e-3."""
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


def _indices(w, per_block, seed):
    layout, ntheta = synth.theta_layout(w.ntypes)
    rng = np.random.default_rng(seed)
    idx = []
    for _name, shape, off in layout:
        n = int(np.prod(shape))
        idx += [off + int(k) for k in rng.choice(n, size=min(per_block, n), replace=False)]
    return np.array(sorted(idx), dtype=np.int64), ntheta


def _targets(om, s, seed):
    ref = om.compute(s.coords, s.types, s.box)
    rng = np.random.default_rng(seed)
    E0 = ref["energy"] - 0.5
    F0 = ref["forces"] + rng.normal(0.0, 0.05, size=ref["forces"].shape)
    return E0, F0


def _gpu_grad(dp, w, s, prec, E0, F0, cE, cF):
    m = dp.DPModel(w, prec, max_atoms=s.natoms)
    x = torch.tensor(s.coords, dtype=torch.float64, device="cuda")
    t = torch.tensor(s.types, dtype=torch.int32, device="cuda")
    f0 = torch.tensor(F0, dtype=torch.float64, device="cuda")
    g, loss = m.param_grad(x, t, s.box, E0, f0, cE, cF)
    out = g.cpu().numpy(), float(loss.item())
    m.close()
    return out


@pytest.fixture(scope="module")
def water64_case(water_weights):
    s = synth.water_box(64, 5)
    om = oracle.Model(water_weights.to_blob())
    E0, F0 = _targets(om, s, 11)
    idx, ntheta = _indices(water_weights, 2, 21)
    cE, cF = 1.0, 0.5
    g, _dE, loss = om.param_grad(s.coords, s.types, s.box, E0, F0, idx, cE, cF)
    return s, E0, F0, cE, cF, idx, ntheta, g, loss


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 2e-3)])
def test_param_grad_matches_oracle_water64(dp, water_weights, water64_case, prec, tol):
    s, E0, F0, cE, cF, idx, ntheta, g_ref, loss_ref = water64_case
    g, loss = _gpu_grad(dp, water_weights, s, prec, E0, F0, cE, cF)
    assert g.shape == (ntheta,)
    assert np.all(np.isfinite(g))
    scale = np.abs(g_ref).max()
    err = np.abs(g[idx] - g_ref)
    assert err.max() <= tol * scale, (prec, err.max() / scale, int(idx[np.argmax(err)]))
    assert loss == pytest.approx(loss_ref, rel=1e-10 if prec == "fp64" else 1e-4)


def test_param_grad_fp32_matches_fp64_everywhere(dp, water_weights, water64_case):
    s, E0, F0, cE, cF = water64_case[:5]
    g64, _ = _gpu_grad(dp, water_weights, s, "fp64", E0, F0, cE, cF)
    g32, _ = _gpu_grad(dp, water_weights, s, "fp32", E0, F0, cE, cF)
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)


@pytest.mark.parametrize("n_mol", [1024, 1400])
def test_param_grad_matches_oracle_large(dp, water_weights, n_mol):
    # 1024 molecules: the 3,072-atom gradient workload (several row chunks per pair);
    # 1400 molecules: 2,800 H centres, more than one centre-atom chunk
    s = synth.water_box(n_mol, 6)
    om = oracle.Model(water_weights.to_blob())
    E0, F0 = _targets(om, s, 12)
    layout, _ = synth.theta_layout(water_weights.ntypes)
    offs = {name: off for name, _shape, off in layout}
    idx = np.array(sorted([offs["emb01.W3"] + 7, offs["emb11.b2"] + 3, offs["fit1.W1"] + 12345,
                           offs["fit0.w4"] + 17, offs["e_bias"] + 1]), dtype=np.int64)
    g_ref, _dE, loss_ref = om.param_grad(s.coords, s.types, s.box, E0, F0, idx, 1.0, 0.5)
    g, loss = _gpu_grad(dp, water_weights, s, "fp64", E0, F0, 1.0, 0.5)
    scale = np.abs(g_ref).max()
    assert np.abs(g[idx] - g_ref).max() <= 1e-9 * scale
    assert loss == pytest.approx(loss_ref, rel=1e-10)


def test_param_grad_rejects_bad_arguments(dp, water_weights):
    s = synth.water_box(8, 1)
    m = dp.DPModel(water_weights, "fp64", max_atoms=s.natoms)
    x = torch.tensor(s.coords, dtype=torch.float64, device="cuda")
    t = torch.tensor(s.types, dtype=torch.int32, device="cuda")
    f0 = torch.zeros_like(x)
    small = dp.DPModel(water_weights, "fp64", max_atoms=8)
    with pytest.raises(dp.DPError) as e:
        small.param_grad(x, t, s.box, 0.0, f0)
    assert e.value.status == 8  # DP_ERR_CAPACITY
    g, loss = m.param_grad(x, t, s.box, 0.0, f0)
    assert torch.isfinite(g).all() and torch.isfinite(loss).all()
    m.close()
    small.close()
