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


def test_param_loss_autograd_matches_oracle(dp, water_weights, water64_case):
    # the torch.autograd.Function: loss.backward() gives the parameter gradient
    s, E0, F0, cE, cF, idx, ntheta, g_ref, loss_ref = water64_case
    m = dp.DPModel(water_weights, "fp64", max_atoms=s.natoms)
    x = torch.tensor(s.coords, dtype=torch.float64, device="cuda")
    t = torch.tensor(s.types, dtype=torch.int32, device="cuda")
    f0 = torch.tensor(F0, dtype=torch.float64, device="cuda")
    theta = torch.tensor(water_weights.theta, dtype=torch.float64, requires_grad=True)
    loss = dp.ParamLoss.apply(theta, m, x, t, s.box, E0, f0, cE, cF)
    loss.backward()
    g = theta.grad.numpy()
    assert loss.item() == pytest.approx(loss_ref, rel=1e-10)
    assert np.abs(g[idx] - g_ref).max() <= 1e-9 * np.abs(g_ref).max()
    m.close()


@pytest.fixture(scope="module")
def water1024_fd(dp, water_weights):
    # 1024 H2O; targets E0, F0 from a second seeded weight set (seed 2002), FP64 GPU
    s = synth.water_box(1024, 3)
    x = torch.tensor(s.coords, dtype=torch.float64, device="cuda")
    t = torch.tensor(s.types, dtype=torch.int32, device="cuda")
    m2 = dp.DPModel(synth.water_weights(2002), "fp64", max_atoms=s.natoms)
    tgt = m2.compute(x, t, s.box)
    m2.close()
    m = dp.DPModel(water_weights, "fp64", max_atoms=s.natoms)
    return s, x, t, m, tgt["energy"].item(), tgt["forces"].clone()


def test_forces_and_virial_match_finite_differences_water1024(water1024_fd):
    s, x, t, m, _E0, _F0 = water1024_fd
    out = m.compute(x, t, s.box)
    F = out["forces"].cpu().numpy()
    vir = out["virial"].cpu().numpy().reshape(3, 3)
    rng = np.random.default_rng(17)
    atoms = rng.choice(s.natoms, size=20, replace=False)
    h = 1e-5
    err = 0.0
    for k in atoms:
        for c in range(3):
            e = []
            for sgn in (1.0, -1.0):
                xp = x.clone()
                xp[k, c] += sgn * h
                e.append(m.compute(xp, t, s.box)["energy"].item())
            err = max(err, abs(-(e[0] - e[1]) / (2 * h) - F[k, c]))
    assert err <= 1e-6 * np.abs(F).max() + 2e-7, err
    # virial diagonal: Xi_aa = -dE/d(eps_aa) under x_a -> (1 + eps) x_a, L_a -> (1 + eps) L_a
    eps = 1e-6
    for a in range(3):
        e = []
        for sgn in (1.0, -1.0):
            sc = torch.ones(3, dtype=torch.float64, device="cuda")
            sc[a] += sgn * eps
            box = np.array(s.box, dtype=np.float64).reshape(3, 3).copy()
            box[a, a] *= 1.0 + sgn * eps
            e.append(m.compute(x * sc, t, box)["energy"].item())
        fd = -(e[0] - e[1]) / (2 * eps)
        assert fd == pytest.approx(vir[a, a], rel=1e-5, abs=1e-6 * np.abs(vir).max())
    np.testing.assert_allclose(vir, vir.T, atol=1e-9 * np.abs(vir).max())


def test_param_grad_matches_finite_differences_50_weights(dp, water_weights, water1024_fd):
    s, x, t, m, E0, F0 = water1024_fd
    cE, cF = 1.0, 1.0
    g, loss = m.param_grad(x, t, s.box, E0, F0, cE, cF)
    g = g.cpu().numpy()
    theta0 = np.array(water_weights.theta, dtype=np.float64)
    layout, ntheta = synth.theta_layout(water_weights.ntypes)
    rng = np.random.default_rng(50)
    blocks = [(off, int(np.prod(shape))) for _n, shape, off in layout]
    pick = rng.choice(len(blocks), size=50, replace=True)
    idx = sorted({blocks[b][0] + int(rng.integers(blocks[b][1])) for b in pick})

    def L(theta):
        m.set_params(theta)
        out = m.compute(x, t, s.box)
        dF = out["forces"] - F0
        return cE * (out["energy"].item() - E0) ** 2 + cF * float((dF * dF).sum().item())

    h = 1e-3
    fd = []
    for p in idx:
        vals = []
        for k in (2, 1, -1, -2):
            th = theta0.copy()
            th[p] += k * h
            vals.append(L(th))
        fd.append((-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h))
    m.set_params(theta0)
    fd = np.array(fd)
    assert L(theta0) == pytest.approx(loss.item(), rel=1e-10)
    scale = max(np.abs(fd).max(), 1e-30)
    assert np.abs(g[idx] - fd).max() <= 1e-6 * scale, (np.abs(g[idx] - fd).max() / scale)
