"""Batched replicas: many independent periodic boxes of uneven size, concatenated
CSR-style and advanced by dp_md_run_batch (one launch per phase for all boxes,
under a CUDA graph), against the oracle run on each replica alone (GPU only)."""
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


def _velocities(reps, seed):
    return [synth.maxwell_boltzmann(s.masses()[s.types], 300.0, seed + r) for r, s in enumerate(reps)]


def _batch_state(dp, w, reps, v0, prec):
    coords, types, offs, boxes = synth.concat(reps)
    m = dp.DPModel(w, prec, max_atoms=len(types), max_replicas=len(reps))
    x = torch.tensor(coords, device="cuda")
    v = torch.tensor(np.concatenate(v0), device="cuda")
    t = torch.tensor(types, device="cuda")
    st = m.md_state(x, v, t, boxes, reps[0].masses(), atom_offsets=offs, rebuild_every=10)
    return m, st, x, v, offs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_md_batch_matches_oracle_per_replica(dp, water_weights, prec):
    reps = synth.water_replicas(5, 3, lo=32, hi=160)
    v0 = _velocities(reps, 40)
    nsteps = 20
    m, st, x, v, offs = _batch_state(dp, water_weights, reps, v0, prec)
    out = m.md_run_batch(st, 0.5, nsteps)
    orc = oracle.Model(water_weights.to_blob())
    tol_x = 1e-10 if prec == "fp64" else 1e-6
    for r, s in enumerate(reps):
        ref = orc.md(s.coords, v0[r], s.types, s.box, s.masses(), 0.5, nsteps, rebuild_every=10)
        sl = slice(offs[r], offs[r + 1])
        np.testing.assert_allclose(x[sl].cpu().numpy(), ref["x"], atol=tol_x)
        np.testing.assert_allclose(v[sl].cpu().numpy(), ref["v"], atol=tol_x)
        rel = 1e-10 if prec == "fp64" else 1e-6
        assert out["potential"][r].item() == pytest.approx(ref["pe"][-1], rel=rel)
        assert out["kinetic"][r].item() == pytest.approx(ref["ke"][-1], rel=10 * rel)
    m.close()


def test_md_batch_equals_separate_runs(dp, water_weights):
    reps = synth.water_replicas(4, 8, lo=32, hi=200)
    v0 = _velocities(reps, 90)
    m, st, x, v, offs = _batch_state(dp, water_weights, reps, v0, "fp64")
    out = m.md_run_batch(st, 0.5, 15)
    for r, s in enumerate(reps):
        m1 = dp.DPModel(water_weights, "fp64", max_atoms=s.natoms)
        x1 = torch.tensor(s.coords, device="cuda")
        v1 = torch.tensor(v0[r], device="cuda")
        t1 = torch.tensor(s.types, device="cuda")
        st1 = m1.md_state(x1, v1, t1, s.box, s.masses(), rebuild_every=10)
        o1 = m1.verlet(st1, 0.5, 15)
        sl = slice(offs[r], offs[r + 1])
        np.testing.assert_allclose(x[sl].cpu().numpy(), x1.cpu().numpy(), atol=1e-12)
        assert out["potential"][r].item() == pytest.approx(o1["potential"].item(), rel=1e-12)
        m1.close()
    m.close()


def test_md_batch_256_replicas_mixed(dp, water_weights):
    # 256 water boxes of 32..2048 molecules (96..6,144 atoms), densities +-3%
    reps = synth.water_replicas(256, 4)
    v0 = _velocities(reps, 1000)
    N = sum(s.natoms for s in reps)
    assert 2.0e5 < N < 6.0e5
    m, st, x, v, offs = _batch_state(dp, water_weights, reps, v0, "mix_fp16")
    # initial energies of the smallest replicas against the oracle (mixed bar: 1e-4 eV/atom)
    coords, types, offs_c, boxes = synth.concat(reps)
    e0 = m.compute_batch(torch.tensor(coords, device="cuda"), torch.tensor(types, device="cuda"), offs_c,
                         boxes)["energy"].cpu().numpy()
    orc = oracle.Model(water_weights.to_blob())
    # per-replica parity on the four smallest replicas and two of mid size: energy per atom,
    # force error relative to the force RMS, per-atom energy deviations (see _parity.py)
    order = np.argsort([s.natoms for s in reps])
    pick = list(order[:4]) + [order[len(order) // 2], order[len(order) // 2 + 1]]
    out0 = m.compute_batch(torch.tensor(coords, device="cuda"), torch.tensor(types, device="cuda"), offs_c, boxes)
    for r in pick:
        ref = orc.compute(reps[r].coords, reps[r].types, reps[r].box)
        assert abs(e0[r] - ref["energy"]) / reps[r].natoms <= 1e-4
        sl = slice(offs_c[r], offs_c[r + 1])
        e = errors({"forces": out0["forces"][sl], "atom_energy": out0["atom_energy"][sl]}, ref, reps[r].types)
        assert e["f_rel"] <= 1e-2, (r, e)
        assert e["dev_rel"] <= 0.3, (r, e)
    # 25 NVE steps: every replica stays finite and conserves its total energy.  (An untrained
    # model has no short-range repulsion: a few of these replicas see two atoms collapse
    # together after ~35 steps, identically in every precision and in the oracle; see
    # test_md_batch_through_close_encounter.)
    out = m.md_run_batch(st, 0.5, 1)
    etot0 = (out["potential"] + out["kinetic"]).cpu().numpy().copy()
    st.resume = 1
    out = m.md_run_batch(st, 0.5, 24)
    etot1 = (out["potential"] + out["kinetic"]).cpu().numpy()
    assert np.all(np.isfinite(etot1))
    natoms = np.array([s.natoms for s in reps])
    drift = np.abs(etot1 - etot0) / natoms
    assert drift.max() <= 2e-4, drift.max()
    m.close()


def test_md_batch_through_close_encounter(dp, water_weights):
    # Replica 177 of the 256-replica set: two atoms collapse together between steps 36 and
    # 41 (max speed ~0.7 A/fs, energy jump ~0.017 eV/atom).  The batch run in FP64 must follow
    # the oracle through that stiff event; two small replicas ride along.
    allreps = synth.water_replicas(256, 4)
    idx = [177, 3, 60]
    reps = [allreps[r] for r in idx]
    v0 = [synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 1000 + r) for r, s in zip(idx, reps)]
    m, st, x, v, offs = _batch_state(dp, water_weights, reps, v0, "fp64")
    m.md_run_batch(st, 0.5, 1)
    st.resume = 1
    out = m.md_run_batch(st, 0.5, 40)  # 41 steps, as the oracle below
    ref = oracle.Model(water_weights.to_blob()).md(reps[0].coords, v0[0], reps[0].types, reps[0].box,
                                                   reps[0].masses(), 0.5, 41, rebuild_every=10)
    e_gpu = out["potential"][0].item() + out["kinetic"][0].item()
    e_ref = ref["pe"][-1] + ref["ke"][-1]
    assert (ref["pe"][-1] + ref["ke"][-1] - ref["pe"][1] - ref["ke"][1]) / reps[0].natoms > 1e-3  # the event
    assert e_gpu == pytest.approx(e_ref, rel=1e-9)
    np.testing.assert_allclose(x[offs[0]:offs[1]].cpu().numpy(), ref["x"], atol=1e-8)
    m.close()


def test_autotune_choices_and_results(dp, water_weights):
    reps = synth.water_replicas(16, 21, lo=32, hi=400)
    coords, types, offs, boxes = synth.concat(reps)
    m = dp.DPModel(water_weights, "mix_fp16", max_atoms=len(types), max_replicas=len(reps))
    x = torch.tensor(coords, device="cuda")
    t = torch.tensor(types, device="cuda")
    ref = m.compute_batch(x, t, offs, boxes)
    e_ref = ref["energy"].cpu().numpy()
    f_ref = ref["forces"].cpu().numpy()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    grids = m.autotune(2)
    allowed = [{1, 2, 3, 6}, {1, 2, 3, 6}, {2, 4, 5, 10}, {4, 8, 16}]
    for g, ok in zip(grids, allowed):
        assert g % sms == 0 and g // sms in ok, grids
    assert m.autotune(0) == grids
    # other launch shapes change only the order of FP32 atomic sums, which can flip a 16-bit
    # rounding downstream (one fp16 ulp ~ 5e-4 relative): compare at the mixed-precision level
    out = m.compute_batch(x, t, offs, boxes)
    np.testing.assert_allclose(out["energy"].cpu().numpy(), e_ref, rtol=1e-6)
    f = out["forces"].cpu().numpy()
    assert np.sqrt(((f - f_ref) ** 2).mean()) <= 1e-3 * np.sqrt((f_ref ** 2).mean())
    m.close()
    # dp_md_run_batch tunes on its first call
    v0 = _velocities(reps, 3)
    m2, st, x2, v2, offs2 = _batch_state(dp, water_weights, reps, v0, "mix_fp16")
    assert m2.autotune(0) == [0, 0, 0, 0]
    m2.md_run_batch(st, 0.5, 2)
    assert all(g > 0 for g in m2.autotune(0))
    m2.close()


@pytest.mark.parametrize("prec", ["fp64", "mix_fp16"])
def test_batch_sums_over_uneven_chunks(dp, water_weights, prec):
    # Replicas of 64, 4096 and 37 molecules: the per-replica energy and virial sums run in
    # chunks of 8,192 atoms, two for the large box and empty trailing chunks for the small
    # ones, before the second pass adds each replica's chunks in order.
    reps = [synth.water_box(64, 1), synth.water_box(4096, 2), synth.water_box(37, 3)]
    coords, types, offs, boxes = synth.concat(reps)
    m = dp.DPModel(water_weights, prec, max_atoms=len(types), max_replicas=len(reps))
    x = torch.tensor(coords, device="cuda")
    t = torch.tensor(types, device="cuda")
    out = m.compute_batch(x, t, offs, boxes)
    Ei = out["atom_energy"].cpu().numpy()
    orc = oracle.Model(water_weights.to_blob())
    for r, s in enumerate(reps):
        sl = slice(offs[r], offs[r + 1])
        # the sum over chunks equals this replica's per-atom energies summed on the host
        assert out["energy"][r].item() == pytest.approx(Ei[sl].sum(), rel=1e-12)
        ref = orc.compute(s.coords, s.types, s.box)
        if prec == "fp64":
            assert out["energy"][r].item() == pytest.approx(ref["energy"], rel=1e-11)
            Fs = np.abs(ref["forces"]).max()
            np.testing.assert_allclose(out["virial"][r].cpu().numpy(), ref["virial"], rtol=1e-9, atol=1e-12 * Fs)
        else:
            # the benchmark spec energy bar per atom
            assert abs(out["energy"][r].item() - ref["energy"]) / s.natoms <= 1e-4
    m.close()
