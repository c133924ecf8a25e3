"""Pins of the FP64 oracle against facts fixed by the mathematics, not by the oracle
itself: brute force, finite differences, dual numbers, invariances, closed forms on
sparse weights, and the analytic harmonic oscillator.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_22867_gb300 import synth


def _rot90_z(coords, L):
    # (x, y, z) -> (L - y, x, z): a symmetry of the periodic cube
    out = np.empty_like(coords)
    out[:, 0] = L - coords[:, 1]
    out[:, 1] = coords[:, 0]
    out[:, 2] = coords[:, 2]
    return out


# ----------------------------------------------------------------- neighbour list
def _py_brute(coords, types, L, rcut, sel):
    """Independent pure-Python brute force: the set of (type_j, j, n) with
    r^2 < rcut^2, in canonical order, from wrapped positions."""
    x = oracle.wrap(coords, np.diag([L, L, L]).ravel())
    N = len(types)
    nmax = math.ceil(rcut / L)
    rng = range(-nmax, nmax + 1)
    out = []
    for i in range(N):
        c = []
        for j in range(N):
            for nx in rng:
                for ny in rng:
                    for nz in rng:
                        if i == j and nx == ny == nz == 0:
                            continue
                        d = [(x[j, a] + n * L) - x[i, a] for a, n in enumerate((nx, ny, nz))]
                        r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
                        if r2 < rcut * rcut:
                            c.append((int(types[j]), j, nx, ny, nz))
        out.append(sorted(c))
    return out


def _unpack(code):
    return ((code >> 20) & 1023) - 512, ((code >> 10) & 1023) - 512, (code & 1023) - 512


def _rows(nl, im, types, sel):
    rows = []
    offs = np.concatenate([[0], np.cumsum(sel)])
    for i in range(nl.shape[0]):
        r = []
        for t in range(len(sel)):
            for k in range(offs[t], offs[t + 1]):
                j = nl[i, k]
                if j < 0:
                    break
                assert types[j] == t
                r.append((t, int(j)) + _unpack(int(im[i, k])))
        rows.append(r)
    return rows


def test_nlist_brute_matches_python_brute_force_multi_image():
    # 8 molecules in a 6.2 A box: rcut 8 A reaches the second periodic image
    s = synth.water_box(8, 3)
    w = synth.water_weights()
    m = oracle.Model(w.to_blob())
    L = s.box[0]
    for rc in (6.0, 8.0):
        sel = (400, 800)
        nl, im, cnt, ovf = m.nlist(s.coords, s.types, s.box, "brute", rcut=rc, sel=sel)
        assert not ovf
        ref = _py_brute(s.coords, s.types, L, rc, sel)
        got = _rows(nl, im, s.types, sel)
        assert got == ref
        assert max(len(r) for r in ref) > 24 * 2  # several images of the same j exist
        assert (cnt.sum(1) == [len(r) for r in ref]).all()


@pytest.mark.parametrize("kind,n,seed", [("water", 64, 0), ("water", 32, 5), ("water", 216, 7), ("cu", 3, 1)])
def test_nlist_cell_equals_brute(kind, n, seed):
    if kind == "water":
        s = synth.water_box(n, seed)
        w = synth.water_weights()
    else:
        s = synth.copper_fcc(n, seed)
        w = synth.copper_weights()
    m = oracle.Model(w.to_blob())
    for rc in (0.0, w.rcut + 2.0):
        sel = None if rc == 0.0 else tuple(4 * x for x in w.sel)
        a = m.nlist(s.coords, s.types, s.box, "brute", rcut=rc, sel=sel)
        b = m.nlist(s.coords, s.types, s.box, "cell", rcut=rc, sel=sel)
        assert not a[3] and not b[3]
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(x, y)


def test_nlist_overflow_is_flagged():
    s = synth.water_box(64, 0)
    w = synth.water_weights()
    m = oracle.Model(w.to_blob())
    _, _, cnt, ovf = m.nlist(s.coords, s.types, s.box, "cell", sel=(10, 10))
    assert ovf and cnt.max() > 10


# ----------------------------------------------------------------- nearest-first truncation
def _py_nearest(coords, types, L, rcut, sel):
    """Independent Python: per atom and neighbour type, the sel_t candidates of the brute-force
    list with the smallest (r^2, j, nx, ny, nz), listed in canonical order."""
    x = oracle.wrap(coords, np.diag([L, L, L]).ravel())
    full = _py_brute(coords, types, L, rcut, [10 ** 6] * len(sel))
    out = []
    for i, c in enumerate(full):
        def key(e):
            _, j, nx, ny, nz = e
            d = [(x[j, a] + n * L) - x[i, a] for a, n in enumerate((nx, ny, nz))]
            return ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2], j, nx, ny, nz)
        keep = []
        for t in range(len(sel)):
            keep += sorted(sorted((e for e in c if e[0] == t), key=key)[:sel[t]])
        out.append(keep)
    return out


@pytest.mark.parametrize("kind", ["water8", "cu_perfect"])
def test_nearest_truncation_matches_python_selection(kind):
    # water: 8 molecules in a 6.2 A box (several images of one j); copper: a perfect 2x2x2 FCC
    # lattice, where whole shells sit at equal distances and the cut falls inside a shell, so
    # the (j, image) tie-break decides
    if kind == "water8":
        s, w, rc, sel = synth.water_box(8, 3), synth.water_weights(), 6.0, (9, 17)
    else:
        s, w, rc, sel = synth.copper_fcc(2, 0, sigma=0.0), synth.copper_weights(), 6.0, (30,)
    m = oracle.Model(w.to_blob())
    L = s.box[0]
    ref = _py_nearest(s.coords, s.types, L, rc, sel)
    full = _py_brute(s.coords, s.types, L, rc, [10 ** 6] * len(sel))
    assert all(sum(1 for e in c if e[0] == t) > sel[t] for c in full for t in range(len(sel)))  # every row truncates
    m.set_truncation(True)
    for method in ("brute", "cell"):
        nl, im, cnt, ovf = m.nlist(s.coords, s.types, s.box, method, rcut=rc, sel=sel)
        assert not ovf
        assert _rows(nl, im, s.types, sel) == ref
        assert (cnt == np.array(sel)[None, :]).all()
    if kind == "cu_perfect":  # the third shell (24 at a sqrt(3/2)) is split: ties were broken
        x = oracle.wrap(s.coords, s.box)
        r2 = [sorted(((x[j] + np.array(n) * L - x[0]) ** 2).sum() for _, j, *n in full[0])]
        assert np.isclose(r2[0][sel[0] - 1], r2[0][sel[0]])


def test_nearest_truncation_is_identity_without_overflow():
    s = synth.water_box(64, 0)
    m = oracle.Model(synth.water_weights().to_blob())
    a = m.nlist(s.coords, s.types, s.box, "cell")
    m.set_truncation(True)
    b = m.nlist(s.coords, s.types, s.box, "cell")
    assert not a[3] and not b[3]
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    e0 = oracle.Model(synth.water_weights().to_blob()).compute(s.coords, s.types, s.box)["energy"]
    assert m.compute(s.coords, s.types, s.box)["energy"] == e0


def _truncating_water():
    # sel (20, 40) against about 30 O and 60 H neighbours within 6 A: every atom truncates
    w = synth.xavier_weights(("O", "H"), 6.0, 0.5, (20, 40), 1001)
    m = oracle.Model(w.to_blob())
    m.set_truncation(True)
    return m


def test_nearest_truncation_md_filter_equals_cell_list():
    # the MD path keeps the nearest entries of the (r_c + skin) list; the force path of a
    # fresh cell list must give the same energy and forces at step 0
    s = synth.water_box(64, 0)
    m = _truncating_water()
    ref = m.compute(s.coords, s.types, s.box)
    md = m.md(s.coords, np.zeros_like(s.coords), s.types, s.box, s.masses(), 0.5, 0)
    assert abs(md["pe"][0] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    np.testing.assert_allclose(md["forces"], ref["forces"], rtol=0, atol=1e-12)


def test_nearest_truncation_forces_are_energy_gradient():
    # away from a change of the kept set, E stays smooth: central differences of E match -F
    s = synth.water_box(64, 0)
    m = _truncating_water()
    ref = m.compute(s.coords, s.types, s.box)
    h = 1e-5
    rng = np.random.default_rng(3)
    for k in rng.choice(len(s.types), 6, replace=False):
        for c in range(3):
            xp = s.coords.copy()
            xm = s.coords.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = -(m.compute(xp, s.types, s.box, forces=False)["energy"]
                   - m.compute(xm, s.types, s.box, forces=False)["energy"]) / (2 * h)
            assert abs(fd - ref["forces"][k, c]) <= 1e-6 + 1e-5 * abs(fd)


# ----------------------------------------------------------------- triclinic cells
def _sheared(s, tilt=((0.3, 0.0), (-0.2, 0.25))):
    """The cubic system s mapped by fractional coordinates into the sheared cell
    H = L [[1, 0, 0], [t10, 1, 0], [t20, t21, 1]] (same volume, distances distorted)."""
    L = s.box[0]
    H = L * np.array([[1.0, 0.0, 0.0], [tilt[0][0], 1.0, 0.0], [tilt[1][0], tilt[1][1], 1.0]])
    x = (s.coords / L) @ H
    return x, H.ravel()


def _py_brute_tri(coords, types, H, rcut):
    """Independent Python brute force in a general cell: every (j, n) with
    d = (x_j + ((n0 H0 + n1 H1) + n2 H2)) - x_i of r^2 < rcut^2, from the oracle's wrapped
    positions, in canonical order."""
    x = oracle.wrap(coords, H.ravel())
    Hm = H.reshape(3, 3)
    V = np.linalg.det(Hm)
    w = [V / np.linalg.norm(np.cross(Hm[(a + 1) % 3], Hm[(a + 2) % 3])) for a in range(3)]
    nmax = [math.ceil(rcut / wa) + 1 for wa in w]
    out = []
    for i in range(len(types)):
        c = []
        for j in range(len(types)):
            for nx in range(-nmax[0], nmax[0] + 1):
                for ny in range(-nmax[1], nmax[1] + 1):
                    for nz in range(-nmax[2], nmax[2] + 1):
                        if i == j and nx == ny == nz == 0:
                            continue
                        d = [(x[j, a] + ((nx * Hm[0, a] + ny * Hm[1, a]) + nz * Hm[2, a])) - x[i, a] for a in range(3)]
                        if (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] < rcut * rcut:
                            c.append((int(types[j]), j, nx, ny, nz))
        out.append(sorted(c))
    return out


def test_triclinic_nlist_matches_python_brute_force():
    s = synth.water_box(8, 3)  # a 6.2 A cell: several images of one j within 6 A
    x, H = _sheared(s)
    m = oracle.Model(synth.water_weights().to_blob())
    sel = (400, 800)
    ref = _py_brute_tri(x, s.types, H, 6.0)
    for method in ("brute", "cell"):
        nl, im, cnt, ovf = m.nlist(x, s.types, H, method, rcut=6.0, sel=sel)
        assert not ovf
        assert _rows(nl, im, s.types, sel) == ref


def test_triclinic_cell_list_equals_brute():
    s = synth.water_box(64, 0)
    x, H = _sheared(s, ((0.45, 0.0), (-0.3, 0.35)))
    m = oracle.Model(synth.water_weights().to_blob())
    a = m.nlist(x, s.types, H, "brute")
    b = m.nlist(x, s.types, H, "cell")
    assert not a[3] and not b[3]
    for p, q in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(p, q)


def test_triclinic_cell_of_a_cubic_lattice_gives_the_cubic_result():
    # rows (a, a + b, b + c) span the same lattice as the cube: the same periodic system
    s = synth.water_box(64, 0)
    L = s.box[0]
    H = np.array([[L, 0, 0], [L, L, 0], [0, L, L]], dtype=np.float64).ravel()
    m = oracle.Model(synth.water_weights().to_blob())
    ref = m.compute(s.coords, s.types, s.box)
    got = m.compute(s.coords, s.types, H)
    assert got["energy"] == pytest.approx(ref["energy"], rel=1e-12)
    np.testing.assert_allclose(got["forces"], ref["forces"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(got["virial"], ref["virial"], rtol=0, atol=1e-10)


def test_triclinic_rotation_invariance():
    s = synth.water_box(64, 0)
    x, H = _sheared(s)
    m = oracle.Model(synth.water_weights().to_blob())
    ref = m.compute(x, s.types, H)
    R = synth._rand_rotation(np.random.default_rng(11))
    got = m.compute(x @ R.T, s.types, (H.reshape(3, 3) @ R.T).ravel())
    assert got["energy"] == pytest.approx(ref["energy"], rel=1e-12)
    np.testing.assert_allclose(got["forces"], ref["forces"] @ R.T, rtol=0, atol=1e-11)
    np.testing.assert_allclose(got["virial"], R @ ref["virial"] @ R.T, rtol=0, atol=1e-10)


def test_triclinic_forces_and_virial_are_derivatives():
    s = synth.water_box(64, 0)
    x, H = _sheared(s)
    m = oracle.Model(synth.water_weights().to_blob())
    ref = m.compute(x, s.types, H)
    # forces: the exact directional derivative (dual numbers) along a random displacement
    w = np.random.default_rng(5).standard_normal(x.shape)
    E, dE = m.dir_deriv(x, s.types, H, w)
    assert E == pytest.approx(ref["energy"], rel=1e-13)
    assert dE == pytest.approx(-(w * ref["forces"]).sum(), rel=1e-11, abs=1e-14)
    # every virial component: x -> x (I + e E_ab), H -> H (I + e E_ab) gives -dE/de = V_ba
    # (central differences at e and 2e, Richardson-extrapolated: error O(e^4))
    eps = 1e-3
    Hm = H.reshape(3, 3)
    for a in range(3):
        for b in range(3):
            def E_at(e):
                S = np.eye(3)
                S[a, b] += e
                return m.energy(x @ S, s.types, (Hm @ S).ravel())
            d1 = (E_at(eps) - E_at(-eps)) / (2 * eps)
            d2 = (E_at(2 * eps) - E_at(-2 * eps)) / (4 * eps)
            fd = -(4 * d1 - d2) / 3
            assert fd == pytest.approx(ref["virial"][b, a], rel=1e-6, abs=1e-9)


def test_triclinic_md_filter_equals_cell_list():
    s = synth.water_box(64, 0)
    x, H = _sheared(s)
    m = oracle.Model(synth.water_weights().to_blob())
    ref = m.compute(x, s.types, H)
    md = m.md(x, np.zeros_like(x), s.types, H, s.masses(), 0.5, 0)
    assert abs(md["pe"][0] - ref["energy"]) <= 1e-12 * abs(ref["energy"])


def test_left_handed_or_flat_cell_is_rejected():
    s = synth.water_box(8, 3)
    m = oracle.Model(synth.water_weights().to_blob())
    L = s.box[0]
    for H in (np.diag([L, L, -L]).ravel(), np.array([[L, 0, 0], [L, 0, 0], [0, 0, L]], dtype=np.float64).ravel()):
        with pytest.raises(oracle.OracleError):
            m.compute(s.coords, s.types, H)


# ----------------------------------------------------------------- forces / virial
def test_forces_match_central_differences(water_oracle, water64):
    s = water64
    ref = water_oracle.compute(s.coords, s.types, s.box)
    rng = np.random.default_rng(11)
    # forces of the random model are ~1e-4 eV/A against E ~ 400 eV, so the step is
    # chosen where rounding of E (~1e-13) and the h^2 truncation are both < 1e-6 F
    h = 1e-4
    for i in rng.choice(s.natoms, 4, replace=False):
        for a in range(3):
            xp = s.coords.copy(); xp[i, a] += h
            xm = s.coords.copy(); xm[i, a] -= h
            fd = -(water_oracle.energy(xp, s.types, s.box) - water_oracle.energy(xm, s.types, s.box)) / (2 * h)
            f = ref["forces"][i, a]
            assert abs(fd - f) <= 1e-5 * abs(f) + 2e-10, (i, a, fd, f)


def test_forces_match_dual_directional_derivative(water_oracle, water64):
    s = water64
    ref = water_oracle.compute(s.coords, s.types, s.box)
    w = np.random.default_rng(3).standard_normal(s.coords.shape)
    E, dE = water_oracle.dir_deriv(s.coords, s.types, s.box, w)
    assert E == pytest.approx(ref["energy"], rel=1e-13)
    lhs = -(w * ref["forces"]).sum()
    assert dE == pytest.approx(lhs, rel=1e-11, abs=1e-14)


def test_virial_matches_strain_derivative_periodic(water_oracle, water64):
    s = water64
    ref = water_oracle.compute(s.coords, s.types, s.box)
    V = ref["virial"]
    eps = 1e-4
    for a in range(3):
        def E_at(e):
            sc = np.ones(3); sc[a] += e
            box = np.diag(np.diag(s.box.reshape(3, 3)) * sc).ravel()
            return water_oracle.energy(s.coords * sc, s.types, box)
        fd = -(E_at(eps) - E_at(-eps)) / (2 * eps)
        assert fd == pytest.approx(V[a, a], rel=1e-5, abs=1e-9)


def _cluster(seed=4, n_mol=6, L=80.0):
    s = synth.water_box(n_mol, seed)
    c = s.coords - s.coords.mean(0) + L / 2
    return c, s.types, np.diag([L, L, L]).ravel()


def test_virial_free_cluster_all_components(water_oracle):
    c, t, box = _cluster()
    ref = water_oracle.compute(c, t, box)
    V, F = ref["virial"], ref["forces"]
    centre = c.mean(0)
    # virial of an isolated cluster equals sum_k F_k x_k^T (translation invariant)
    np.testing.assert_allclose(V, F.T @ (c - centre), rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(V, V.T, rtol=1e-10, atol=1e-14)
    eps = 1e-4
    for a in range(3):
        for b in range(3):
            def E_at(e):
                S = np.eye(3); S[a, b] += e
                return water_oracle.energy((c - centre) @ S.T + centre, t, box)
            fd = -(E_at(eps) - E_at(-eps)) / (2 * eps)
            assert fd == pytest.approx(V[a, b], rel=1e-5, abs=1e-10)


def test_virial_symmetric_and_force_sum_zero(water_oracle, water64):
    s = water64
    ref = water_oracle.compute(s.coords, s.types, s.box)
    V, F = ref["virial"], ref["forces"]
    scale = np.abs(V).max()
    assert np.abs(V - V.T).max() <= 1e-12 * scale
    assert np.abs(F.sum(0)).max() <= 1e-12 * np.abs(F).max() * s.natoms


# ----------------------------------------------------------------- invariances
def test_energy_invariances_periodic(water_oracle, water64):
    s = water64
    L = s.box[0]
    E0 = water_oracle.compute(s.coords, s.types, s.box)
    e0 = E0["energy"]
    # translation
    et = water_oracle.energy(s.coords + np.array([1.37, -4.1, 7.9]), s.types, s.box)
    assert et == pytest.approx(e0, rel=1e-12)
    # 90-degree rotation about z is a symmetry of the cube
    er = _rot90_z(s.coords, L)
    Er = water_oracle.compute(er, s.types, s.box)
    assert Er["energy"] == pytest.approx(e0, rel=1e-12)
    np.testing.assert_allclose(Er["atom_energy"], E0["atom_energy"], rtol=1e-11, atol=1e-12)
    # the rotated forces are the rotated forces
    Fr = np.stack([-E0["forces"][:, 1], E0["forces"][:, 0], E0["forces"][:, 2]], 1)
    np.testing.assert_allclose(Er["forces"], Fr, rtol=1e-9, atol=1e-13)
    # same-type permutation
    perm = np.arange(s.natoms)
    O = np.where(s.types == 0)[0]
    H = np.where(s.types == 1)[0]
    rng = np.random.default_rng(5)
    perm[O] = rng.permutation(O)
    perm[H] = rng.permutation(H)
    Ep = water_oracle.compute(s.coords[perm], s.types[perm], s.box)
    assert Ep["energy"] == pytest.approx(e0, rel=1e-12)
    np.testing.assert_allclose(Ep["atom_energy"], E0["atom_energy"][perm], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(Ep["forces"], E0["forces"][perm], rtol=1e-9, atol=1e-13)


def test_energy_invariant_under_random_rotation_free_cluster(water_oracle):
    c, t, box = _cluster()
    e0 = water_oracle.energy(c, t, box)
    R = synth._rand_rotation(np.random.default_rng(9))
    centre = c.mean(0)
    e1 = water_oracle.energy((c - centre) @ R.T + centre, t, box)
    assert e1 == pytest.approx(e0, rel=1e-12)


def test_type_swap_changes_energy(water_oracle, water64):
    # a guard that the tests above can fail: permuting across types changes E
    s = water64
    t2 = s.types.copy()
    t2[0], t2[1] = t2[1], t2[0]
    assert abs(water_oracle.energy(s.coords, t2, s.box) - water_oracle.energy(s.coords, s.types, s.box)) > 1e-5


# ----------------------------------------------------------------- switch continuity
@pytest.mark.parametrize("kind", [0, 1])
def test_switch_c1_across_rs_and_rc(kind):
    w = synth.xavier_weights(("O", "H"), 6.0, 0.5, (46, 92), 1001, switch_kind=kind)
    m = oracle.Model(w.to_blob())
    L = 60.0
    box = np.diag([L, L, L]).ravel()
    t = np.array([0, 1], np.int32)
    for r0 in (0.5, 6.0):
        for side in (-1, 1):
            r = r0 + side * 1e-4
            x = np.array([[20.0, 20.0, 20.0], [20.0 + r, 20.0, 20.0]])
            res = m.compute(x, t, box)
            # force on atom 1 equals -dE/dr; compare to a finite difference on that side
            h = 1e-6
            xp = x.copy(); xp[1, 0] += h
            xm = x.copy(); xm[1, 0] -= h
            fd = -(m.energy(xp, t, box) - m.energy(xm, t, box)) / (2 * h)
            assert fd == pytest.approx(res["forces"][1, 0], rel=1e-5, abs=1e-10)
        # value and slope continuity across the knot
        ea = m.compute(np.array([[20.0, 20, 20], [20.0 + r0 - 1e-7, 20, 20]]), t, box)
        eb = m.compute(np.array([[20.0, 20, 20], [20.0 + r0 + 1e-7, 20, 20]]), t, box)
        assert ea["energy"] == pytest.approx(eb["energy"], abs=1e-7)
        assert ea["forces"][1, 0] == pytest.approx(eb["forces"][1, 0], abs=1e-5)
    # beyond r_c the pair does not interact: E equals the sum of two isolated atoms
    far = m.compute(np.array([[20.0, 20, 20], [20.0 + 6.5, 20, 20]]), t, box)
    assert np.abs(far["forces"]).max() == 0.0


# ----------------------------------------------------------------- closed forms
def _sparse_weights(switch_kind=0, davg=None, dstd=None):
    """Water-sized model with almost all parameters zero, so the energy of a dimer
    has a short closed form that exercises every index of the definition."""
    w = synth.xavier_weights(("O", "H"), 6.0, 0.5, (46, 92), 7, switch_kind=switch_kind)
    w.theta[:] = 0.0
    rng = np.random.default_rng(2024)
    for ti in range(2):
        for tj in range(2):
            p = f"emb{ti}{tj}."
            w.block(p + "W1")[:] = rng.normal(0, 0.8, (1, 25))
            w.block(p + "b1")[:] = rng.normal(0, 0.5, 25)
            w.block(p + "b2")[:] = rng.normal(0, 0.5, 50)
            w.block(p + "b3")[:] = rng.normal(0, 0.5, 100)
            w.block(p + "W2")[3, 7] = 0.9 + 0.1 * ti + 0.05 * tj
            w.block(p + "W3")[5, 60] = -1.1 + 0.1 * tj
    for t in range(2):
        p = f"fit{t}."
        W1 = w.block(p + "W1")
        W1[37 * 16 + 5, 11] = 3.0 + t
        W1[2 * 16 + 9, 11] = -2.0
        W1[60 * 16 + 3, 4] = 1.5
        w.block(p + "b1")[:] = rng.normal(0, 0.3, 240)
        w.block(p + "W2")[11, 20] = 0.7
        w.block(p + "b2")[:] = rng.normal(0, 0.3, 240)
        w.block(p + "W3")[20, 30] = -0.6
        w.block(p + "b3")[:] = rng.normal(0, 0.3, 240)
        w.block(p + "w4")[:] = rng.normal(0, 0.2, 240)
        w.block(p + "b4")[:] = 0.3 - t
    w.block("e_bias")[:] = [0.25, -0.5]
    if davg is not None:
        w.davg[:] = davg
    if dstd is not None:
        w.dstd[:] = dstd
    return w


def _sparse_G(w, ti, tj, x):
    """Embedding output G of pair (ti, tj) for input x with the sparse weights above,
    written out scalar by scalar."""
    p = f"emb{ti}{tj}."
    W1, b1, b2, b3 = (w.block(p + k) for k in ("W1", "b1", "b2", "b3"))
    h1 = np.tanh(x * W1[0] + b1)
    h2 = np.concatenate([h1, h1]) + np.tanh(b2)
    h2[7] = h1[7] + math.tanh(h1[3] * w.block(p + "W2")[3, 7] + b2[7])
    G = np.concatenate([h2, h2]) + np.tanh(b3)
    G[60] = h2[10] + math.tanh(h2[5] * w.block(p + "W3")[5, 60] + b3[60])
    return G


def _closed_form_dimer(w, r, u, ti, tj):
    """E_i of atom i (type ti) whose only neighbour (type tj) sits at r*u, with the
    sparse weights above, written out scalar by scalar.  Every one of the S = 46 + 92
    slots enters T: the neighbour's row (when r < r_c) and the padded slots, whose
    un-normalised row is zero, so R_hat = -davg/dstd with G of that input."""
    rs, rc = w.rcut_smth, w.rcut
    if r < rs:
        sw = 1.0
    elif r >= rc:
        sw = 0.0
    else:
        x = (r - rs) / (rc - rs)
        sw = x ** 3 * (-6 * x * x + 15 * x - 10) + 1 if w.switch_kind == 0 else 0.5 * math.cos(math.pi * x) + 0.5
    s = sw / r
    Rt = np.array([s, s * u[0], s * u[1], s * u[2]])
    Rh = (Rt - w.davg[ti]) / w.dstd[ti]
    Rp = (0.0 - w.davg[ti]) / w.dstd[ti]
    S = 138.0
    npad = [46, 92]
    T = np.zeros((4, 100))
    if r < rc:
        T += np.outer(Rh, _sparse_G(w, ti, tj, Rh[0]))
        npad[tj] -= 1
    for t in (0, 1):
        T += npad[t] * np.outer(Rp, _sparse_G(w, ti, t, Rp[0]))
    T /= S
    D = lambda a, b: float(T[:, a] @ T[:, b])  # noqa: E731
    f = f"fit{ti}."
    W1f, b1f, b2f, b3f, w4, b4 = (w.block(f + k) for k in ("W1", "b1", "b2", "b3", "w4", "b4"))
    h1f = np.tanh(b1f)
    h1f[11] = math.tanh(W1f[37 * 16 + 5, 11] * D(37, 5) + W1f[2 * 16 + 9, 11] * D(2, 9) + b1f[11])
    h1f[4] = math.tanh(W1f[60 * 16 + 3, 4] * D(60, 3) + b1f[4])
    t2 = np.tanh(b2f)
    t2[20] = math.tanh(w.block(f + "W2")[11, 20] * h1f[11] + b2f[20])
    h2f = h1f + t2
    t3 = np.tanh(b3f)
    t3[30] = math.tanh(w.block(f + "W3")[20, 30] * h2f[20] + b3f[30])
    h3f = h2f + t3
    return float(h3f @ w4 + b4[0] + w.block("e_bias")[ti])


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("r", [0.3, 1.7, 4.2, 5.99, 7.0])
def test_dimer_energy_closed_form(kind, r):
    w = _sparse_weights(kind)
    m = oracle.Model(w.to_blob())
    L = 50.0
    box = np.diag([L, L, L]).ravel()
    u = np.array([2.0, -1.0, 0.5]); u /= np.linalg.norm(u)
    x = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0] + r * u])
    t = np.array([0, 1], np.int32)
    res = m.compute(x, t, box)
    e0 = _closed_form_dimer(w, r, u, 0, 1)
    e1 = _closed_form_dimer(w, r, -u, 1, 0)
    assert res["atom_energy"][0] == pytest.approx(e0, rel=1e-13, abs=1e-14)
    assert res["atom_energy"][1] == pytest.approx(e1, rel=1e-13, abs=1e-14)


def test_dimer_closed_form_with_normalisation():
    davg = np.array([[0.05, 0.01, -0.02, 0.03], [0.1, 0.0, 0.0, 0.0]])
    dstd = np.array([[0.7, 1.3, 0.9, 1.1], [2.0, 0.5, 0.6, 0.8]])
    w = _sparse_weights(0, davg, dstd)
    m = oracle.Model(w.to_blob())
    box = np.diag([50.0] * 3).ravel()
    u = np.array([0.3, 0.9, -0.2]); u /= np.linalg.norm(u)
    for r in (1.1, 3.3):
        x = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0] + r * u])
        res = m.compute(x, np.array([0, 1], np.int32), box)
        assert res["atom_energy"][0] == pytest.approx(_closed_form_dimer(w, r, u, 0, 1), rel=1e-13)
        assert res["atom_energy"][1] == pytest.approx(_closed_form_dimer(w, r, -u, 1, 0), rel=1e-13)


def test_dimer_closed_form_normalised_across_cutoff():
    # With davg != 0 the padded slots carry R_hat = -davg/dstd; the dimer's energy follows the
    # closed form on both sides of r_c, including r > r_c where every slot is padded.
    davg = np.array([[0.08, 0.01, -0.02, 0.03], [0.12, 0.0, 0.0, 0.0]])
    dstd = np.array([[0.15, 0.09, 0.08, 0.1], [0.13, 0.07, 0.06, 0.08]])
    w = _sparse_weights(0, davg, dstd)
    m = oracle.Model(w.to_blob())
    box = np.diag([50.0] * 3).ravel()
    u = np.array([-0.4, 0.2, 0.7]); u /= np.linalg.norm(u)
    for r in (0.4, 2.5, 5.5, 6.5):
        x = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0] + r * u])
        res = m.compute(x, np.array([0, 1], np.int32), box)
        assert res["atom_energy"][0] == pytest.approx(_closed_form_dimer(w, r, u, 0, 1), rel=1e-13)
        assert res["atom_energy"][1] == pytest.approx(_closed_form_dimer(w, r, -u, 1, 0), rel=1e-13)


@pytest.mark.parametrize("kind", [0, 1])
def test_normalised_energy_continuous_at_cutoff(kind):
    # A padded slot is the row of a neighbour at r_c, so E and dE/dr are continuous as a
    # neighbour leaves the cutoff.  A zero padded row (after normalisation) would make E
    # jump there by (1/S) R_hat_pad^T G(R_hat_pad) through the fitting net.
    w = synth.with_statistics(synth.xavier_weights(("O", "H"), 6.0, 0.5, (46, 92), 1001, switch_kind=kind,
                                                   fit_gain=10.0),
                              [[0.05, 0.0, 0.0, 0.0], [0.05, 0.0, 0.0, 0.0]],
                              [[0.14, 0.09, 0.09, 0.09], [0.13, 0.08, 0.08, 0.08]])
    m = oracle.Model(w.to_blob())
    box = np.diag([60.0] * 3).ravel()
    t = np.array([0, 1], np.int32)
    e = {}
    for side in (-1, 1):
        x = np.array([[20.0, 20.0, 20.0], [20.0 + 6.0 + side * 1e-7, 20.0, 20.0]])
        e[side] = m.compute(x, t, box)
    assert e[-1]["energy"] == pytest.approx(e[1]["energy"], abs=1e-9)
    assert abs(e[-1]["forces"][1, 0]) < 1e-6 and e[1]["forces"][1, 0] == 0.0
    # and the padded rows do change E: the isolated-atom energy differs from davg = 0
    w0 = synth.with_statistics(w, np.zeros((2, 4)), w.dstd)
    e0 = oracle.Model(w0.to_blob()).compute(np.array([[20.0, 20, 20], [40.0, 40, 40]]), t, box)["energy"]
    e1 = m.compute(np.array([[20.0, 20, 20], [40.0, 40, 40]]), t, box)["energy"]
    assert abs(e1 - e0) > 1e-3


def test_env_stats_closed_form():
    # An O-H pair inside r_s (sw = 1, s = 1/r) and one at r_s < r < r_c with the quintic
    # switch, far from each other, plus an isolated H, in a 60 A box.
    w = synth.water_weights()
    m = oracle.Model(w.to_blob())
    box = np.diag([60.0] * 3).ravel()
    r1, r2 = 0.45, 3.1
    u = np.array([1.0, 2.0, -2.0]) / 3.0
    x = np.array([[5.0, 5, 5], [5.0, 5, 5] + r1 * u, [30.0, 30, 30], [30.0, 30, 30] + r2 * u, [50.0, 10, 50]])
    t = np.array([0, 1, 0, 1, 1], np.int32)
    out = m.env_stats(x, t, box)
    xq = (r2 - 0.5) / 5.5
    s2 = (xq ** 3 * (-6 * xq * xq + 15 * xq - 10) + 1) / r2
    s1 = 1.0 / r1
    for ti, nat in ((0, 2), (1, 3)):
        assert out[ti, 0] == 138 * nat and out[ti, 4] == nat
        assert out[ti, 1] == pytest.approx(s1 + s2, rel=1e-14)
        assert out[ti, 2] == pytest.approx(s1 * s1 + s2 * s2, rel=1e-14)
        assert out[ti, 3] == pytest.approx(s1 * s1 + s2 * s2, rel=1e-13)  # |u| = 1


def _normalised_water():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "env_stats.json")) as f:
        return synth.normalised_weights("water", json.load(f))


def test_normalised_model_forces_match_central_differences():
    w = _normalised_water()
    m = oracle.Model(w.to_blob())
    s = synth.water_box(16, 4)
    r = m.compute(s.coords, s.types, s.box)
    assert np.sqrt((r["forces"] ** 2).mean()) > 0.1  # a force scale like a trained model's
    rng = np.random.default_rng(3)
    h = 1e-5
    for i in rng.choice(s.natoms, 6, replace=False):
        for a in range(3):
            xp = s.coords.copy(); xp[i, a] += h
            xm = s.coords.copy(); xm[i, a] -= h
            fd = -(m.energy(xp, s.types, s.box) - m.energy(xm, s.types, s.box)) / (2 * h)
            assert fd == pytest.approx(r["forces"][i, a], rel=1e-6, abs=1e-8)
    # virial against the strain derivative
    eps = 1e-6
    def E_strain(e):
        return m.energy(s.coords * (1 + e), s.types, s.box * (1 + e))
    dE = (E_strain(eps) - E_strain(-eps)) / (2 * eps)
    assert -dE == pytest.approx(np.trace(r["virial"]), rel=1e-6)


def test_normalised_param_grad_dual_matches_finite_differences():
    # The padded slots' G depends on the embedding parameters: the dual-number gradient
    # must carry that term as the finite differences do.
    w = _normalised_water()
    s = synth.water_box(8, 12)
    m = oracle.Model(w.to_blob())
    E0, F0 = 0.9 * m.energy(s.coords, s.types, s.box), np.zeros((s.natoms, 3))
    layout, _ = synth.theta_layout(2)
    off = {name: o for name, _, o in layout}
    idx = [off["emb01.b1"] + 3, off["emb10.W3"] + 17, off["emb11.b3"] + 42, off["emb00.W1"] + 5,
           off["fit0.W1"] + 1234]
    g, dE, loss = m.param_grad(s.coords, s.types, s.box, E0, F0, idx)
    h = 1e-4

    def L_at(p, e):
        th = w.theta.copy(); th[p] += e
        w2 = synth.Weights(w.ntypes, w.type_names, w.rcut, w.rcut_smth, w.sel, th, w.davg, w.dstd)
        r = oracle.Model(w2.to_blob()).compute(s.coords, s.types, s.box)
        return (r["energy"] - E0) ** 2 + ((r["forces"] - F0) ** 2).sum()

    for p, gp in zip(idx, g):
        fd = (8 * (L_at(p, h) - L_at(p, -h)) - (L_at(p, 2 * h) - L_at(p, -2 * h))) / (12 * h)
        assert fd == pytest.approx(gp, rel=1e-5, abs=1e-8), p


def test_isolated_atom_energy_is_fit_of_zero():
    w = _sparse_weights()
    m = oracle.Model(w.to_blob())
    box = np.diag([50.0] * 3).ravel()
    res = m.compute(np.array([[1.0, 2, 3], [30.0, 30, 30]]), np.array([1, 0], np.int32), box)
    for i, t in enumerate((1, 0)):
        f = f"fit{t}."
        h1 = np.tanh(w.block(f + "b1"))
        t2 = np.tanh(w.block(f + "b2"))
        t2[20] = math.tanh(w.block(f + "W2")[11, 20] * h1[11] + w.block(f + "b2")[20])
        h2 = h1 + t2
        t3 = np.tanh(w.block(f + "b3"))
        t3[30] = math.tanh(w.block(f + "W3")[20, 30] * h2[20] + w.block(f + "b3")[30])
        h3 = h2 + t3
        e = h3 @ w.block(f + "w4") + w.block(f + "b4")[0] + w.block("e_bias")[t]
        assert res["atom_energy"][i] == pytest.approx(e, rel=1e-14)
    assert np.abs(res["forces"]).max() == 0.0


# ----------------------------------------------------------------- integrator
def test_verlet_matches_harmonic_oscillator():
    m = np.array([2.0, 15.0])
    k = 0.8  # eV/A^2
    x0 = np.array([[0.3, -0.1, 0.2], [0.05, 0.4, -0.3]])
    v0 = np.array([[0.01, 0.0, -0.02], [0.0, 0.005, 0.001]])
    kappa = synth.ACC_CONV
    T = 200.0
    errs = []
    for dt in (0.5, 0.25):
        n = int(T / dt)
        traj = oracle.md_harmonic(x0, v0, m, k, dt, n)
        w = np.sqrt(k * kappa / m)[:, None]
        t = n * dt
        exact = x0 * np.cos(w * t) + v0 / w * np.sin(w * t)
        errs.append(np.abs(traj[-1] - exact).max())
    assert errs[0] < 1e-3
    # second order: halving dt divides the error by ~4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_oracle_nve_energy_conservation(water_oracle):
    s = synth.water_box(64, 0)
    v = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    r = water_oracle.md(s.coords, v, s.types, s.box, s.masses(), 0.5, 40, rebuild_every=10, skin=2.0)
    etot = r["pe"] + r["ke"]
    assert np.abs(etot - etot[0]).max() < 1e-4 * s.natoms ** 0.5
    # momentum is conserved by the pairwise force construction
    p = (s.masses()[s.types][:, None] * r["v"]).sum(0)
    p0 = (s.masses()[s.types][:, None] * v).sum(0)
    np.testing.assert_allclose(p, p0, atol=1e-10)


# ----------------------------------------------------------------- parameter gradient
def test_param_grad_dual_matches_finite_differences():
    w = synth.water_weights(1001)
    wt = synth.water_weights(2002)
    s = synth.water_box(8, 12)
    m = oracle.Model(w.to_blob())
    mt = oracle.Model(wt.to_blob())
    tgt = mt.compute(s.coords, s.types, s.box)
    E0, F0 = tgt["energy"], tgt["forces"]
    rng = np.random.default_rng(1)
    layout, n = synth.theta_layout(2)
    # a few parameters from every block kind
    idx = []
    for name, shape, off in layout:
        if name.startswith("emb0") or name.startswith("fit1") or name == "e_bias":
            idx.append(off + int(rng.integers(0, int(np.prod(shape)))))
    g, dE, loss = m.param_grad(s.coords, s.types, s.box, E0, F0, idx)
    h = 2e-3  # dE/dtheta ~ 1e-5 against E ~ 50: smaller steps are rounding-bound

    def L_of(theta):
        w2 = synth.Weights(w.ntypes, w.type_names, w.rcut, w.rcut_smth, w.sel, theta, w.davg, w.dstd)
        r = oracle.Model(w2.to_blob()).compute(s.coords, s.types, s.box)
        return (r["energy"] - E0) ** 2 + ((r["forces"] - F0) ** 2).sum()

    def L_at(p, e):
        t = w.theta.copy(); t[p] += e
        return L_of(t)

    for p, gp in zip(idx, g):
        # fourth-order central stencil: truncation ~h^4, rounding ~1e-13 / h
        fd = (8 * (L_at(p, h) - L_at(p, -h)) - (L_at(p, 2 * h) - L_at(p, -2 * h))) / (12 * h)
        assert fd == pytest.approx(gp, rel=1e-5, abs=1e-9), p


# ----------------------------------------------------------------- regression fixture
def test_golden_water64_regression(water_oracle, water64):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "water64_oracle.txt")
    r = water_oracle.compute(water64.coords, water64.types, water64.box, method="brute")
    for line in open(path):
        if line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "energy":
            assert r["energy"] == pytest.approx(float(tok[1]), rel=1e-13)
        elif tok[0] == "atom_energy":
            assert r["atom_energy"][int(tok[1])] == pytest.approx(float(tok[2]), rel=1e-13)
        elif tok[0] == "force":
            np.testing.assert_allclose(r["forces"][int(tok[1])], [float(v) for v in tok[2:]], rtol=1e-10, atol=1e-16)
        elif tok[0] == "virial":
            np.testing.assert_allclose(r["virial"].ravel(), [float(v) for v in tok[1:]], rtol=1e-10, atol=1e-16)


# ----------------------------------------------------------------- tabulated embedding
def _table_range(w):
    """Input range of the tables: from the padded value (a neighbour at r_c) to the input of a
    neighbour at 0.5 A, with a margin."""
    x0 = min(-w.davg[t][0] / w.dstd[t][0] for t in range(w.ntypes)) - 0.05
    x1 = max((2.0 - w.davg[t][0]) / w.dstd[t][0] for t in range(w.ntypes)) + 0.05
    return x0, x1


def test_embedding_jets_match_central_differences():
    # the first and second derivatives that feed the table nodes against differences of G
    w = _normalised_water()
    m = oracle.Model(w.to_blob())
    x = np.array([-0.3, 0.7, 2.9, 6.1])
    h = 1e-4
    g, g1, g2 = m.emb_eval(1, x)
    gp, _, _ = m.emb_eval(1, x + h)
    gm, _, _ = m.emb_eval(1, x - h)
    np.testing.assert_allclose(g1, (gp - gm) / (2 * h), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(g2, (gp - 2 * g + gm) / (h * h), rtol=1e-4, atol=1e-5)


def test_table_reproduces_net_at_nodes_and_is_c2():
    w = _normalised_water()
    m = oracle.Model(w.to_blob())
    x0, x1 = _table_range(w)
    n = 128
    m.tabulate(x0, x1, n)
    step = (x1 - x0) / n
    nodes = x0 + step * np.array([1, 17, 64, 127])
    for pair in range(4):
        g, g1, g2 = m.emb_eval(pair, nodes)
        t, t1, t2 = m.emb_eval(pair, nodes, tabulated=True)
        np.testing.assert_allclose(t, g, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(t1, g1, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(t2, g2, rtol=1e-8, atol=1e-9)
        # value, slope and curvature agree from both sides of a node
        eps = 1e-9 * step
        l, l1, l2 = m.emb_eval(pair, nodes - eps, tabulated=True)
        r, r1, r2 = m.emb_eval(pair, nodes + eps, tabulated=True)
        np.testing.assert_allclose(l, r, atol=1e-11)
        np.testing.assert_allclose(l1, r1, rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(l2, r2, rtol=1e-5, atol=1e-7)


def test_table_error_falls_at_sixth_order():
    # the quintic Hermite interpolant's error is O(h^6): halving the interval divides it by ~64
    w = _normalised_water()
    m = oracle.Model(w.to_blob())
    x0, x1 = _table_range(w)
    xs = np.linspace(x0, x1, 3001)
    g, _, _ = m.emb_eval(2, xs)
    err = []
    for n in (64, 128):
        m.tabulate(x0, x1, n)
        t, _, _ = m.emb_eval(2, xs, tabulated=True)
        err.append(np.abs(t - g).max())
    assert err[0] < 1e-6
    assert 40.0 < err[0] / err[1] < 90.0, err


def test_tabulated_model_forces_and_energy():
    w = _normalised_water()
    m = oracle.Model(w.to_blob())
    s = synth.water_box(16, 4)
    e_net = m.compute(s.coords, s.types, s.box)
    m.tabulate(*_table_range(w), 256)
    r = m.compute(s.coords, s.types, s.box)
    # the table changes E by no more than its interpolation error carried through the descriptor
    assert abs(r["energy"] - e_net["energy"]) / s.natoms < 1e-8
    assert np.abs(r["forces"] - e_net["forces"]).max() < 1e-7
    # forces are the gradient of the tabulated energy
    h = 1e-5
    rng = np.random.default_rng(8)
    for i in rng.choice(s.natoms, 4, replace=False):
        for a in range(3):
            xp = s.coords.copy(); xp[i, a] += h
            xm = s.coords.copy(); xm[i, a] -= h
            fd = -(m.energy(xp, s.types, s.box) - m.energy(xm, s.types, s.box)) / (2 * h)
            assert fd == pytest.approx(r["forces"][i, a], rel=1e-6, abs=1e-8)


# ----------------------------------------------------------------- per-atom virial and RDF
def test_atom_virial_is_strain_derivative_of_atom_energy():
    # E_i depends only on the pair vectors of i's neighbours, so under a homogeneous strain
    # (1 + eps e_ab) the derivative of E_i is -W_i[a][b] with W_i = -sum_j g_ij (x) d_ij
    w = _normalised_water()
    m = oracle.Model(w.to_blob())
    s = synth.water_box(16, 2)
    r = m.compute(s.coords, s.types, s.box, atom_virial=True)
    W = r["atom_virial"]
    np.testing.assert_allclose(W.sum(0), r["virial"], rtol=1e-12, atol=1e-12)
    eps = 1e-6
    for a in range(3):  # normal strain of the periodic box along a
        def Ei(e):
            G = np.eye(3); G[a, a] += e
            return m.compute(s.coords @ G.T, s.types, (s.box.reshape(3, 3) @ G.T).ravel(),
                             forces=False)["atom_energy"]
        dE = (Ei(eps) - Ei(-eps)) / (2 * eps)
        np.testing.assert_allclose(-dE, W[:, a, a], rtol=1e-6, atol=1e-8)
    # off-diagonal: a free cluster (no box constraint), shear strain applied to the coordinates
    L = 60.0
    cl = synth.water_box(4, 5)
    x = cl.coords - cl.coords.mean(0) + L / 2
    box = np.diag([L, L, L]).ravel()
    rc_ = m.compute(x, cl.types, box, atom_virial=True)
    for a, b in ((0, 1), (1, 2), (2, 0)):
        def Ei(e):
            G = np.eye(3); G[a, b] += e
            return m.compute((x - L / 2) @ G.T + L / 2, cl.types, box, forces=False)["atom_energy"]
        dE = (Ei(eps) - Ei(-eps)) / (2 * eps)
        np.testing.assert_allclose(-dE, rc_["atom_virial"][:, a, b], rtol=1e-6, atol=1e-8)


def test_rdf_of_perfect_fcc_counts_the_shells():
    # FCC shells within 8 A (a = 3.634): radii a sqrt(k/2), coordination 12, 6, 24, 12, 24, 8, 48, 6, 36
    c = synth.copper_fcc(6, 0, sigma=0.0)
    w = synth.copper_weights()
    m = oracle.Model(w.to_blob())
    nbins, rmax = 800, 8.0
    counts = m.rdf(c.coords, c.types, c.box, nbins, rmax)[0, 0]
    shells = {1: 12, 2: 6, 3: 24, 4: 12, 5: 24, 6: 8, 7: 48, 8: 6, 9: 36}
    expect = np.zeros(nbins, dtype=np.int64)
    for k, n in shells.items():
        expect[int(3.634 * math.sqrt(k / 2) / (rmax / nbins))] += n * c.natoms
    np.testing.assert_array_equal(counts.astype(np.int64), expect)
