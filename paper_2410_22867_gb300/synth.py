"""Seeded synthetic inputs: water boxes, copper FCC crystals, replica sets,
model weight blobs and initial velocities.

This module only *creates inputs*; it holds none of the Deep Potential
arithmetic (no switch, no environment matrix, no network, no force).  Both the
CUDA library and the FP64 test oracle consume what it writes, so it is the one
piece of code the two sides share.

Workloads follow the systems of the paper's evaluation (Section IV): water with
r_c = 6 A and neighbour caps 46 (O) / 92 (H), copper with r_c = 8 A and cap 512,
a fitting net of (240, 240, 240), time steps 0.5 fs (water) and 1 fs (Cu), skin
2 A.  The trained models and AIMD data of the paper are not available, so
weights are Xavier-initialised from a seed instead.

Weight blob layout (little-endian), shared interface of both readers:

  offset  type        field
  0       char[4]     magic "DPW1"
  4       int32       version (1)
  8       int32       ntypes
  12      int32       switch kind (0 = quintic C2 polynomial, 1 = cosine)
  16      float64     rcut
  24      float64     rcut_smth
  32      int32[3]    embedding widths (25, 50, 100)
  44      int32       axis width M2 (16)
  48      int32[3]    fitting widths (240, 240, 240)
  60      int32       reserved (0)
  64      int32[nt]   sel per neighbour type, padded with zeros to a multiple of 2
  ...     char[nt][8] type names, NUL padded
  ...     float64[]   theta: for ti, for tj: embedding net (W1,b1,W2,b2,W3,b3);
                      for t: fitting net (W1,b1,W2,b2,W3,b3,w4,b4); e_bias[nt]
  ...     float64     davg[nt][4], dstd[nt][4]

Weight matrices are stored row-major as [fan_in][fan_out].
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field

import numpy as np

MASS_AMU = {"O": 15.999, "H": 1.008, "Cu": 63.546}
WATER_G_PER_MOL = 18.015
AVOGADRO_PER_A3 = 0.602214076  # (g/cm^3) / (g/mol) -> molecules per A^3
KB_EV = 8.617333262e-5
# A * fs^-2 per (eV / A / amu)
ACC_CONV = 9.648533e-3

EMB = (25, 50, 100)
AXIS = 16
FIT = (240, 240, 240)


@dataclass
class System:
    coords: np.ndarray            # [N, 3] float64, Angstrom
    types: np.ndarray             # [N] int32
    box: np.ndarray               # [9] float64 row-major, orthorhombic
    type_names: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def natoms(self) -> int:
        return int(self.coords.shape[0])

    def masses(self) -> np.ndarray:
        return np.array([MASS_AMU[n] for n in self.type_names], dtype=np.float64)


def _cubic_box(L: float) -> np.ndarray:
    return np.array([L, 0, 0, 0, L, 0, 0, 0, L], dtype=np.float64)


def _rand_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_box(n_mol: int, seed: int, density: float = 1.0, jitter: float = 0.2,
              noise: float = 0.05) -> System:
    """Periodic cubic water box: O on a jittered cubic lattice, H at 0.9572 A with a
    104.52 degree angle in a uniformly random orientation, Gaussian noise on every atom.
    Atom order is molecule-major (O, H, H); types O=0, H=1."""
    rng = np.random.default_rng(seed)
    L = (n_mol * WATER_G_PER_MOL / (AVOGADRO_PER_A3 * density)) ** (1.0 / 3.0)
    n = 1
    while n ** 3 < n_mol:
        n += 1
    sites = np.array([(a, b, c) for a in range(n) for b in range(n) for c in range(n)], dtype=np.float64)
    if len(sites) > n_mol:
        pick = np.sort(rng.choice(len(sites), size=n_mol, replace=False))
        sites = sites[pick]
    spacing = L / n
    O = (sites + 0.5) * spacing + rng.uniform(-jitter, jitter, size=(n_mol, 3))
    b = 0.9572
    half = math.radians(104.52) / 2.0
    ref = np.array([[b * math.sin(half), b * math.cos(half), 0.0],
                    [-b * math.sin(half), b * math.cos(half), 0.0]])
    coords = np.empty((3 * n_mol, 3))
    for m in range(n_mol):
        R = _rand_rotation(rng)
        coords[3 * m] = O[m]
        coords[3 * m + 1:3 * m + 3] = O[m] + ref @ R.T
    coords += rng.normal(0.0, noise, size=coords.shape)
    types = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    return System(coords, types, _cubic_box(L), ("O", "H"),
                  {"kind": "water", "n_mol": n_mol, "L": L, "seed": seed, "density": density})


def copper_fcc(ncell: int, seed: int, a: float = 3.634, sigma: float = 0.08) -> System:
    """Periodic FCC copper crystal of ncell^3 conventional cells with Gaussian thermal
    displacement sigma per component."""
    rng = np.random.default_rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(ncell, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    coords = ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)
    coords = coords + rng.normal(0.0, sigma, size=coords.shape)
    types = np.zeros(len(coords), dtype=np.int32)
    L = ncell * a
    return System(coords, types, _cubic_box(L), ("Cu",),
                  {"kind": "copper", "ncell": ncell, "L": L, "seed": seed})


def water_replicas(nrep: int, seed: int, lo: int = 32, hi: int = 2048,
                   density_jitter: float = 0.03) -> list[System]:
    """Independent periodic water boxes with molecule counts drawn log-uniformly in
    [lo, hi] and densities jittered uniformly by +-density_jitter."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(lo), math.log(hi), size=nrep))
    counts = np.clip(np.rint(counts).astype(int), lo, hi)
    dens = 1.0 + rng.uniform(-density_jitter, density_jitter, size=nrep)
    seeds = rng.integers(0, 2 ** 31 - 1, size=nrep)
    return [water_box(int(c), int(s), density=float(d)) for c, s, d in zip(counts, seeds, dens)]


def concat(systems: list[System]):
    """CSR-style concatenation of replicas: coords [sum N, 3], types, atom_offsets
    [nrep + 1] int32 and boxes [nrep, 9]."""
    offs = np.zeros(len(systems) + 1, dtype=np.int32)
    offs[1:] = np.cumsum([s.natoms for s in systems])
    coords = np.concatenate([s.coords for s in systems])
    types = np.concatenate([s.types for s in systems]).astype(np.int32)
    boxes = np.stack([s.box for s in systems])
    return coords, types, offs, boxes


def theta_layout(ntypes: int, emb=EMB, axis=AXIS, fit=FIT):
    """Names, shapes and offsets of every parameter block of the flat theta vector,
    in blob order."""
    n1, n2, n3 = emb
    f1, f2, f3 = fit
    blocks = []
    for ti in range(ntypes):
        for tj in range(ntypes):
            p = f"emb{ti}{tj}."
            blocks += [(p + "W1", (1, n1)), (p + "b1", (n1,)), (p + "W2", (n1, n2)), (p + "b2", (n2,)),
                       (p + "W3", (n2, n3)), (p + "b3", (n3,))]
    for t in range(ntypes):
        p = f"fit{t}."
        blocks += [(p + "W1", (n3 * axis, f1)), (p + "b1", (f1,)), (p + "W2", (f1, f2)), (p + "b2", (f2,)),
                   (p + "W3", (f2, f3)), (p + "b3", (f3,)), (p + "w4", (f3,)), (p + "b4", (1,))]
    blocks += [("e_bias", (ntypes,))]
    out, off = [], 0
    for name, shape in blocks:
        n = int(np.prod(shape))
        out.append((name, shape, off))
        off += n
    return out, off


@dataclass
class Weights:
    ntypes: int
    type_names: tuple
    rcut: float
    rcut_smth: float
    sel: tuple
    theta: np.ndarray
    davg: np.ndarray  # [nt, 4]
    dstd: np.ndarray  # [nt, 4]
    switch_kind: int = 0

    def block(self, name: str) -> np.ndarray:
        for n, shape, off in theta_layout(self.ntypes)[0]:
            if n == name:
                return self.theta[off:off + int(np.prod(shape))].reshape(shape)
        raise KeyError(name)

    def to_blob(self) -> bytes:
        nt = self.ntypes
        head = struct.pack("<4si i i d d 3i i 3i i", b"DPW1", 1, nt, self.switch_kind,
                           float(self.rcut), float(self.rcut_smth), *EMB, AXIS, *FIT, 0)
        assert len(head) == 64
        sel = list(self.sel) + [0] * (nt % 2)
        head += struct.pack(f"<{len(sel)}i", *sel)
        for name in self.type_names:
            head += name.encode()[:7].ljust(8, b"\0")
        body = np.ascontiguousarray(self.theta, dtype="<f8").tobytes()
        body += np.ascontiguousarray(self.davg, dtype="<f8").tobytes()
        body += np.ascontiguousarray(self.dstd, dtype="<f8").tobytes()
        return head + body


def xavier_weights(type_names, rcut: float, rcut_smth: float, sel, seed: int,
                   switch_kind: int = 0, fit_gain: float = 1.0) -> Weights:
    """Xavier-normal weights W ~ N(0, 2/(fan_in + fan_out)), biases ~ N(0, 1), e_bias = 0,
    davg = 0, dstd = 1 (random weights come with no training statistics).  fit_gain
    multiplies the fitting nets' first-layer weights (their standard deviation) after
    the draw; the draw itself does not depend on it."""
    nt = len(type_names)
    rng = np.random.default_rng(seed)
    layout, total = theta_layout(nt)
    theta = np.zeros(total)
    for name, shape, off in layout:
        n = int(np.prod(shape))
        leaf = name.split(".")[-1]
        if name == "e_bias":
            vals = np.zeros(n)
        elif leaf.startswith("W") or leaf == "w4":
            fan_in, fan_out = (shape[0], shape[1]) if len(shape) == 2 else (shape[0], 1)
            vals = rng.normal(0.0, math.sqrt(2.0 / (fan_in + fan_out)), size=n)
        else:
            vals = rng.normal(0.0, 1.0, size=n)
        if leaf == "W1" and name.startswith("fit"):
            vals = vals * fit_gain
        theta[off:off + n] = vals
    davg = np.zeros((nt, 4))
    dstd = np.ones((nt, 4))
    return Weights(nt, tuple(type_names), rcut, rcut_smth, tuple(int(s) for s in sel), theta,
                   davg, dstd, switch_kind)


def water_weights(seed: int = 1001) -> Weights:
    return xavier_weights(("O", "H"), 6.0, 0.5, (46, 92), seed)


def copper_weights(seed: int = 1001) -> Weights:
    return xavier_weights(("Cu",), 8.0, 2.0, (512,), seed)


def with_statistics(w: Weights, davg, dstd) -> Weights:
    """A copy of w whose input normalisation is (davg, dstd), each [ntypes][4]."""
    davg = np.array(davg, dtype=np.float64).reshape(w.ntypes, 4)
    dstd = np.array(dstd, dtype=np.float64).reshape(w.ntypes, 4)
    return Weights(w.ntypes, w.type_names, w.rcut, w.rcut_smth, w.sel, w.theta.copy(), davg, dstd,
                   w.switch_kind)


# Gain on the fitting nets' first layer of the normalised test models: with the
# environment statistics in place it brings the forces of the water model to the scale
# of a trained one (about 0.6 eV/A rms at 300 K) with the first-layer tanh unsaturated.
NORMALISED_FIT_GAIN = 10.0


def normalised_weights(kind: str, stats: dict, seed: int = 1001) -> Weights:
    """The water ("water") or copper ("copper") model with its per-type environment
    statistics stats[kind]["davg"], stats[kind]["dstd"] (as written by the oracle script
    tests/golden/make_env_stats.py) and NORMALISED_FIT_GAIN on the fitting input layer."""
    if kind == "water":
        w = xavier_weights(("O", "H"), 6.0, 0.5, (46, 92), seed, fit_gain=NORMALISED_FIT_GAIN)
    elif kind == "copper":
        w = xavier_weights(("Cu",), 8.0, 2.0, (512,), seed, fit_gain=NORMALISED_FIT_GAIN)
    else:
        raise KeyError(kind)
    if tuple(stats[kind]["type_names"]) != w.type_names:
        raise ValueError("statistics are for other types")
    return with_statistics(w, stats[kind]["davg"], stats[kind]["dstd"])


def maxwell_boltzmann(masses_per_atom: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Initial velocities [N, 3] in A/fs: Maxwell-Boltzmann at `temperature`, centre-of-mass
    velocity removed, then rescaled so the kinetic temperature with 3N - 3 degrees of
    freedom is exactly `temperature`."""
    rng = np.random.default_rng(seed)
    m = np.asarray(masses_per_atom, dtype=np.float64)
    sigma = np.sqrt(KB_EV * temperature * ACC_CONV / m)  # A/fs
    v = rng.standard_normal((len(m), 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    ke = 0.5 * (m[:, None] * v * v).sum() / ACC_CONV
    dof = 3 * len(m) - 3
    t_now = 2.0 * ke / (dof * KB_EV)
    return v * math.sqrt(temperature / t_now)
