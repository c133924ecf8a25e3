"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never loads it, and
the oracle shares no code with the library: both read the same seeded inputs
written by ``paper_2410_22867_gb300.synth``.

Every function here is a thin ctypes wrapper around ``dp_oracle.cpp`` (plain
C++, FP64, compiled with ``-ffp-contract=off``).  Parity of the absolute energy
is pinned only by closed forms on sparse weights and by self-consistency
(finite differences, invariances); the paper prints no worked example.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dp_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libdporacle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (g++, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O3", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.oracle_model_load.restype = _P
            L.oracle_model_load.argtypes = [_P, ctypes.c_size_t]
            L.oracle_model_free.argtypes = [_P]
            L.oracle_model_ntheta.restype = ctypes.c_longlong
            L.oracle_model_ntheta.argtypes = [_P]
            L.oracle_model_S.argtypes = [_P]
            L.oracle_set_threads.argtypes = [_I]
            L.oracle_get_threads.restype = _I
            L.oracle_wrap.argtypes = [_I, _P, _P, _P]
            L.oracle_nlist.argtypes = [_P, _I, _P, _P, _P, _D, _P, _I, _P, _P, _P]
            L.oracle_compute.argtypes = [_P, _I, _P, _P, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P]
            L.oracle_rdf.argtypes = [_P, _I, _P, _P, _P, _I, _D, _P]
            L.oracle_dir_deriv.argtypes = [_P, _I, _P, _P, _P, _P, _P]
            L.oracle_param_grad.argtypes = [_P, _I, _P, _P, _P, _D, _P, _D, _D, _I, _P, _P, _P, _P]
            L.oracle_md.argtypes = [_P, _I, _P, _P, _P, _P, _P, _D, _I, _I, _D, _P, _P, _P]
            L.oracle_md_harmonic.argtypes = [_I, _P, _P, _P, _D, _D, _I, _P]
            L.oracle_model_ntypes.argtypes = [_P]
            L.oracle_env_stats.argtypes = [_P, _I, _P, _P, _P, _P]
            L.oracle_tabulate.argtypes = [_P, _D, _D, _I]
            L.oracle_emb_eval.argtypes = [_P, _I, _I, _P, _I, _P, _P, _P]
            L.oracle_set_truncation.argtypes = [_P, _I]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleError(RuntimeError):
    pass


_STATUS = {1: "bad argument", 4: "unsupported box", 5: "neighbour overflow", 6: "skin exceeded",
           9: "bad weights"}


def _check(st):
    if st != 0:
        raise OracleError(f"oracle status {st}: {_STATUS.get(st, '?')}")


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


class Model:
    """Oracle model built from a weight blob (``synth.Weights.to_blob()``)."""

    def __init__(self, blob: bytes):
        self._blob = ctypes.create_string_buffer(blob, len(blob))
        self.h = lib().oracle_model_load(self._blob, len(blob))
        if not self.h:
            raise OracleError("oracle rejected the weight blob")
        self.S = int(lib().oracle_model_S(self.h))
        self.ntheta = int(lib().oracle_model_ntheta(self.h))
        self.ntypes = int(lib().oracle_model_ntypes(self.h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.oracle_model_free(h)
            self.h = None

    def set_truncation(self, nearest: bool):
        """Neighbour overflow policy: False = more than sel_t neighbours of a type is an error,
        True = keep the sel_t nearest (r^2, then neighbour index, then image)."""
        lib().oracle_set_truncation(self.h, 1 if nearest else 0)

    # -- neighbour list -------------------------------------------------------
    def nlist(self, coords, types, box, method: str = "cell", rcut: float = 0.0, sel=None):
        coords, types, box = _f64(coords), _i32(types), _f64(box)
        N = len(types)
        S = self.S if sel is None else int(sum(sel))
        nl = np.empty((N, S), np.int32)
        im = np.empty((N, S), np.int32)
        selarr = None if sel is None else _i32(sel)
        counts = np.empty((N, self.ntypes), np.int32)
        st = lib().oracle_nlist(self.h, N, _ptr(coords), _ptr(types), _ptr(box), float(rcut), _ptr(selarr),
                                0 if method == "brute" else 1, _ptr(nl), _ptr(im), _ptr(counts))
        if st not in (0, 5):
            _check(st)
        return nl, im, counts, st == 5

    # -- evaluation -----------------------------------------------------------
    def compute(self, coords, types, box, method: str = "cell", centre_mask=None, forces: bool = True,
                intermediates: bool = False, atom_virial: bool = False):
        coords, types, box = _f64(coords), _i32(types), _f64(box)
        N = len(types)
        E = np.zeros(1)
        Ei = np.zeros(N)
        F = np.zeros((N, 3)) if forces else None
        V = np.zeros(9) if forces else None
        T = D = dD = None
        if intermediates:
            T = np.zeros((N, 4, 100))
            D = np.zeros((N, 1600))
            dD = np.zeros((N, 1600)) if forces else None
        mask = None if centre_mask is None else np.ascontiguousarray(centre_mask, dtype=np.uint8)
        W = np.zeros((N, 3, 3)) if (atom_virial and forces) else None
        st = lib().oracle_compute(self.h, N, _ptr(coords), _ptr(types), _ptr(box),
                                  0 if method == "brute" else 1, _ptr(mask), int(forces), _ptr(E), _ptr(Ei),
                                  _ptr(F), _ptr(V), _ptr(T), _ptr(D), _ptr(dD), _ptr(W))
        _check(st)
        out = {"energy": float(E[0]), "atom_energy": Ei}
        if forces:
            out["forces"] = F
            out["virial"] = V.reshape(3, 3)
        if intermediates:
            out.update(T=T, D=D, dD=dD)
        if W is not None:
            out["atom_virial"] = W
        return out

    def rdf(self, coords, types, box, nbins: int, r_max: float):
        """Pair-distance histogram counts [ntypes, ntypes, nbins] of all pairs within r_max (each
        pair counted from both ends)."""
        coords, types, box = _f64(coords), _i32(types), _f64(box)
        out = np.zeros((self.ntypes, self.ntypes, nbins), dtype=np.uint64)
        _check(lib().oracle_rdf(self.h, len(types), _ptr(coords), _ptr(types), _ptr(box), int(nbins), float(r_max),
                                _ptr(out)))
        return out

    def energy(self, coords, types, box) -> float:
        return self.compute(coords, types, box, forces=False)["energy"]

    def env_stats(self, coords, types, box):
        """Per centre type t: [slots, sum s, sum s^2, sum of squared angular components,
        atoms] over every neighbour slot (padded slots are zero rows) of the
        un-normalised environment rows; shape [ntypes, 5]."""
        coords, types, box = _f64(coords), _i32(types), _f64(box)
        out = np.zeros((self.ntypes, 5))
        _check(lib().oracle_env_stats(self.h, len(types), _ptr(coords), _ptr(types), _ptr(box), _ptr(out)))
        return out

    def tabulate(self, x0: float, x1: float, n: int) -> None:
        """Replace every embedding net by its quintic table on n uniform intervals of [x0, x1]
        (the compressed model); n = 0 goes back to the networks."""
        _check(lib().oracle_tabulate(self.h, float(x0), float(x1), int(n)))

    def emb_eval(self, pair: int, x, tabulated: bool = False):
        """Embedding output of pair ti * ntypes + tj at inputs x: (G, G', G''), each [len(x), 100],
        from the network or from the table."""
        x = _f64(np.atleast_1d(x))
        g, g1, g2 = (np.zeros((len(x), 100)) for _ in range(3))
        _check(lib().oracle_emb_eval(self.h, int(pair), len(x), _ptr(x), int(tabulated), _ptr(g), _ptr(g1),
                                     _ptr(g2)))
        return g, g1, g2

    def dir_deriv(self, coords, types, box, w):
        coords, types, box, w = _f64(coords), _i32(types), _f64(box), _f64(w)
        out = np.zeros(2)
        _check(lib().oracle_dir_deriv(self.h, len(types), _ptr(coords), _ptr(types), _ptr(box), _ptr(w), _ptr(out)))
        return float(out[0]), float(out[1])

    def param_grad(self, coords, types, box, E0, F0, idx, cE=1.0, cF=1.0):
        coords, types, box, F0 = _f64(coords), _i32(types), _f64(box), _f64(F0)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        g = np.zeros(len(idx))
        dE = np.zeros(len(idx))
        loss = np.zeros(1)
        _check(lib().oracle_param_grad(self.h, len(types), _ptr(coords), _ptr(types), _ptr(box), float(E0),
                                       _ptr(F0), float(cE), float(cF), len(idx), _ptr(idx), _ptr(g), _ptr(dE),
                                       _ptr(loss)))
        return g, dE, float(loss[0])

    def md(self, coords, velocities, types, box, masses_by_type, dt, nsteps, rebuild_every=10, skin=2.0):
        x = _f64(coords).copy()
        v = _f64(velocities).copy()
        types, box, mt = _i32(types), _f64(box), _f64(masses_by_type)
        pe = np.zeros(nsteps + 1)
        ke = np.zeros(nsteps + 1)
        F = np.zeros_like(x)
        _check(lib().oracle_md(self.h, len(types), _ptr(x), _ptr(v), _ptr(types), _ptr(box), _ptr(mt), float(dt),
                               int(nsteps), int(rebuild_every), float(skin), _ptr(pe), _ptr(ke), _ptr(F)))
        return {"x": x, "v": v, "pe": pe, "ke": ke, "forces": F}


def md_harmonic(coords, velocities, masses, k_spring, dt, nsteps):
    """The oracle's velocity-Verlet loop driven by F = -k x; returns positions per step."""
    x = _f64(coords).copy()
    v = _f64(velocities).copy()
    m = _f64(masses)
    traj = np.zeros((nsteps + 1,) + x.shape)
    _check(lib().oracle_md_harmonic(len(m), _ptr(x), _ptr(v), _ptr(m), float(k_spring), float(dt), int(nsteps),
                                    _ptr(traj)))
    return traj


def wrap(coords, box):
    coords, box = _f64(coords), _f64(box)
    out = np.empty_like(coords)
    _check(lib().oracle_wrap(len(coords), _ptr(coords), _ptr(box), _ptr(out)))
    return out
