"""GB300 Deep Potential library: Python binding of the C ABI in include/dp.h.

This module only marshals arguments (device pointers from torch tensors, the
current CUDA stream) into ``libdpgb300.so``; every step of the computation runs
in the library's CUDA kernels.  There is no CPU fallback: if the library is
missing or no GPU is present, calls raise.

    from paper_2410_22867_gb300 import DPModel, synth
    w = synth.water_weights()
    m = DPModel(w, precision="fp32", max_atoms=20000)
    out = m.compute(coords_cuda, types_cuda, box)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpgb300.so")
_lock = threading.Lock()
_lib = None

PRECISIONS = {"fp64": 0, "fp32": 1, "mix_bf16": 2, "mix_fp16": 3}
STATUS = {0: "DP_OK", 1: "DP_ERR_ARG", 2: "DP_ERR_CUDA", 3: "DP_ERR_OOM", 4: "DP_ERR_UNSUPPORTED",
          5: "DP_ERR_SEL_OVERFLOW", 6: "DP_ERR_SKIN_EXCEEDED", 7: "DP_ERR_WAIT_TIMEOUT", 8: "DP_ERR_CAPACITY",
          9: "DP_ERR_WEIGHTS"}

# exported symbols of include/dp.h
EXPORTS = ("dp_create", "dp_compute", "dp_compute_batch", "dp_verlet_step", "dp_md_run_batch", "dp_param_grad",
           "dp_ntheta", "dp_get_nlist", "dp_phase_times", "dp_kernel_launches", "dp_sync", "dp_last_error",
           "dp_destroy", "dp_version", "dp_selftest", "dp_selftest_noalloc", "dp_set_params", "dp_autotune",
           "dp_wait_selftest", "dp_measure_peak", "dp_tabulate", "dp_rdf", "dp_atom_virial",
           "dp_set_truncation")

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


class DPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MDState(ctypes.Structure):
    """Mirror of dp_md_state."""
    _fields_ = [("natoms", _I), ("nrep", _I), ("atom_offsets", _P), ("boxes", _P), ("x", _P), ("v", _P),
                ("types", _P), ("mass_by_type", _P), ("forces", _P), ("potential", _P), ("kinetic", _P),
                ("virial", _P), ("step", ctypes.c_longlong), ("rebuild_every", _I), ("resume", _I)]


def build(force: bool = False) -> str:
    """Compile libdpgb300.so for sm_103a (see buildlib.py)."""
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """Load libdpgb300.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_22867_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            L.dp_create.argtypes = [ctypes.POINTER(_P), _I, _P, _D, _D, _P, ctypes.c_char_p, _P, ctypes.c_size_t, _I,
                                    _I, _I, _D, _P]
            L.dp_compute.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P, _P]
            L.dp_compute_batch.argtypes = [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P]
            L.dp_verlet_step.argtypes = [_P, ctypes.POINTER(MDState), _D, _I, _I]
            L.dp_md_run_batch.argtypes = [_P, ctypes.POINTER(MDState), _D, _I]
            L.dp_param_grad.argtypes = [_P, _I, _P, _P, _P, _D, _P, _D, _D, _P, _P]
            L.dp_ntheta.argtypes = [_P]
            L.dp_ntheta.restype = ctypes.c_longlong
            L.dp_get_nlist.argtypes = [_P, _P, _P]
            L.dp_sync.argtypes = [_P]
            L.dp_last_error.argtypes = [_P]
            L.dp_last_error.restype = ctypes.c_char_p
            L.dp_destroy.argtypes = [_P]
            L.dp_version.restype = ctypes.c_char_p
            L.dp_phase_times.argtypes = [_P, _I, _P]
            L.dp_kernel_launches.argtypes = [_P]
            L.dp_kernel_launches.restype = ctypes.c_longlong
            L.dp_selftest.argtypes = [_I, _P]
            L.dp_selftest_noalloc.argtypes = [_P, _I, _P]
            L.dp_set_params.argtypes = [_P, _P, ctypes.c_longlong]
            L.dp_autotune.argtypes = [_P, _I, _P]
            L.dp_wait_selftest.argtypes = [ctypes.c_uint]
            L.dp_measure_peak.argtypes = [_I, _P]
            L.dp_tabulate.argtypes = [_P, _D, _D, _I]
            L.dp_rdf.argtypes = [_P, _I, _D, _P]
            L.dp_atom_virial.argtypes = [_P, _P]
            L.dp_set_truncation.argtypes = [_P, _I]
            for name in ("dp_create", "dp_compute", "dp_compute_batch", "dp_verlet_step", "dp_md_run_batch",
                         "dp_param_grad", "dp_get_nlist", "dp_phase_times", "dp_sync", "dp_selftest",
                         "dp_selftest_noalloc", "dp_set_params", "dp_autotune", "dp_wait_selftest",
                         "dp_measure_peak", "dp_tabulate", "dp_rdf", "dp_atom_virial", "dp_set_truncation"):
                getattr(L, name).restype = _I
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _host_f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def selftest(which: int):
    """Run the library's tensor-core layout self check; returns (max error, max value)."""
    out = (ctypes.c_double * 2)()
    st = lib().dp_selftest(int(which), ctypes.cast(out, _P))
    if st != 0:
        raise DPError(st, "dp_selftest failed")
    return out[0], out[1]


def wait_selftest(spin_limit: int = 4096) -> int:
    """dp_wait_selftest: run a bounded wait that nothing completes; returns the status
    (DP_ERR_WAIT_TIMEOUT = 7 when the wait gave up, as it should)."""
    return int(lib().dp_wait_selftest(int(spin_limit)))


PEAK_KINDS = {"tanh": 0, "ex2": 1, "rcp": 2, "ffma": 3, "dfma": 4}


def measure_peak(kind: str) -> float:
    """dp_measure_peak: measured rate of one arithmetic unit on the current device
    (tanh, ex2, rcp: results/s; ffma, dfma: FLOP/s)."""
    r = ctypes.c_double(0.0)
    st = lib().dp_measure_peak(PEAK_KINDS[kind], ctypes.byref(r))
    if st != 0:
        raise DPError(st, f"dp_measure_peak({kind}) failed")
    return r.value


SELFTEST_NOALLOC_MAX_CASES = 16


def selftest_noalloc(cases):
    """dp_selftest_noalloc: the self check for each case in ``cases`` with no
    allocation (fixed scratch inside the library); returns [(max error, max value)]."""
    cases = [int(c) for c in cases]
    n = len(cases)
    which = (ctypes.c_int * max(n, 1))(*cases)
    out = (ctypes.c_double * max(2 * n, 2))()
    st = lib().dp_selftest_noalloc(ctypes.cast(which, _P), n, ctypes.cast(out, _P))
    if st != 0:
        raise DPError(st, "dp_selftest_noalloc failed")
    return [(out[2 * i], out[2 * i + 1]) for i in range(n)]


class DPModel:
    """A model on the current CUDA device (one C-ABI dp_model handle).

    weights: ``synth.Weights`` or a blob (bytes).  precision: fp64 | fp32 |
    mix_bf16 | mix_fp16.  stream: torch.cuda.Stream or None (current stream).
    """

    def __init__(self, weights, precision: str = "fp64", max_atoms: int = 1 << 16, max_replicas: int = 1,
                 skin: float = 2.0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("DPModel needs a CUDA GPU")
        if isinstance(weights, (bytes, bytearray)):
            raise ValueError("pass synth.Weights so the type map, cutoffs and sel can be checked")
        blob = weights.to_blob()
        self.weights = weights
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.device("cuda", torch.cuda.current_device())
        nt = weights.ntypes
        names = (ctypes.c_char_p * nt)(*[n.encode() for n in weights.type_names])
        sel = (ctypes.c_int * nt)(*weights.sel)
        self._blob = ctypes.create_string_buffer(bytes(blob), len(blob))
        h = _P()
        st = lib().dp_create(ctypes.byref(h), nt, ctypes.cast(names, _P), float(weights.rcut), float(weights.rcut_smth),
                             ctypes.cast(sel, _P), None, ctypes.cast(self._blob, _P), len(blob), PRECISIONS[precision],
                             int(max_atoms), int(max_replicas), float(skin), _P(self.stream.cuda_stream))
        if st != 0:
            raise DPError(st, "dp_create failed")
        self.h = h
        self.S = int(sum(weights.sel))
        self.ntypes = nt
        self.max_atoms = max_atoms

    def close(self):
        if getattr(self, "h", None):
            lib().dp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise DPError(st, lib().dp_last_error(self.h).decode())

    def sync(self):
        """Wait for the model's stream and raise the sticky device error, if any."""
        self._check(lib().dp_sync(self.h))

    # ------------------------------------------------------------------ compute
    def compute(self, coords, types, box, sync: bool = True):
        """coords [N,3] float64 cuda, types [N] int32 cuda, box: 9 host floats."""
        import torch
        N = int(types.shape[0])
        out = {"energy": torch.empty(1, dtype=torch.float64, device=coords.device),
               "atom_energy": torch.empty(N, dtype=torch.float64, device=coords.device),
               "forces": torch.empty(N, 3, dtype=torch.float64, device=coords.device),
               "virial": torch.empty(3, 3, dtype=torch.float64, device=coords.device)}
        b = _host_f64(box).ravel()
        self._check(lib().dp_compute(self.h, N, _ptr(coords), _ptr(types), b.ctypes.data_as(_P), _ptr(out["energy"]),
                                     _ptr(out["atom_energy"]), _ptr(out["forces"]), _ptr(out["virial"])))
        if sync:
            self.sync()
        return out

    def compute_batch(self, coords, types, atom_offsets, boxes, sync: bool = True):
        import torch
        offs = np.ascontiguousarray(atom_offsets, dtype=np.int32)
        bx = _host_f64(boxes).reshape(-1)
        nrep = len(offs) - 1
        N = int(offs[-1])
        dev = coords.device
        out = {"energy": torch.empty(nrep, dtype=torch.float64, device=dev),
               "atom_energy": torch.empty(N, dtype=torch.float64, device=dev),
               "forces": torch.empty(N, 3, dtype=torch.float64, device=dev),
               "virial": torch.empty(nrep, 3, 3, dtype=torch.float64, device=dev)}
        self._check(lib().dp_compute_batch(self.h, nrep, offs.ctypes.data_as(_P), _ptr(coords), _ptr(types),
                                           bx.ctypes.data_as(_P), _ptr(out["energy"]), _ptr(out["atom_energy"]),
                                           _ptr(out["forces"]), _ptr(out["virial"])))
        if sync:
            self.sync()
        return out

    def get_nlist(self):
        import torch
        N = self._last_n
        nl = torch.empty(N, self.S, dtype=torch.int32, device=self.device)
        im = torch.empty(N, self.S, dtype=torch.int32, device=self.device)
        self._check(lib().dp_get_nlist(self.h, _ptr(nl), _ptr(im)))
        return nl, im

    # ------------------------------------------------------------------ MD
    def md_state(self, x, v, types, boxes, masses_by_type, atom_offsets=None, rebuild_every: int = 10):
        """Build a dp_md_state over caller-owned cuda tensors x, v [N,3] float64 (updated in place)."""
        import torch
        N = int(types.shape[0])
        offs = None if atom_offsets is None else np.ascontiguousarray(atom_offsets, dtype=np.int32)
        nrep = 1 if offs is None else len(offs) - 1
        bx = _host_f64(boxes).reshape(-1)
        mt = _host_f64(masses_by_type)
        dev = x.device
        keep = {"offs": offs, "boxes": bx, "masses": mt,
                "forces": torch.zeros(N, 3, dtype=torch.float64, device=dev),
                "potential": torch.zeros(nrep, dtype=torch.float64, device=dev),
                "kinetic": torch.zeros(nrep, dtype=torch.float64, device=dev),
                "virial": torch.zeros(nrep, 3, 3, dtype=torch.float64, device=dev),
                "x": x, "v": v, "types": types}
        st = MDState(N, nrep, None if offs is None else offs.ctypes.data_as(_P), bx.ctypes.data_as(_P), _ptr(x),
                     _ptr(v), _ptr(types), mt.ctypes.data_as(_P), _ptr(keep["forces"]), _ptr(keep["potential"]),
                     _ptr(keep["kinetic"]), _ptr(keep["virial"]), 0, int(rebuild_every))
        st._keep = keep
        self._last_n = N
        return st

    def verlet(self, state: MDState, dt: float, nsteps: int, capture_graph: bool = True, sync: bool = True):
        self._check(lib().dp_verlet_step(self.h, ctypes.byref(state), float(dt), int(nsteps), int(capture_graph)))
        if sync:
            self.sync()
        return state._keep

    def md_run_batch(self, state: MDState, dt: float, nsteps: int, sync: bool = True):
        self._check(lib().dp_md_run_batch(self.h, ctypes.byref(state), float(dt), int(nsteps)))
        if sync:
            self.sync()
        return state._keep

    # ------------------------------------------------------------------ measurement
    def phase_times(self, repeats: int = 3):
        """Mean ms of [format, descriptor, fitting, embedding backward, whole evaluation,
        embedding forward kernel, embedding backward kernel] (dp_phase_times)."""
        ms = (ctypes.c_float * 8)()
        self._check(lib().dp_phase_times(self.h, int(repeats), ctypes.cast(ms, _P)))
        return list(ms)[:7]

    def set_truncation(self, nearest: bool):
        """dp_set_truncation: False = more than sel_t neighbours of a type within r_c is
        DP_ERR_SEL_OVERFLOW; True = keep the sel_t nearest (DeePMD's convention)."""
        self._check(lib().dp_set_truncation(self.h, 1 if nearest else 0))

    def tabulate(self, n_intervals: int = 256, x_min: float | None = None, x_max: float | None = None):
        """dp_tabulate: replace the embedding nets by their quintic tables (the compressed model).
        The default range runs from the normalised input of a neighbour at r_c (-davg/dstd) to that
        of a neighbour at 0.5 A, over all centre types, with a margin of 0.05; n_intervals = 0 goes
        back to the nets.  Returns (x_min, x_max, n_intervals)."""
        w = self.weights
        if x_min is None:
            x_min = min(-w.davg[t][0] / w.dstd[t][0] for t in range(w.ntypes)) - 0.05
        if x_max is None:
            x_max = max((2.0 - w.davg[t][0]) / w.dstd[t][0] for t in range(w.ntypes)) + 0.05
        self._check(lib().dp_tabulate(self.h, float(x_min), float(x_max), int(n_intervals)))
        return float(x_min), float(x_max), int(n_intervals)

    def rdf(self, nbins: int, r_max: float):
        """dp_rdf: pair-distance histogram [ntypes, ntypes, nbins] (uint64) of the last evaluation."""
        out = np.zeros((self.ntypes, self.ntypes, int(nbins)), dtype=np.uint64)
        self._check(lib().dp_rdf(self.h, int(nbins), float(r_max), out.ctypes.data_as(_P)))
        return out

    def atom_virial(self, sync: bool = True):
        """dp_atom_virial: per-atom virial [N, 3, 3] (caller order) of the last evaluation."""
        import torch
        out = torch.empty(self._last_n, 3, 3, dtype=torch.float64, device=self.device)
        self._check(lib().dp_atom_virial(self.h, _ptr(out)))
        if sync:
            self.sync()
        return out

    def autotune(self, repeats: int = 3):
        """dp_autotune: choose the launch grids of the mixed kernels on the current state;
        returns [embedding forward, embedding backward, dE/dT, descriptor] (0 = not tuned).
        repeats = 0 only reports the current choices."""
        g = (ctypes.c_int * 4)()
        self._check(lib().dp_autotune(self.h, int(repeats), ctypes.cast(g, _P)))
        return list(g)

    def kernel_launches(self) -> int:
        return int(lib().dp_kernel_launches(self.h))

    # ------------------------------------------------------------------ gradient
    def ntheta(self) -> int:
        return int(lib().dp_ntheta(self.h))

    def set_params(self, theta):
        """Replace the network parameters (dp_set_params): theta [ntheta] float64 in the weight
        blob's parameter order (numpy array or torch tensor on any device)."""
        if hasattr(theta, "detach"):
            theta = theta.detach().to("cpu").numpy()
        th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
        self._check(lib().dp_set_params(self.h, th.ctypes.data_as(_P), int(th.size)))

    def param_grad(self, coords, types, box, E0, F0, cE=1.0, cF=1.0, sync: bool = True):
        import torch
        N = int(types.shape[0])
        g = torch.empty(self.ntheta(), dtype=torch.float64, device=coords.device)
        loss = torch.empty(1, dtype=torch.float64, device=coords.device)
        b = _host_f64(box).ravel()
        self._check(lib().dp_param_grad(self.h, N, _ptr(coords), _ptr(types), b.ctypes.data_as(_P), float(E0),
                                        _ptr(F0), float(cE), float(cF), _ptr(g), _ptr(loss)))
        if sync:
            self.sync()
        return g, loss


def _remember_n(fn):
    def wrap(self, coords, types, *a, **k):
        self._last_n = int(types.shape[0])
        return fn(self, coords, types, *a, **k)
    return wrap


DPModel.compute = _remember_n(DPModel.compute)
DPModel.compute_batch = _remember_n(DPModel.compute_batch)


def rdf_g(counts, natoms_by_type, volume: float, r_max: float):
    """g_ab(r) at the bin centres from dp_rdf counts [nt, nt, nbins]: counts / (N_a rho_b 4 pi r^2 dr),
    rho_b = N_b / V (N_b - 1 for a = b).  Returns (r, g)."""
    c = np.asarray(counts, dtype=np.float64)
    nt, _, nb = c.shape
    dr = r_max / nb
    r = (np.arange(nb) + 0.5) * dr
    shell = 4.0 * np.pi * r * r * dr
    g = np.zeros_like(c)
    for a in range(nt):
        for b in range(nt):
            nb_ = natoms_by_type[b] - (1 if a == b else 0)
            g[a, b] = c[a, b] / (natoms_by_type[a] * (nb_ / volume) * shell)
    return r, g


def _make_param_loss():
    import torch

    class ParamLoss(torch.autograd.Function):
        """L(theta) = cE (E - E0)^2 + cF sum_k |F_k - F0_k|^2 of one box as a differentiable
        function of the network parameters theta (float64 tensor [ntheta]).  The forward
        loads theta into `model` (dp_set_params) and runs dp_param_grad, which returns the
        loss and its full gradient; the backward scales that gradient.  coords, types, F0
        are device tensors in the caller's atom order, box a host 3x3."""

        @staticmethod
        def forward(ctx, theta, model, coords, types, box, E0, F0, cE=1.0, cF=1.0):
            model.set_params(theta)
            g, loss = model.param_grad(coords, types, box, float(E0), F0, float(cE), float(cF))
            ctx.save_for_backward(g.to(theta.device, theta.dtype))
            return loss.to(theta.device, theta.dtype).reshape(())

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g, None, None, None, None, None, None, None, None

    return ParamLoss


def _make_potential():
    import torch
    from torch.autograd.function import once_differentiable

    class Potential(torch.autograd.Function):
        """E(x) of one periodic box as a differentiable function of the coordinates.

        forward(coords, model, types, box) -> (energy, virial): coords [N, 3] float64 cuda
        (caller order), types [N] int32 cuda, box a host 3x3; energy is a 0-d float64
        tensor, virial [3, 3] (not differentiable).  One dp_compute call evaluates E, the
        forces F = -dE/dx and the virial (prod_force / prod_virial of the backward pass);
        backward returns grad_E * (-F) for coords.  The backward is not itself
        differentiable (no second derivatives)."""

        @staticmethod
        def forward(ctx, coords, model, types, box):
            out = model.compute(coords.detach().contiguous(), types, box)
            ctx.save_for_backward(out["forces"])
            ctx.mark_non_differentiable(out["virial"])
            return out["energy"].reshape(()), out["virial"]

        @staticmethod
        @once_differentiable
        def backward(ctx, g_energy, g_virial):
            (F,) = ctx.saved_tensors
            return -g_energy * F, None, None, None

    return Potential


try:
    ParamLoss = _make_param_loss()
    Potential = _make_potential()
except ImportError:  # torch is needed only for the autograd wrappers
    ParamLoss = None
    Potential = None
