#!/usr/bin/env python
"""Throughput of the Deep Potential MD step on one GB300 (or N independent replicas).

One step = one velocity-Verlet NVE step: half kick, drift, neighbour rebuild every
10 steps (else the skin check), the list filter, environment matrix, embedding net,
descriptor, fitting net, force/virial backward, half kick.  Metric: atom-steps/s
(atoms x steps / s) and ns/day at dt = 0.5 fs.  Inputs are synthetic (seeded) with
the paper's sizes; the working set of one step (>1 GB) is larger than L2, so no
explicit flush is needed between timed iterations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--workload cu131k|water12k] [--precision mix_bf16|mix_fp16|fp32|fp64]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DP energy+force atom-steps/s and ns/day on 1 GB300: mixed vs FP64 at stated error"
DT_FS = 0.5
REBUILD = 10

WORKLOADS = {
    "cu131k": "Cu FCC 32x32x32 cells (131,072 atoms), a 3.634 A, sigma 0.08 A, r_c 8 A, r_s 2 A, sel 512, "
              "NVE dt 0.5 fs from 300 K, rebuild every 10 steps, skin 2 A",
    "water12k": "4096 H2O (12,288 atoms) at 1.0 g/cm3, r_c 6 A, r_s 0.5 A, sel 46/92, NVE dt 0.5 fs from 300 K, "
                "rebuild every 10 steps, skin 2 A",
    # a smaller copper box for kernel profiles: same model, density and neighbour count per atom
    "cu32k": "Cu FCC 20x20x20 cells (32,000 atoms), a 3.634 A, sigma 0.08 A, r_c 8 A, r_s 2 A, sel 512, "
             "NVE dt 0.5 fs from 300 K, rebuild every 10 steps, skin 2 A",
}

# per real neighbour: embedding recompute + backward MACs (x2 FLOP); forward embedding + T
EMB_BWD_FLOP_PER_NEIGHBOUR = 2 * (6275 + 7075)
EMB_FWD_FLOP_PER_NEIGHBOUR = 2 * (6275 + 400)
FIT_FLOP_PER_ATOM = 2 * (499440 * 2)  # forward + data-gradient backward


def load_workload(name):
    from paper_2410_22867_gb300 import synth
    if name == "cu131k":
        s = synth.copper_fcc(32, 0)
        w = synth.copper_weights(1001)
    elif name == "cu32k":
        s = synth.copper_fcc(20, 0)
        w = synth.copper_weights(1001)
    elif name == "water12k":
        s = synth.water_box(4096, 0)
        w = synth.water_weights(1001)
    else:
        raise SystemExit(f"unknown workload {name}")
    v = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 1)
    return s, w, v


def cpu_sample(name):
    """A bounded CPU sample of the same workload: same model and density, smaller box."""
    from paper_2410_22867_gb300 import synth
    if name in ("cu131k", "cu32k"):
        return synth.copper_fcc(8, 0), synth.copper_weights(1001)
    return synth.water_box(256, 0), synth.water_weights(1001)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"dp_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            tok = [t.strip() for t in line.split(",")]
            if len(tok) >= 9:
                rows.append(tok)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        if torch.cuda.is_available():
            torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest of the ranks' values (timed regions: the slowest rank sets the time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, natoms_per_rank, steps, t_ms):
    """Whole-job atom-steps/s: every rank advances its own replica of natoms_per_rank atoms
    for `steps` steps; t_ms is the max over ranks of the timed region."""
    return world * natoms_per_rank * steps / (t_ms * 1e-3)


def oracle_rate(name, seconds_target=None, nsteps=1):
    """Oracle (FP64 CPU) atom-steps/s on the bounded sample; returns (rate, cores, sample, per_step_s)."""
    import oracle
    s, w = cpu_sample(name)
    m = oracle.Model(w.to_blob())
    m.compute(s.coords, s.types, s.box)  # warm
    t0 = time.perf_counter()
    for _ in range(nsteps):
        m.compute(s.coords, s.types, s.box)
    dt = time.perf_counter() - t0
    return s.natoms * nsteps / dt, oracle.get_threads(), \
        f"{s.natoms}-atom periodic box of the same model and density, full energy+force evaluation", dt / nsteps


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    oracle.set_threads(len(os.sched_getaffinity(0)))
    rate_w, cores, sample, per = oracle_rate(args.workload, nsteps=1)
    for _ in range(max(0, args.warmup - 1)):
        oracle_rate(args.workload, nsteps=1)
    rate, cores, sample, per = oracle_rate(args.workload, nsteps=max(1, args.steps))
    line = {"metric": METRIC, "value": rate, "unit": "atom-steps/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "sample": sample, "threads": cores},
            "cpu_baseline": {"value": rate, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Algorithmic tanh per real neighbour row of the embedding net (25 + 50 + 100); the backward
# recomputes the forward, and tanh' = 1 - t^2 needs no further tanh.
TANH_PER_NEIGHBOUR = 175

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the 32,000-atom copper box, per real neighbour row (embedding kernels) or per atom (fitting),
# scaled to a launch by the row or atom count.  Each entry names the source file of the kernel
# and its SHA-1 at the capture: when the file has changed since, the figure no longer describes
# the kernel and `traffic` is reported as null.
TRAFFIC_PER_ROW = {
    ("embedding_backward", "mix_fp16"): {"bytes_per_unit": (171.784448e6 + 4.521984e6) / 5726060, "unit": "row",
                                         "source": "paper_2410_22867_gb300/csrc/mix_embed.cu",
                                         "sha1": "6f6ae8c2452f3221d1e7684b71aefd4ddf1483f5"},
    ("embedding_forward", "mix_fp16"): {"bytes_per_unit": (95.683328e6 + 21.243904e6) / 5726060, "unit": "row",
                                        "source": "paper_2410_22867_gb300/csrc/mix_embed.cu",
                                        "sha1": "6f6ae8c2452f3221d1e7684b71aefd4ddf1483f5"},
    ("fitting", "mix_fp16"): {"bytes_per_unit": (106.631680e6 + 75.120640e6) / 32000, "unit": "atom",
                              "source": "paper_2410_22867_gb300/csrc/mix_fit.cu",
                              "sha1": "a9afad59b8d8cbab7736d97dcdeeb23fd961956c"},
}


def _sha1(path):
    import hashlib
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            return hashlib.sha1(f.read()).hexdigest()
    except OSError:
        return None


def traffic_per_launch(kernel, prec, rows, atoms):
    e = TRAFFIC_PER_ROW.get((kernel, prec))
    if e is None or _sha1(e["source"]) != e["sha1"]:
        return None
    return e["bytes_per_unit"] * (rows if e["unit"] == "row" else atoms)


def measured_peaks(dp):
    """Rates of the arithmetic units measured on this device right now (dp_measure_peak):
    tanh / ex2 / rcp results per second, FP32 and FP64 FLOP/s."""
    out = {}
    for k in ("tanh", "ex2", "rcp", "ffma", "dfma"):
        try:
            out[k] = dp.measure_peak(k)
        except Exception as e:  # noqa: BLE001
            out[k] = None
            out[k + "_error"] = str(e)
    return out


def kernel_times(ph):
    return {"format": ph[0], "embedding_forward": ph[5], "descriptor": max(0.0, ph[1] - ph[5]),
            "fitting": ph[2], "dE_dT": max(0.0, ph[3] - ph[6]), "embedding_backward": ph[6]}


def hbm_bytes_per_atom(kernel, ntypes):
    """Algorithmic HBM bytes per atom of the mixed-precision dE/dT and descriptor kernels:
    dE/dT reads dE/dD (1600 x fp16) and T (400 x FP32) and writes dE/dT (400 x FP32); the
    descriptor reads the partial T of each neighbour type (400 x FP32 each) and writes T
    (400 x FP32) and D (1600 x 16 bit)."""
    if kernel == "dE_dT":
        return 2 * 1600 + 4 * 400 + 4 * 400
    if kernel == "descriptor":
        return 4 * 400 * ntypes + 4 * 400 + 2 * 1600
    return None


def roofline(prec, kernel, ms, N, n_neigh, alu, ntypes=1):
    """Roofline entry of one kernel of a force evaluation.  alu: measured_peaks().
    Mixed precisions: embedding kernels against max(tensor, SFU) with the SFU rate measured
    by dp_measure_peak('tanh'); fitting against the burst bf16 tensor peak (the kernel is timed
    in millisecond phases, not a sustained loop); dE/dT and descriptor against the measured
    HBM copy rate.  FP32 / FP64: FMA-pipe work of the dense contractions against the measured
    FFMA / DFMA rate."""
    pk, src = peaks()
    t = ms * 1e-3
    mixed = prec.startswith("mix")
    out = {"kernel": kernel, "kernel_ms": ms, "traffic": traffic_per_launch(kernel, prec, n_neigh, N)}
    if kernel in ("embedding_forward", "embedding_backward"):
        flop = n_neigh * (EMB_FWD_FLOP_PER_NEIGHBOUR if kernel == "embedding_forward" else EMB_BWD_FLOP_PER_NEIGHBOUR)
    elif kernel == "fitting":
        flop = N * FIT_FLOP_PER_ATOM
    else:
        flop = 0
    if mixed and kernel in ("embedding_forward", "embedding_backward"):
        tanh = n_neigh * TANH_PER_NEIGHBOUR
        sfu = (alu.get("tanh") or 0.0) / 1e12
        tens = pk.get("bf16_tflops", 1900.0)
        out.update({"bound": "alu", "achieved": tanh / t / 1e12, "peak": sfu, "unit": "Ttanh/s",
                    "frac": (tanh / t / 1e12 / sfu) if sfu else None,
                    "peak_source": "measured: dp_measure_peak(tanh.approx.f32) on this device, this run",
                    "tensor": {"achieved": flop / t / 1e12, "peak": tens, "unit": "TFLOP/s",
                               "frac": flop / t / 1e12 / tens, "peak_source": f"{src} bf16 burst"}})
        return out
    if mixed and kernel == "fitting":
        tens = pk.get("bf16_tflops", 1900.0)
        out.update({"bound": "tensor", "achieved": flop / t / 1e12, "peak": tens, "unit": "TFLOP/s",
                    "frac": flop / t / 1e12 / tens, "peak_source": f"{src} bf16 burst (fp16 runs at the bf16 rate)"})
        return out
    if kernel in ("format", "dE_dT", "descriptor"):
        bpa = hbm_bytes_per_atom(kernel, ntypes) if mixed else None
        ach = bpa * N / t / 1e9 if (bpa and t > 0) else None
        hbm = pk.get("hbm_gbs")
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": (ach / hbm) if (ach and hbm) else None, "peak_source": f"{src} hbm copy"})
        if bpa:
            out["bytes_per_atom"] = bpa
        return out
    key = "dfma" if prec == "fp64" else "ffma"
    peak = (alu.get(key) or 0.0) / 1e12
    ach = flop / t / 1e12
    out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak if peak else None,
                "peak_source": f"measured: dp_measure_peak({key}) on this device, this run"})
    return out


def neighbour_count(m):
    nl, _ = m.get_nlist()
    return int((nl >= 0).sum().item())


def run_mine(args, world, rank, local):
    import torch
    import paper_2410_22867_gb300 as dp
    dp.build()
    s, w, v0 = load_workload(args.workload)
    N = s.natoms
    prec = args.precision
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        m = dp.DPModel(w, prec, max_atoms=N, skin=2.0, stream=stream)
        x = torch.tensor(s.coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=REBUILD)
        m.verlet(st, DT_FS, args.warmup, capture_graph=True)  # warm-up (builds lists, captures graphs)
        st.resume = 1
        n_neigh = neighbour_count(m)
        launches0 = m.kernel_launches()
        clocks = ClockSampler(local)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        ev0.record(stream)
        m.verlet(st, DT_FS, args.steps, capture_graph=True, sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ck = clocks.stop()
        m.sync()
        t_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
        launches = m.kernel_launches() - launches0
        ms_step = t_ms / args.steps
        value = aggregate_rate(world, N, args.steps, t_ms)
        # [format, descriptor phase, fitting, embedding-backward phase, total, embedding forward
        #  kernel, embedding backward kernel] from events on the model's stream
        phases = m.phase_times(args.phase_repeats)
        if rank != 0:
            m.close()

    extra = {}
    if rank == 0:
        alu = measured_peaks(dp)
        kern = kernel_times(phases)
        dominant = max(kern, key=kern.get)
        extra["roofline"] = roofline(prec, dominant, kern[dominant], N, n_neigh, alu, w.ntypes)
        extra["rooflines"] = {k: roofline(prec, k, v, N, n_neigh, alu, w.ntypes) for k, v in kern.items()}
        extra["kernels_ms"] = {k: round(v, 4) for k, v in kern.items()}
        extra["measured_peaks"] = {"values": alu, "units": {"tanh": "1/s", "ex2": "1/s", "rcp": "1/s",
                                                            "ffma": "FLOP/s", "dfma": "FLOP/s"},
                                   "how": "dp_measure_peak: 8 blocks x 256 threads per SM, 8 dependent chains per "
                                          "thread, CUDA events, best of 3 after a warm-up"}
        # precision ladder: every precision on the copper and water boxes
        if args.ladder_steps > 0:
            extra["ladder"] = ladder(args, stream, alu)
        # FP64 comparison (speed and error) on the same configuration
        if not args.no_fp64 and prec != "fp64":
            lad = extra.get("ladder", {}).get(args.workload)
            if lad and prec in lad:
                f = lad["fp64"]
                extra["fp64"] = {"value": f["value"], "unit": f["unit"], "ms_per_step": f["ms_per_step"],
                                 "steps": f["steps"], "error_vs_fp64_gpu": lad[prec]["error_vs_fp64_gpu"],
                                 "from": "ladder"}
            else:
                extra["fp64"] = fp64_compare(args, s, w, v0, m, stream)
        # errors of every precision on the normalised models (environment statistics, O(1) rows)
        if args.ladder_steps > 0:
            extra["normalised_errors"] = normalised_errors(stream)
        # latency: the 192-atom water box, microseconds per MD step
        if args.latency_steps > 0:
            extra["latency"] = latency_leg(args, stream)
        # the water box of the same model family
        if args.water_steps > 0 and args.workload != "water12k":
            extra["water"] = water_leg(args, stream)
        # batched replicas (dp_md_run_batch)
        if args.batch_steps > 0:
            extra["batch"] = batch_leg(args, stream)
        # end-to-end through the public API with host buffers
        extra["e2e"] = e2e(m, s, stream, args.e2e_steps)
        # CPU oracle baseline: all host cores, and one core
        try:
            import oracle
            oracle.build()
            ncores = len(os.sched_getaffinity(0))
            oracle.set_threads(ncores)
            rate, cores, sample, _ = oracle_rate(args.workload, nsteps=1)
            oracle.set_threads(1)
            rate1, _, _, _ = oracle_rate(args.workload, nsteps=1)
            oracle.set_threads(ncores)
            extra["cpu_baseline"] = {"value": rate, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                                     "sample": sample, "one_core": {"value": rate1, "cores": 1}}
        except Exception as e:  # noqa: BLE001
            extra["cpu_baseline"] = {"value": None, "unit": "atom-steps/s", "cores": 0, "kind": "oracle",
                                     "sample": f"unavailable: {e}"}
        dtype = {"fp64": "f64", "fp32": "f32", "mix_bf16": "bf16", "mix_fp16": "f16"}[prec]
        line = {"metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": WORKLOADS[args.workload], "precision": prec, "natoms": N, "dt_fs": DT_FS,
                           "rebuild_every": REBUILD, "real_neighbours": n_neigh,
                           "l2": "working set per step > 1 GB, larger than the 129 MB L2; no flush",
                           "parallelism": "replicas" if world > 1 else "1 GPU"},
                "ns_per_day": (1e3 / ms_step) * DT_FS * 86400 * 1e-6,
                "gpu_launches": launches, "clocks": ck,
                "context": {"paper_ns_per_day": 149.0, "paper_prior_ns_per_day": 4.7,
                            "paper_hardware": "12,000 Fugaku A64FX nodes, 0.54 M atoms Cu, dt 1 fs (context only)"}}
        line.update(extra)
        print(json.dumps(line), flush=True)


TAB_INTERVALS = 256


def md_rate(w, s, v0, prec, stream, steps, dt=DT_FS, warm=3, tabulate=0):
    """NVE MD throughput of one box (graph replay); returns (ms per step, model kept open).
    tabulate > 0: the embedding nets replaced by tables of that many intervals (dp_tabulate)."""
    import torch
    import paper_2410_22867_gb300 as dp
    with torch.cuda.stream(stream):
        m = dp.DPModel(w, prec, max_atoms=s.natoms, skin=2.0, stream=stream)
        if tabulate:
            m.tabulate(tabulate)
        x = torch.tensor(s.coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=REBUILD)
        m.verlet(st, dt, warm, capture_graph=True)
        st.resume = 1
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        m.verlet(st, dt, steps, capture_graph=True, sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        m.sync()
    return ev0.elapsed_time(ev1) / steps, m


def force_errors(out, ref):
    """Error of one force evaluation against the FP64 GPU path: absolute and relative."""
    import torch
    dF = out["forces"] - ref["forces"]
    rmse = float(torch.sqrt((dF ** 2).mean()).item())
    rms = float(torch.sqrt((ref["forces"] ** 2).mean()).item())
    N = out["forces"].shape[0]
    return {"force_rmse_eV_per_A": rmse, "force_rms_eV_per_A": rms, "force_rel_rmse": rmse / rms if rms else None,
            "energy_eV_per_atom": abs(out["energy"].item() - ref["energy"].item()) / N,
            "max_atom_energy_eV": float((out["atom_energy"] - ref["atom_energy"]).abs().max().item())}


def ladder(args, stream, alu):
    """Every precision on the 131,072-atom copper box and the 12,288-atom water box: MD
    throughput (ns/day at 0.5 fs; copper also run at the paper's 1.0 fs), the dominant kernel's
    roofline, and the error of one force evaluation against the FP64 GPU path."""
    import torch
    out = {}
    for wl in ("cu131k", "water12k"):
        s, w, v0 = load_workload(wl)
        x = torch.tensor(s.coords, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        ref = None
        res = {}
        for prec in ("fp64", "fp32", "mix_bf16", "mix_fp16"):
            steps = args.ladder_steps if prec != "fp64" else max(2, args.ladder_steps // 10)
            if wl == "water12k":
                steps = min(steps, args.water_steps or steps)  # the window stays before the first collapse
            ms, m = md_rate(w, s, v0, prec, stream, steps)
            n_neigh = neighbour_count(m)
            ph = m.phase_times(3)
            kern = kernel_times(ph)
            dom = max(kern, key=kern.get)
            with torch.cuda.stream(stream):
                r = m.compute(x, t, s.box)
            e = {"value": s.natoms / (ms * 1e-3), "unit": "atom-steps/s", "ms_per_step": ms, "steps": steps,
                 "ns_per_day_0.5fs": (1e3 / ms) * 0.5 * 86400 * 1e-6,
                 "roofline": roofline(prec, dom, kern[dom], s.natoms, n_neigh, alu, w.ntypes),
                 "kernels_ms": {k: round(v, 4) for k, v in kern.items()}}
            if prec == "fp64":
                ref = {k: v.clone() for k, v in r.items()}
            else:
                e["error_vs_fp64_gpu"] = force_errors(r, ref)
            res[prec] = e
            m.close()
        if wl == "cu131k":
            ms, m = md_rate(w, s, v0, "mix_fp16", stream, args.ladder_steps, dt=1.0)
            m.close()
            res["mix_fp16_dt1fs"] = {"value": s.natoms / (ms * 1e-3), "unit": "atom-steps/s", "ms_per_step": ms,
                                     "ns_per_day_1fs": (1e3 / ms) * 1.0 * 86400 * 1e-6, "steps": args.ladder_steps}
        # the compressed model: embedding nets replaced by quintic tables (dp_tabulate)
        for prec in ("fp32", "mix_fp16"):
            steps = min(args.ladder_steps, args.water_steps or args.ladder_steps) if wl == "water12k" \
                else args.ladder_steps
            ms, m = md_rate(w, s, v0, prec, stream, steps, tabulate=TAB_INTERVALS)
            ph = m.phase_times(3)
            kern = kernel_times(ph)
            with torch.cuda.stream(stream):
                r = m.compute(x, t, s.box)
            res[prec + "_tabulated"] = {"value": s.natoms / (ms * 1e-3), "unit": "atom-steps/s", "ms_per_step": ms,
                                        "steps": steps, "ns_per_day_0.5fs": (1e3 / ms) * 0.5 * 86400 * 1e-6,
                                        "intervals": TAB_INTERVALS,
                                        "kernels_ms": {k: round(v, 4) for k, v in kern.items()},
                                        "error_vs_fp64_gpu": force_errors(r, ref)}
            m.close()
        out[wl] = {"workload": WORKLOADS[wl], **res}
    return out


def normalised_errors(stream):
    """Error of every precision against the FP64 GPU path on the normalised models: the
    per-type environment statistics of each system (written by the oracle script under
    tests/golden) and a gain of 10 on the fitting input layer, so the environment rows are
    O(1) and the forces have the scale of a trained model."""
    import torch
    import paper_2410_22867_gb300 as dp
    from paper_2410_22867_gb300 import synth
    with open(os.path.join(ROOT, "tests", "golden", "env_stats.json")) as f:
        stats = json.load(f)
    out = {}
    for wl, kind in (("cu131k", "copper"), ("water12k", "water")):
        s, _, _ = load_workload(wl)
        w = synth.normalised_weights(kind, stats)
        x = torch.tensor(s.coords, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        ref = None
        res = {}
        with torch.cuda.stream(stream):
            for prec, tab in (("fp64", 0), ("fp32", 0), ("mix_bf16", 0), ("mix_fp16", 0), ("fp64", TAB_INTERVALS),
                              ("fp32", TAB_INTERVALS), ("mix_fp16", TAB_INTERVALS)):
                m = dp.DPModel(w, prec, max_atoms=s.natoms, stream=stream)
                if tab:
                    m.tabulate(tab)
                r = m.compute(x, t, s.box)
                if prec == "fp64" and not tab:
                    ref = {k: v.clone() for k, v in r.items()}
                    res["fp64_force_rms_eV_per_A"] = float(torch.sqrt((ref["forces"] ** 2).mean()).item())
                else:
                    res[prec + ("_tabulated" if tab else "")] = force_errors(r, ref)
                m.close()
        out[wl] = res
    return out


def batch_leg(args, stream):
    """256 water replicas of 32..2048 molecules (96..6,144 atoms each) advanced together by
    dp_md_run_batch: one launch per phase for all boxes, replayed from a CUDA graph."""
    import torch
    import paper_2410_22867_gb300 as dp
    from paper_2410_22867_gb300 import synth
    reps = synth.water_replicas(256, 4)
    w = synth.water_weights(1001)
    coords, types, offs, boxes = synth.concat(reps)
    v0 = np.concatenate([synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 1000 + r) for r, s in enumerate(reps)])
    N = len(types)
    with torch.cuda.stream(stream):
        m = dp.DPModel(w, args.precision, max_atoms=N, max_replicas=len(reps), skin=2.0, stream=stream)
        x = torch.tensor(coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        t = torch.tensor(types, device="cuda")
        st = m.md_state(x, v, t, boxes, reps[0].masses(), atom_offsets=offs, rebuild_every=REBUILD)
        keep = m.md_run_batch(st, DT_FS, 3)
        e_start = (keep["potential"] + keep["kinetic"]).cpu().numpy().copy()
        st.resume = 1
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        m.md_run_batch(st, DT_FS, args.batch_steps, sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        m.sync()
        ms = ev0.elapsed_time(ev1) / args.batch_steps
        e_end = (keep["potential"] + keep["kinetic"]).cpu().numpy()
        nat = np.diff(np.asarray(offs))
        drift = np.abs(e_end - e_start) / nat
        grids = m.autotune(0)  # launch grids the autotuner chose on the first call
        m.close()
    return {"workload": f"256 H2O replicas, 32..2048 molecules each ({N} atoms), r_c 6 A, sel 46/92, "
                        f"NVE dt 0.5 fs, rebuild every {REBUILD} steps",
            "value": N / (ms * 1e-3), "unit": "atom-steps/s", "ms_per_step": ms, "steps": args.batch_steps,
            "replicas": len(reps), "natoms": N,
            "energy_drift_eV_per_atom": {"max": float(drift.max()), "mean": float(drift.mean()),
                                         "over_steps": args.batch_steps},
            "autotuned_grids": dict(zip(["embedding_forward", "embedding_backward", "dE_dT", "descriptor"], grids))}


def latency_leg(args, stream):
    """Latency of one MD step on the smallest workload, 64 H2O (192 atoms): microseconds per
    step with graph replay (each step = half kick, drift, list filter or rebuild, force
    evaluation, half kick), and the kernels launched per step."""
    import torch
    import paper_2410_22867_gb300 as dp
    from paper_2410_22867_gb300 import synth
    s = synth.water_box(64, 0)
    w = synth.water_weights(1001)
    v0 = synth.maxwell_boltzmann(s.masses()[s.types], 300.0, 77)
    out = {"workload": "64 H2O (192 atoms), r_c 6 A, sel 46/92, NVE dt 0.5 fs, rebuild every 10 steps",
           "steps": args.latency_steps}
    for prec in ("mix_fp16", "fp32", "fp64"):
        with torch.cuda.stream(stream):
            m = dp.DPModel(w, prec, max_atoms=s.natoms, skin=2.0, stream=stream)
            x = torch.tensor(s.coords, device="cuda")
            v = torch.tensor(v0, device="cuda")
            t = torch.tensor(s.types, device="cuda")
            st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=REBUILD)
            m.verlet(st, DT_FS, 3, capture_graph=True)
            st.resume = 1
            k0 = m.kernel_launches()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            m.verlet(st, DT_FS, args.latency_steps, capture_graph=True, sync=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            m.sync()
            us = ev0.elapsed_time(ev1) * 1e3 / args.latency_steps
            kernels = (m.kernel_launches() - k0) / args.latency_steps
            ph = m.phase_times(10)
            m.close()
        out[prec] = {"us_per_step": us, "kernels_per_step": kernels,
                     "ns_per_day_0.5fs": (1e6 / us) * 0.5 * 86400 * 1e-6, "atom_steps_per_s": s.natoms / (us * 1e-6),
                     "phases_us": {k: round(v * 1e3, 1) for k, v in kernel_times(ph).items()}}
    return out


def water_leg(args, stream):
    """Throughput of the 4096-H2O box (12,288 atoms) in the same precision: MD with graph
    replay; the window stays before the first random-weight collapse (step ~31)."""
    import torch
    import paper_2410_22867_gb300 as dp
    s, w, v0 = load_workload("water12k")
    with torch.cuda.stream(stream):
        m = dp.DPModel(w, args.precision, max_atoms=s.natoms, skin=2.0, stream=stream)
        x = torch.tensor(s.coords, device="cuda")
        v = torch.tensor(v0, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        st = m.md_state(x, v, t, s.box, s.masses(), rebuild_every=REBUILD)
        m.verlet(st, DT_FS, 3)
        st.resume = 1
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        m.verlet(st, DT_FS, args.water_steps, capture_graph=True, sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        m.sync()
        ms = ev0.elapsed_time(ev1) / args.water_steps
        m.close()
    return {"workload": WORKLOADS["water12k"], "value": s.natoms / (ms * 1e-3), "unit": "atom-steps/s",
            "ms_per_step": ms, "ns_per_day": (1e3 / ms) * DT_FS * 86400 * 1e-6, "steps": args.water_steps}


def fp64_compare(args, s, w, v0, m_mixed, stream):
    import torch
    import paper_2410_22867_gb300 as dp
    N = s.natoms
    with torch.cuda.stream(stream):
        m64 = dp.DPModel(w, "fp64", max_atoms=N, stream=stream)
        x = torch.tensor(s.coords, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        r64 = m64.compute(x, t, s.box)
        rmx = m_mixed.compute(x, t, s.box)
        dF = (rmx["forces"] - r64["forces"])
        rmse = float(torch.sqrt((dF ** 2).mean()).item())
        rms = float(torch.sqrt((r64["forces"] ** 2).mean()).item())
        de = abs(rmx["energy"].item() - r64["energy"].item()) / N
        dEi = float((rmx["atom_energy"] - r64["atom_energy"]).abs().max().item())
        xx = torch.tensor(s.coords, device="cuda")
        vv = torch.tensor(v0, device="cuda")
        st = m64.md_state(xx, vv, t, s.box, s.masses(), rebuild_every=REBUILD)
        m64.verlet(st, DT_FS, 1, capture_graph=True)
        st.resume = 1
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        m64.verlet(st, DT_FS, args.fp64_steps, capture_graph=True, sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        m64.sync()
        ms = ev0.elapsed_time(ev1) / args.fp64_steps
        m64.close()
    rate = N / (ms * 1e-3)
    return {"value": rate, "unit": "atom-steps/s", "ms_per_step": ms, "steps": args.fp64_steps,
            "error_vs_fp64_gpu": {"force_rmse_eV_per_A": rmse, "force_rms_eV_per_A": rms,
                                  "force_rel_rmse": rmse / rms if rms > 0 else None,
                                  "energy_eV_per_atom": de, "max_atom_energy_eV": dEi}}


def e2e(m, s, stream, nsteps):
    """dp_compute through the public API with the coordinates in pinned host memory:
    every step copies coordinates H2D, evaluates (rebuilding the list), and reads
    energy and forces back D2H."""
    import torch
    N = s.natoms
    host_x = torch.tensor(s.coords, dtype=torch.float64).pin_memory()
    host_F = torch.empty(N, 3, dtype=torch.float64).pin_memory()
    host_E = torch.empty(1, dtype=torch.float64).pin_memory()
    with torch.cuda.stream(stream):
        x = torch.empty(N, 3, dtype=torch.float64, device="cuda")
        t = torch.tensor(s.types, device="cuda")
        out = m.compute(x.copy_(host_x, non_blocking=True), t, s.box)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nsteps):
            x.copy_(host_x, non_blocking=True)
            out = m.compute(x, t, s.box, sync=False)
            host_F.copy_(out["forces"], non_blocking=True)
            host_E.copy_(out["energy"], non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        m.sync()
    return {"value": N * nsteps / dt, "unit": "atom-steps/s", "h2d_bytes_per_step": 24 * N,
            "d2h_bytes_per_step": 24 * N + 8, "steps": nsteps,
            "path": "dp_compute per step (list rebuilt every call), coordinates from pinned host memory"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="cu131k", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["mix_bf16", "mix_fp16", "fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--phase-repeats", type=int, default=10)
    ap.add_argument("--batch-steps", type=int, default=22)  # + 3 warm-up: before the first collapse (step ~35)
    ap.add_argument("--water-steps", type=int, default=20)  # + 4 warm-up: before the first collapse (step ~31)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--latency-steps", type=int, default=25, help="timed MD steps of the 192-atom latency leg "
                                                                   "(0 skips it)")
    ap.add_argument("--ladder-steps", type=int, default=20, help="timed MD steps per precision of the ladder "
                                                                  "(FP64: a tenth, at least 2); 0 skips the ladder")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.precision is None:
        args.precision = os.environ.get("DP_BENCH_PRECISION", "mix_fp16")
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_mine(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
