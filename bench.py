#!/usr/bin/env python
"""Benchmark of the EAM lattice-list MD step on one GB300 (or N replicas).

Workload (the roofline headline case): bcc Fe-like crystal of 300 x 300 x 300
cells (54,000,000 atoms), Finnis-Sinclair/Morse EAM tabulated on 5000-knot
splines, an equilibrated crystal at 600 K (Gaussian displacements of
0.1 A sqrt(T / 600 K) per component, Maxwell velocities, seed 2), a 10 keV
knock-on atom along a seeded direction, adaptive timestep (1 fs cap, 0.02 A max displacement),
hash update every 10 steps, FP32 force path with FP64 integration.  A bench
"step" is one full MD step (kick/drift, hash update, density, embedding,
force, kick, next timestep).  The state (~8 GB) is far larger than L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the baseline arm).
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_2107_07866_gb300 import synth  # noqa: E402

METRIC = "EAM atom-steps/s at 54M atoms, FP32-force vs FP64 path; % HBM roofline"
UNIT = "atom-steps/s"

# Algorithmic work per site and pass: FP32 flops with
# FMA = 2, counted from the method's arithmetic: 112 offset candidates (the
# neighbour offset index out to rc + 2 skin), 58 pairs inside rc per atom of
# the crystal.
CAND, PAIRS = 112, 58
FLOP_CAND, FLOP_DENS_PAIR, FLOP_FORCE_PAIR = 11, 21, 41
FLOPS_FORCE_SITE = CAND * FLOP_CAND + PAIRS * FLOP_FORCE_PAIR
FLOPS_DENS_SITE = CAND * FLOP_CAND + PAIRS * FLOP_DENS_PAIR
# FP32 peak: 152 SMs x 128 lanes x 2 flops (FMA) x 2.07 GHz max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic HBM bytes per atom-step of the whole FP32-force step:
#   kick/drift: read u64, v64, a32 (60), write u64, v64, u32 shadow (60)
#   density:    read u32 (12), write F' (4) and the sparse-shell mask (8)
#   force:      read u32 (12), F' (4), mask (8), v64 (24); write v64 (24), a32 (12)
BYTES_STEP_FP32 = 120 + 24 + 84
BYTES_FORCE_SITE = 84
# DRAM traffic of the force pass (k_force_p) per launch at the 54M-atom
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by the kernel sources it was measured on.
NCU_FORCE_TRAFFIC = {"source_sha": "ed485315566d1dd6", "bytes_per_launch": 4.8495e9,
                     "note": "k_force_p<8,8,12> at 300^3 cells: 2.956e9 B read + 1.893e9 B written per launch "
                             "(mean of 3 launches), 89.8 B/site vs 84 algorithmic"}
# Shared-memory (LSU) and texture wavefronts per site of the two gathers from
# one ncu capture of the 2M-atom case (equilibrated crystal), same keying;
# the L1 data pipe serves one wavefront per SM per clock.
NCU_WAVEFRONTS = {"source_sha": "ed485315566d1dd6", "density": (27.4, 16.4), "force": (37.5, 23.6)}


def kernel_source_sha():
    """Hash of every CUDA source and header of the library (the ncu figures
    below are valid only for the sources they were captured on)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2107_07866_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "misa.h"), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [t.strip() for t in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


WORKLOADS = {
    # headline: the 54M-atom FP32-force cascade
    "c3": dict(n=300, T=600.0, seed=2, pka_eV=10000.0, dx_max=0.02, reassign=10, run_length=500,
               desc="300x300x300 cells (54,000,000 atoms), equilibrated at 600 K (seed 2), 10 keV PKA, FP32 forces, "
                    "adaptive dt (1 fs, 0.02 A), hash update every 10 steps; the timed steps end at step 500, the "
                    "cascade's run length"),
    # smaller cascade (parity-size check of the bench path)
    "c2": dict(n=100, T=600.0, seed=1, pka_eV=5000.0, dx_max=0.02, reassign=1, checkpoints=(0, 100),
               fp64_full=True, ra_scan=True,
               desc="100x100x100 cells (2,000,000 atoms), equilibrated at 600 K (seed 1), 5 keV PKA, adaptive dt, "
                    "hash update every step; FP32 and FP64 paths over the same steps from the same inputs, oracle "
                    "error at steps 0, 100 and the last (run with --steps 1000 for the configuration's length)"),
    # batched cascades: 64 uneven replicas in one handle, one launch per pass
    "c4": dict(n=None, nrep=64, seed=4, dx_max=0.02, reassign=10,
               desc="64 batched replicas, dims ~ U{20..60}^3 cells (seeded), equilibrated at 300-900 K, 1-5 keV PKA each, "
                    "FP32 forces, adaptive dt per replica, steps captured in a CUDA graph, autotuned tile"),
    # alloy: three atom types (Eq. eam_base and eam_force_ij with types)
    "alloy": dict(n=100, T=600.0, seed=3, pka_eV=5000.0, dx_max=0.02, reassign=10, nsp=3, fractions=(0.7, 0.2, 0.1),
                  desc="100x100x100 cells (2,000,000 atoms), three atom types (70/20/10 %), equilibrated at 600 K "
                       "(seed 3), 5 keV PKA, FP32 forces, adaptive dt, hash update every 10 steps"),
    # potential fitting: knot gradient of the force-matching + energy loss
    "c5": dict(n=16, nrep=16, seed=5, sigma=0.02, adjoint=True,
               desc="16 thermal snapshots of 16x16x16 cells (8,192 atoms each, 300-1500 K), targets from knots "
                    "scaled by 1 + N(0, 0.02^2); one step = loss + gradient w.r.t. 3 x 5000 knots, FP32 pair "
                    "arithmetic and bins, FP64 reduction"),
}


def thermal_sigma(T):
    """Displacement std (A per component) of the equilibrated crystal at T."""
    return 0.1 * math.sqrt(T / 600.0)


def equilibrated(nx, ny, nz, T, seed):
    """Positions and velocities of a crystal at temperature T: a cascade run
    starts from an equilibrated lattice, not from perfect sites."""
    x = synth.thermal_snapshot(nx, ny, nz, thermal_sigma(T), seed + 500)
    v = synth.maxwell_velocities(len(x), T, synth.MASS_FE, seed)
    return x, v


def batch_inputs(w):
    reps = synth.batch_replicas(w["nrep"], w["seed"])
    dims = [(r.nx, r.ny, r.nz) for r in reps]
    xv = [equilibrated(r.nx, r.ny, r.nz, r.T, r.seed) for r in reps]
    return reps, dims, np.concatenate([a for a, _ in xv]), np.concatenate([b for _, b in xv])


def init_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if os.environ.get("MISA_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier_max(ws, value):
    """Max of a per-rank value over all ranks (NCCL on the GPUs, gloo on the host)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def make_inputs(w, rank):
    n = w["n"]
    x, v = equilibrated(n, n, n, w["T"], w["seed"] + 1000 * rank)
    d = synth.random_direction(w["seed"] + 17 + 1000 * rank)
    return x, v, d


def cpu_baseline(target_s=12.0, max_cells=100):
    """The oracle as it stands (cell list, OpenMP on all host cores): velocity
    Verlet steps on a sub-box of the same crystal, potential and temperature,
    grown until the sample takes ~target_s.  atom-steps/s."""
    from oracle import oracle as O
    O.build()
    pot = synth.potential()
    op = O.Pot(pot)
    n = 20
    while True:
        x, v = equilibrated(n, n, n, 600.0, 2)
        L = synth.box(n, n, n)
        t0 = time.perf_counter()
        _, _, a, _, _ = O.md_run(op, x, v, L, synth.MASS_FE, 1.0, 0.02, 1, mode=1)
        t1 = time.perf_counter()
        # the first call also evaluates the initial forces (2 force passes);
        # time a clean second step
        t2 = time.perf_counter()
        O.md_run(op, x, v, L, synth.MASS_FE, 1.0, 0.02, 1, mode=1, a=a)
        t3 = time.perf_counter()
        dt = t3 - t2
        if dt * 4 >= target_s or n >= max_cells:
            steps = max(1, int(target_s / max(dt, 1e-3)))
            t4 = time.perf_counter()
            O.md_run(op, x, v, L, synth.MASS_FE, 1.0, 0.02, steps, mode=1, a=a)
            t5 = time.perf_counter()
            val = len(x) * steps / (t5 - t4)
            return {"value": val, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                    "sample": f"{steps} velocity-Verlet steps of a {n}x{n}x{n}-cell ({len(x)}-atom) box of the same "
                              f"crystal, potential and temperature (FP64 cell-list oracle; its cost per atom-step "
                              f"does not depend on box size)", "seconds": t5 - t4}
        n = min(max_cells, int(n * 1.6))


def fitting_inputs(w, rank=0):
    pot = synth.potential()
    target = pot.scaled(*synth.knot_perturbation(pot.n, w["sigma"], w["seed"] + 1000 * rank))
    _, snaps = synth.fitting_snapshots(w["nrep"], w["n"], w["seed"] + 1000 * rank)
    return pot, target, snaps


def oracle_grad_rate(w, n_snap=None, seconds=None):
    """The oracle's loss gradient (target forces + gradient per snapshot) on
    n_snap snapshots, or on as many as fit in ``seconds``; returns
    (full-set gradient evaluations/s, snapshots done, seconds, cores).  The
    oracle's gradient is a serial loop, so the whole sample runs on one core."""
    from oracle import oracle as O
    O.build()
    pot, target, snaps = fitting_inputs(w)
    op, ot = O.Pot(pot), O.Pot(target)
    n = w["n"]
    L = synth.box(n, n, n)
    t0 = time.perf_counter()
    k = 0
    while True:
        xs = snaps[k % len(snaps)]
        _, _, e_, f_ = O.eam(ot, xs, L, mode=1, nthreads=1)
        O.loss_grad(op, xs, L, f_, e_.sum(), mode=1)
        k += 1
        el = time.perf_counter() - t0
        if (n_snap is not None and k >= n_snap) or (seconds is not None and el > seconds):
            break
    return k / len(snaps) / el, k, el, 1


def run_reference_adjoint(args, ws):
    w = WORKLOADS[args.workload]
    oracle_grad_rate(w, n_snap=max(1, args.warmup // 3))
    val, k, el, cores = oracle_grad_rate(w, n_snap=args.steps)
    unit = "gradient evaluations/s"
    line = {"impl": "reference", "metric": "gradient evaluations/s (loss + d loss / d knots over the snapshot set)",
            "value": val, "unit": unit, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"oracle sample: one snapshot per step of the {args.workload} workload "
                                   f"({w['desc']}), scaled to the {w['nrep']}-snapshot evaluation", "cache": "cpu"},
            "cpu_baseline": {"value": val, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"{k} snapshots (target forces + gradient each)"},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_alloy(args, ws):
    """The oracle's alloy evaluation (densities, energies, forces) on a
    bounded sample of the alloy workload; it has no alloy MD loop, so one
    step is one force evaluation of the sample."""
    w = WORKLOADS[args.workload]
    from oracle import oracle as O
    O.build()
    al = synth.alloy_potential(w["nsp"])
    oal = O.Alloy(al)
    n = args.ref_cells
    x, _ = equilibrated(n, n, n, w["T"], w["seed"])
    t = synth.random_types(len(x), w["fractions"], w["seed"] + 77)
    L = synth.box(n, n, n)
    for _ in range(max(1, args.warmup // 3)):
        O.eam_alloy(oal, x, t, L, mode=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.eam_alloy(oal, x, t, L, mode=1)
    el = time.perf_counter() - t0
    val = len(x) * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"oracle sample: {n}x{n}x{n} cells ({len(x)} atoms) of the {args.workload} "
                                   f"workload ({w['desc']}); one step = one alloy force evaluation", "cache": "cpu"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} alloy force evaluations of a {n}^3-cell box"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference(args):
    ws, rank, _ = init_dist()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    if w.get("adjoint"):
        return run_reference_adjoint(args, ws)
    if w.get("nsp"):
        return run_reference_alloy(args, ws)
    from oracle import oracle as O
    O.build()
    pot = synth.potential()
    op = O.Pot(pot)
    if w.get("nrep"):
        # batched workload: the oracle runs one replica-like box per sample
        rep = synth.batch_replicas(w["nrep"], w["seed"])[0]
        w = dict(w, T=rep.T, pka_eV=rep.pka_energy)
    # one bench step = one oracle MD step of a bounded sample of the workload:
    # a 24^3-cell box of the same crystal, potential, temperature and PKA
    n = args.ref_cells
    x, v = equilibrated(n, n, n, w["T"], w["seed"])
    O.insert_pka(v, synth.pka_atom(n, n, n), synth.MASS_FE, w["pka_eV"], synth.random_direction(w["seed"] + 17))
    L = synth.box(n, n, n)
    x, v, a, _, _ = O.md_run(op, x, v, L, synth.MASS_FE, 1.0, w["dx_max"], args.warmup, mode=1)
    t0 = time.perf_counter()
    x, v, a, _, _ = O.md_run(op, x, v, L, synth.MASS_FE, 1.0, w["dx_max"], args.steps, mode=1, a=a)
    el = time.perf_counter() - t0
    val = len(x) * args.steps / el
    cores = O.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"oracle sample: {n}x{n}x{n} cells ({len(x)} atoms) of the {args.workload} "
                                   f"workload ({w['desc']})", "cache": "cpu"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} MD steps of a {n}^3-cell box per run"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_adjoint(args):
    """Gradient evaluations/s of misa_loss_grad on the fitting workload."""
    import torch

    ws, rank, local = init_dist()
    torch.cuda.set_device(local)
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa

    w = WORKLOADS[args.workload]
    n, nrep = w["n"], w["nrep"]
    pot, target, snaps = fitting_inputs(w, rank)
    x = np.concatenate(snaps)
    natoms = len(x)
    dims = [(n, n, n)] * nrep
    N = 2 * n ** 3
    with misa.Sim(target, replicas=dims, precision="fp64") as t:
        t.set_state(x)
        Fref = t.forces()
        _, _, e = t.energies(per_atom=True)
        Eref = np.array([e[k * N:(k + 1) * N].sum() for k in range(nrep)])
    out = {}
    for prec in ("fp32", "fp64"):
        sim = misa.Sim(pot, replicas=dims, precision=prec)
        sim.set_state(x)
        Fd = torch.from_numpy(Fref).cuda()
        Ed = torch.from_numpy(Eref).cuda()
        gd = torch.empty(3 * pot.n, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            sim.loss_grad(Fd, Ed, grad=gd)
        l0 = sim.stats()["launches"]
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local) if prec == "fp32" else None
        if clk:
            clk.__enter__()
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            loss, _ = sim.loss_grad(Fd, Ed, grad=gd)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        if clk:
            clk.__exit__(None, None, None)
        el = barrier_max(ws, e0.elapsed_time(e1))
        launches = sim.stats()["launches"] - l0
        # e2e: knots, targets from host memory, gradient back to host
        kh = [torch.from_numpy(a.copy()).pin_memory() for a in (pot.f, pot.phi, pot.F)]
        Fh, Eh = torch.from_numpy(Fref).pin_memory(), torch.from_numpy(Eref).pin_memory()
        gh = torch.empty(3 * pot.n, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.set_tables(*kh)
            sim.loss_grad(Fh, Eh, grad=gh)
        el2 = barrier_max(ws, time.perf_counter() - t0)
        out[prec] = {"ms": el / args.steps, "value": ws * args.steps / (el / 1e3), "launches": launches,
                     "loss": loss, "grad": gd.cpu().numpy(), "e2e": ws * args.steps / el2,
                     "clocks": clk.summary() if clk else None}
        # central differences (h = 1e-6) of the FP64 loss on 32 seeded knots,
        # against the FP64 and the FP32 gradient (an FP32 loss cannot resolve
        # the step: its rounding is larger than the change)
        if prec == "fp64":
            g = out[prec]["grad"]
            g32_ = out["fp32"]["grad"]
            rng = np.random.default_rng(3)
            hot = np.flatnonzero(np.abs(g) > 1e-3 * np.abs(g).max())
            tabs = [pot.f.copy(), pot.phi.copy(), pot.F.copy()]
            errs, errs32 = [], []
            for k in rng.choice(hot, 32, replace=False):
                tb, j = divmod(int(k), pot.n)
                h = 1e-6 * max(1.0, abs(tabs[tb][j]))
                y0 = tabs[tb][j]
                tabs[tb][j] = y0 + h
                sim.set_tables(*tabs)
                lp, _ = sim.loss_grad(Fref, Eref, grad=np.empty(3 * pot.n))
                tabs[tb][j] = y0 - h
                sim.set_tables(*tabs)
                lm, _ = sim.loss_grad(Fref, Eref, grad=np.empty(3 * pot.n))
                tabs[tb][j] = y0
                fd = (lp - lm) / (2 * h)
                errs.append(abs(g[k] - fd) / np.abs(g).max())
                errs32.append(abs(g32_[k] - fd) / np.abs(g32_).max())
            out[prec]["fd_err"] = max(errs)
            out["fp32"]["fd_err"] = max(errs32)
        sim.close()
    g32, g64 = out["fp32"]["grad"], out["fp64"]["grad"]
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        val, k, _, cores = oracle_grad_rate(w, seconds=min(args.cpu_seconds, 20.0))
        cpu = {"value": val, "unit": "gradient evaluations/s", "cores": cores, "kind": "oracle",
               "sample": f"{k} snapshots of {N} atoms (target forces + loss gradient each), scaled to the "
                         f"{nrep}-snapshot evaluation"}
    if rank == 0:
        r32 = out["fp32"]
        line = {"metric": "gradient evaluations/s (loss + d loss / d knots over the snapshot set)",
                "value": r32["value"], "unit": "gradient evaluations/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r32["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w["desc"], "atoms": natoms, "parallelism": f"replicas{ws}",
                           "cache": "working set ~20 MB fits L2; each evaluation re-reads it (no flush)"},
                "roofline": None, "cpu_baseline": cpu,
                "e2e": {"value": r32["e2e"], "unit": "gradient evaluations/s",
                        "h2d_bytes_per_step": 8 * (3 * pot.n + 3 * natoms + nrep),
                        "d2h_bytes_per_step": 8 * (3 * pot.n + 1),
                        "note": "knots, target forces and energies from pinned host memory; gradient and loss back"},
                "gpu_launches": r32["launches"], "clocks": r32["clocks"],
                "fp64_path": {"value": out["fp64"]["value"], "ms_per_step": out["fp64"]["ms"],
                              "fd_rel_err": out["fp64"]["fd_err"]},
                "fd_rel_err": r32["fd_err"],
                "fd_note": "max over 32 seeded knots of |gradient - central difference of the FP64 loss "
                           "(h = 1e-6)| / max |gradient|",
                "fp32_vs_fp64_grad_rel": float(np.abs(g32 - g64).max() / np.abs(g64).max())}
        print(json.dumps(line))
    return 0


def norm_err(x, xo):
    """max_i |X_i - X_i^o| / max(|X_i^o|, rms |X^o|), the error norm of the
    parity tests (per-atom vectors or scalars)."""
    x = np.asarray(x, dtype=np.float64).reshape(len(x), -1)
    xo = np.asarray(xo, dtype=np.float64).reshape(len(xo), -1)
    mag = np.linalg.norm(xo, axis=1)
    rms = float(np.sqrt(np.mean(mag * mag))) if len(mag) else 0.0
    return float(np.max(np.linalg.norm(x - xo, axis=1) / np.maximum(mag, max(rms, 1e-300)))) if len(mag) else 0.0


def oracle_error(sim, pot, w, alloy=None, types=None, n_random=400, seed=7):
    """Error of the current state's densities, per-atom energies and forces
    against the FP64 oracle on the same positions, outside any timed region.
    Single boxes: the knock-on atom's neighbourhood (rc + 1 A), every
    run-away and n_random seeded atoms, evaluated one by one by the oracle;
    alloys: every atom (the oracle's alloy evaluation); batches: four seeded
    replicas, sampled the same way."""
    from oracle import oracle as O
    O.build()
    x = sim.positions()
    f = sim.forces()
    rho = sim.density()
    _, _, e = sim.energies(per_atom=True)
    _, ra = sim.site_map()
    rng = np.random.default_rng(seed)
    if alloy is not None:
        L = synth.box(*sim.replicas[0])
        r_o, _, e_o, f_o = O.eam_alloy(O.Alloy(alloy), x, types, L, mode=1)
        return {"rho": norm_err(rho, r_o), "E": norm_err(e, e_o), "F": norm_err(f, f_o),
                "atoms": len(x), "sample": "every atom"}
    op = O.Pot(pot)
    boxes = list(range(len(sim.replicas)))
    if len(boxes) > 1:
        boxes = sorted(int(b) for b in rng.choice(len(boxes), 4, replace=False))
    errs = {"rho": 0.0, "E": 0.0, "F": 0.0}
    count = 0
    for r in boxes:
        d, base, n = sim.replica_info(r)
        L = synth.box(*d)
        xr = x[base:base + n]
        pka = synth.pka_atom(*d)
        dd = xr - xr[pka]
        dd -= L * np.round(dd / L)
        near = np.flatnonzero(np.einsum("ij,ij->i", dd, dd) < (synth.RC + 1.0) ** 2)
        ra_r = ra[(ra >= base) & (ra < base + n)] - base
        t = np.unique(np.concatenate([near, ra_r, rng.choice(n, min(n, n_random), replace=False)]))
        r_o, e_o, f_o = O.eam_sample(op, xr, L, t)
        errs["rho"] = max(errs["rho"], norm_err(rho[base + t], r_o))
        errs["E"] = max(errs["E"], norm_err(e[base + t], e_o))
        errs["F"] = max(errs["F"], norm_err(f[base + t], f_o))
        count += len(t)
    errs["atoms"] = count
    errs["sample"] = ("knock-on neighbourhood (rc + 1 A), every run-away, "
                      f"{n_random} seeded atoms" + (f" in each of replicas {boxes}" if len(boxes) > 1 else ""))
    return errs


def run_timed(sim, stream, pre, K, checkpoints, sample):
    """pre untimed steps, then K steps timed with CUDA events on the
    library's stream, split at the checkpoint steps (absolute step counts)
    where sample(step) records the oracle error outside the timed region.
    Returns the summed device time (ms) of the K steps and the kernels the
    library launched for them."""
    import torch
    step0 = sim.stats()["step"]
    done = 0
    cps = sorted(set(int(c) for c in checkpoints))

    def advance(n):
        nonlocal done
        while n > 0:
            nxt = [c - (step0 + done) for c in cps if c - (step0 + done) > 0]
            k = min([n] + nxt)
            sim.step(k)
            done += k
            n -= k
            if step0 + done in cps:
                sample(step0 + done)

    if step0 in cps:
        sample(step0)
    advance(pre)
    torch.cuda.synchronize()
    total = 0.0
    launches = 0
    remaining = K
    while remaining > 0:
        nxt = [c - (step0 + done) for c in cps if c - (step0 + done) > 0]
        k = min([remaining] + nxt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = sim.stats()["launches"]
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
        launches += sim.stats()["launches"] - l0
        done += k
        remaining -= k
        if step0 + done in cps:
            sample(step0 + done)
    return total, launches


def run_gpu(args):
    import torch

    ws, rank, local = init_dist()
    torch.cuda.set_device(local)
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa

    w = WORKLOADS[args.workload]
    # issue-rate microbenchmarks of this device: the arithmetic roofline's
    # denominators (run before anything else, outside any timed region)
    peaks = misa.measure_peaks()
    fp32_peak = max(peaks["fp32_ffma_tflops"], peaks["fp32_ffma2_tflops"])
    pot = synth.potential()
    alloy = types = None
    if w.get("nsp"):
        alloy = synth.alloy_potential(w["nsp"])
        pot = alloy.species(0)  # grids of the alloy tables
        args.no_cpu = True      # the oracle's MD loop is single-type
    batched = w.get("nrep") is not None
    if batched:
        reps, dims, x, v = batch_inputs(w)
        natoms = len(v)
        n = None
        args.no_e2e = True
    else:
        n = w["n"]
        natoms = 2 * n ** 3
        x, v, d = make_inputs(w, rank)
        if alloy is not None:
            types = synth.random_types(natoms, w["fractions"], w["seed"] + 77 + 1000 * rank)

    def fresh(prec):
        if batched:
            s = misa.Sim(pot, replicas=dims, precision=prec, dt_max=1.0, dx_max=w["dx_max"],
                         reassign_period=w["reassign"], tile=args.tile)
            s.set_state(x, v)
            if not args.tile:
                s.retune()
            for r, rep in enumerate(reps):
                s.insert_pka_replica(r, rep.pka_energy, rep.pka_dir)
            return s
        s = misa.Sim(pot, n, precision=prec, dt_max=1.0, dx_max=w["dx_max"], reassign_period=w["reassign"],
                     tile=args.tile)
        if alloy is not None:
            s.set_species(alloy, types)
        s.set_state(x, v)
        if not args.tile:
            s.retune()  # tile shapes for the equilibrated crystal, not the perfect one
        s.insert_pka(-1, w["pka_eV"], d)
        return s

    want_err = rank == 0 and not args.no_oracle_err

    # ---- FP32-force path: the timed value ---------------------------------
    # The timed K steps end at the workload's run length (the C3 cascade is
    # timed at the state its 500 steps reach: untimed steps before it); the
    # oracle error is taken at the checkpoint steps, outside the timed time.
    sim = fresh("fp32")
    tile_used = sim.tile()
    tile_force = sim.tile_force()
    run_length = w.get("run_length", 0) if args.run_length is None else args.run_length
    pre = max(args.warmup, run_length - args.steps)
    checkpoints = [pre + args.steps] + [c for c in w.get("checkpoints", ()) if c <= pre + args.steps]
    errs32 = {}

    def sample32(step):
        if want_err:
            errs32[str(step)] = oracle_error(sim, pot, w, alloy, types)

    stream = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        barrier(ws)
        el_ms, gpu_launches = run_timed(sim, stream, pre, args.steps,
                                        [c for c in checkpoints if c < pre + args.steps] + [-1], sample32)
        barrier(ws)
    st1 = sim.stats()
    if want_err:
        errs32[str(st1["step"])] = oracle_error(sim, pot, w, alloy, types)
    clocks = clk.summary()
    # per-phase device time (events between the launches; separate, shorter run)
    sim.timing(True)
    sim.step(max(3, min(args.steps, 10)))
    phases, nsteps = sim.timing_get()
    sim.timing(False)
    el_max = barrier_max(ws, el_ms)
    value = natoms * ws * args.steps / (el_max / 1e3)

    # roofline of the dominant kernel (force pass) measured inside the timed region
    t_force = phases["force"] / max(nsteps, 1) / 1e3
    t_dens = phases["density"] / max(nsteps, 1) / 1e3
    ach = FLOPS_FORCE_SITE * natoms / t_force / 1e12
    traffic = None
    if NCU_FORCE_TRAFFIC["source_sha"] == kernel_source_sha() and args.workload == "c3":
        traffic = NCU_FORCE_TRAFFIC["bytes_per_launch"]  # captured on this workload only
    mp = measured_peaks()
    hbm_peak = mp.get("hbm_gbs", 6800.0)
    step_s = el_ms / 1e3 / args.steps
    sha = kernel_source_sha()
    l1 = None
    if NCU_WAVEFRONTS["source_sha"] == sha and alloy is None and not batched:
        # per-site wavefronts of the single-box crystal (2M-atom capture); not
        # carried over to the batch of small boxes; ncu's peak of the shared-
        # memory data pipe is one wavefront per SM per clock (at the sampled
        # SM clock)
        clk_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
        pipe = peaks["num_sms"] * clk_hz
        l1 = {k: {"lsu_wavefronts_per_site": NCU_WAVEFRONTS[k][0], "tex_wavefronts_per_site": NCU_WAVEFRONTS[k][1],
                  "lsu_frac": NCU_WAVEFRONTS[k][0] * natoms / (t * pipe)}
              for k, t in (("density", t_dens), ("force", t_force))}
    kname = "k_force_p (force pass)" if alloy is None else "k_force_pa (alloy force pass; flops counted as for one type)"
    roofline = {"bound": "alu", "kernel": kname, "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": traffic,
                "peak_note": "measured on this device by misa_measure_peaks: the faster of scalar FP32 FMA "
                             f"({peaks['fp32_ffma_tflops']:.1f}) and packed FP32x2 FMA "
                             f"({peaks['fp32_ffma2_tflops']:.1f} TFLOP/s) at {peaks['sm_clock_mhz']:.0f} MHz",
                "algorithmic_flops_per_site": FLOPS_FORCE_SITE,
                "force_ms": 1e3 * t_force, "density_ms": 1e3 * t_dens,
                "density_tflops": FLOPS_DENS_SITE * natoms / t_dens / 1e12,
                "step_hbm": {"bytes_per_atom_step": BYTES_STEP_FP32,
                             "achieved_gbs": BYTES_STEP_FP32 * natoms / step_s / 1e9,
                             "peak_gbs": hbm_peak, "frac": BYTES_STEP_FP32 * natoms / step_s / 1e9 / hbm_peak,
                             "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)"},
                "phase_ms_per_step": {k: v_ / max(nsteps, 1) for k, v_ in phases.items()},
                "l1_data_pipe": l1, "kernel_source_sha": sha, "measured_peaks": peaks}
    # the density pass with Newton's third law inside tiles, on the same
    # state (its own autotuned tile shape), beside the full-neighbour pass
    newton3 = None
    if alloy is None and not args.no_newton3:
        sim.set_density_variant(1)
        if not args.tile:
            sim.retune()
        sim.step(2)
        sim.timing(True)
        sim.step(max(3, min(args.steps, 10)))
        ph3, n3s = sim.timing_get()
        sim.timing(False)
        newton3 = {"density_ms": ph3["density"] / max(n3s, 1), "full_neighbour_density_ms": 1e3 * t_dens,
                   "tile": list(sim.tile()),
                   "speedup": 1e3 * t_dens / (ph3["density"] / max(n3s, 1)),
                   "note": "density pass with each in-tile dense-shell pair evaluated once (Sec. 4.2 halving), "
                           "pairs reaching outside the tile evaluated by the site; same state, steps after the timed ones"}
        sim.set_density_variant(0)
    stats_end = sim.stats()
    frenkel = [int(c) for c in sim.defects()]
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # ---- run-away load: per-phase times of the same box with 10^2..10^4
    # interstitial atoms (a developed cascade's run-away count) -------------
    ra_load = None
    if w.get("ra_scan") and not args.no_ra_scan:
        ra_load = []
        for nint in (100, 1000, 10000):
            s = misa.Sim(pot, n, precision="fp32", dt_max=1.0, dx_max=w["dx_max"], reassign_period=w["reassign"],
                         tile=args.tile, runaway_capacity=16384)
            xi = synth.interstitial_snapshot(n, n, n, thermal_sigma(w["T"]), nint, w["seed"] + 900)
            s.set_state(xi, v)
            if not args.tile:
                s.retune()
            s.step(3)
            s.timing(True)
            s.step(10)
            ph, ns_ = s.timing_get()
            s.timing(False)
            st_ = s.stats()
            ra_load.append({"interstitials": nint, "n_runaway": st_["n_runaway"], "status": st_["status"],
                            "ms_per_step": sum(ph.values()) / ns_,
                            "phase_ms_per_step": {k: v_ / ns_ for k, v_ in ph.items()}})
            s.close()
            del s
            torch.cuda.empty_cache()

    # ---- e2e through the C ABI with host buffers ----------------------------
    e2e = None
    if not args.no_e2e:
        s = misa.Sim(pot, n, precision="fp32", dt_max=1.0, dx_max=w["dx_max"], reassign_period=w["reassign"],
                     tile=args.tile)
        if alloy is not None:
            s.set_species(alloy, types)
        x_host = torch.from_numpy(x).pin_memory()
        v0 = v.copy()
        pka = synth.pka_atom(n, n, n)
        spd = math.sqrt(2.0 * w["pka_eV"] / synth.MASS_FE / synth.EV_PER_AMU_A2_FS2)
        v0[pka] = spd * d
        v_host = torch.from_numpy(v0).pin_memory()
        e_host = [torch.empty(natoms, dtype=torch.float64).pin_memory() for _ in range(2)]
        inner = max(10, w["reassign"])
        iters = max(10, args.e2e_iters)
        s.stage_state(x_host, v_host)
        s.set_state_staged()
        s.step(inner)
        s.energies(per_atom=True)
        s.energies_async(e_host[0])
        s.wait_outputs()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        s.stage_state(x_host, v_host)            # H2D of the first state
        for it in range(iters):
            s.set_state_staged()
            if it + 1 < iters:
                s.stage_state(x_host, v_host)    # H2D of the next state, beside this one's steps
            s.step(inner, energies=True)         # the last step also evaluates E_i
            # D2H of the state's per-atom energies E_i, beside the next state's
            # steps (two pinned buffers in turn)
            s.energies_async(e_host[it % 2])
        s.wait_outputs()
        torch.cuda.synchronize()
        el = barrier_max(ws, time.perf_counter() - t0)
        e2e = {"value": natoms * ws * inner * iters / el, "unit": UNIT,
               "h2d_bytes_per_step": 48 * natoms, "d2h_bytes_per_step": 8 * natoms + 16,
               "iterations": iters,
               "note": f"one e2e step = state (x, v) from pinned host memory + {inner} MD steps + the per-atom "
                       "energies E_i of the state reached (evaluated inside the last step's passes) back to "
                       "pinned host memory (two buffers in turn, copied beside the next state's steps); "
                       "each state is staged on the library's copy stream while the previous one is simulated"}
        s.close()
        del s
        torch.cuda.empty_cache()

    # ---- FP64 path on the same inputs -----------------------------------------
    fp64 = None
    if not args.no_fp64:
        s = fresh("fp64")
        errs64 = {}

        def sample64(step):
            if want_err:
                errs64[str(step)] = oracle_error(s, pot, w, alloy, types)

        k64 = args.fp64_steps if not w.get("fp64_full") else args.steps
        pre64 = 1 if not w.get("fp64_full") else pre
        cps64 = [c for c in w.get("checkpoints", ()) if w.get("fp64_full") and c < pre64 + k64] + [-1]
        with ClockSampler(local) as clk64:
            el64, _ = run_timed(s, stream, pre64, k64, cps64, sample64)
        if want_err:
            errs64[str(s.stats()["step"])] = oracle_error(s, pot, w, alloy, types)
        s.timing(True)
        s.step(1 if not w.get("fp64_full") else 3)
        ph64, n64 = s.timing_get()
        s.timing(False)
        t_gather = (ph64["density"] + ph64["force"]) / max(n64, 1) / 1e3
        ach64 = (FLOPS_DENS_SITE + FLOPS_FORCE_SITE) * natoms / t_gather / 1e12
        fp64 = {"value": natoms * k64 / (el64 / 1e3), "unit": UNIT, "steps": k64, "ms_per_step": el64 / k64,
                "start_step": pre64, "clocks": clk64.summary(),
                "fp64_pipe": {"kernels": "k_density + k_force (FP64 gathers)", "achieved_tflops": ach64,
                              "peak_tflops": peaks["fp64_dfma_tflops"], "frac": ach64 / peaks["fp64_dfma_tflops"],
                              "flops_per_site": FLOPS_DENS_SITE + FLOPS_FORCE_SITE,
                              "peak_note": "FP64 FMA issue rate measured on this device (misa_measure_peaks)"},
                "oracle_err": errs64 or None}
        s.close()
        del s
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": el_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w["desc"], "atoms": natoms, "parallelism": f"replicas{ws}",
                           "cache": f"state ~{148 * natoms / 1e9:.1f} GB >> 129 MB L2 (no flush needed)",
                           "timed_steps": [pre, pre + args.steps],
                           "tile": list(tile_used), "tile_force": list(tile_force)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "clocks": clocks, "fp64_path": fp64,
                "oracle_err": errs32 or None, "runaway_load": ra_load, "newton3_density": newton3,
                "end_state": {"step": stats_end["step"], "time_fs": stats_end["time"],
                              "n_runaway": stats_end["n_runaway"], "status": stats_end["status"],
                              "frenkel_pairs": sum(frenkel)}}
        print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="misa", choices=["misa", "reference"])
    ap.add_argument("--workload", default="c3", choices=list(WORKLOADS))
    ap.add_argument("--tile", type=int, default=0,
                    help="pin both gathers to tile shape K (1-based, see misa.tile_shapes()); 0: autotune")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-iters", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-cells", type=int, default=24)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--run-length", type=int, default=None,
                    help="step at which the timed steps end (default: the workload's; 0: right after warm-up)")
    ap.add_argument("--no-ra-scan", action="store_true", help="skip the run-away load scan (c2)")
    ap.add_argument("--no-newton3", action="store_true", help="skip the Newton-3 density-pass comparison")
    ap.add_argument("--no-oracle-err", action="store_true",
                    help="skip the oracle error of the benchmarked states (taken outside the timed region)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload].get("adjoint"):
        return run_adjoint(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
