#!/usr/bin/env python
"""Throughput of the MTP hot path on one GB300 (Matom*steps/s), one JSON line on stdout.

Workloads (--config, default C4):
  C4  fcc random solid solution of three species, a = 3.6 A, 64^3 conventional cells
      (1,048,576 atoms), sigma = 0.1 A, level-20 ternary MTP (m = 651), R_cut 5 A; active set
      chosen by MaxVol from the parameter rows of a 2048-atom companion snapshot
  C1  fcc unary 108 atoms, level 8 (m = 26), diagonally dominant active set
  C2  B2 binary 40^3 bcc cells (128,000 atoms), level 16 (no grade)
  C5  liquid-like quaternary, 2,097,152 atoms, R_cut 6 A, level 24 (m = 1636), diagonally
      dominant active set
One step = a real neighbor rebuild (positions are shifted each step) + energies, forces and
virial [+ per-atom grade gamma_i against the active set + compaction of the atoms with
gamma_i > 2], through the C ABI (mtp_build_neighbors, mtp_step).  The mixed path (FP32 with
FP64 sums) is the headline; the all-FP64 path is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config C4]

Under torchrun each rank runs its own independent configuration (weak scaling, no
collective); rank 0 prints.  The CPU leg (rank 0, N = 1) runs the FP64 oracle on the host
cores on sampled atoms of the benchmarked state: its timing is `cpu_baseline` and its results
give `errors_vs_oracle`.  --impl reference times the oracle alone on a bounded sample of the
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MTP energy+force Matom/s, mixed vs FP64 path on 1 GB300, at stated force error"
UNIT = "Matom*steps/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
N_SM = 152
FP32_LANES_PER_SM = 128

# per-config settings: default timed steps, FP64 steps, grade, active set, CPU-leg sample
CONFIGS = {
    "C1": {"steps": 200, "fp64_steps": 50, "grade": True, "active": "diag", "a_seed": 8, "sample": 108,
           "flush_l2": True},
    "C2": {"steps": 20, "fp64_steps": 2, "grade": False, "active": None, "sample": 24, "flush_l2": False},
    "C4": {"steps": 10, "fp64_steps": 2, "grade": True, "active": "maxvol", "sample": 16, "flush_l2": False},
    "C5": {"steps": 4, "fp64_steps": 1, "grade": True, "active": "diag", "a_seed": 9, "sample": 6,
           "flush_l2": False},
}
# companion snapshot of the MaxVol active set (C4): same lattice, independent displacements
COMPANION = {"seed": 444, "cells": 8, "eps": 1e-2}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the kernel on a 32^3-cell case of the C4 workload (131,072 atoms, inputs and outputs larger
# than L2); the traffic grows with the atom count, so a launch over N atoms moves bytes * N / atoms.
# Reported only while the kernel source is the one that was captured (same SHA-1).
MEASURED_TRAFFIC = {
    # the three kernels of the split per-neighborhood pass (k_moments + k_contract + k_adjoint)
    "site_pass": {"source": "paper_2304_13144_gb300/csrc/site_split.cu",
                  "sha1": "a96d5804ed0c32be967a076262210f102105bd9e",
                  "atoms": 131072, "bytes": (119737600 + 103305472) + (162931968 + 400208896) + (294791424 + 422636800)},
    "grade_tc_tf32x3": {"source": "paper_2304_13144_gb300/csrc/grade_tc.cu",
                        "sha1": "62e17e87b10aee78ab8b421d2404bd3a45d54efa",
                        "atoms": 131072, "bytes": 507654656 + 2607872},
}


def measured_traffic(kernel, n_atoms, config):
    rec = MEASURED_TRAFFIC.get(kernel)
    if rec is None or config != "C4":
        return None
    import hashlib
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        if hashlib.sha1(f.read()).hexdigest() != rec["sha1"]:
            return None
    return rec["bytes"] * n_atoms / rec["atoms"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------------------------
# workload
# ------------------------------------------------------------------------------------

def gauge_completion(rows, D):
    """The n_gauge null directions of the rows, scaled to the rows' magnitude, below them."""
    return np.vstack([rows, D / np.linalg.norm(D, axis=1, keepdims=True) * np.abs(rows).max()])


def companion_start(synth, m, g):
    comp = synth.fcc_ternary(seed=COMPANION["seed"], n=COMPANION["cells"])
    pick = synth.sample_atoms(COMPANION["seed"], len(comp["type"]), m - g)
    return comp, pick


def maxvol_active_set(api, synth, torch, desc, theta, sizes):
    """MaxVol active set (Section II.D) through the library: FP64 parameter rows of a companion
    snapshot (2048 atoms); start = m - n_gauge rows drawn without replacement plus the gauge
    completion; then swaps while some |(B A^-1)_ij| > 1 + eps over all companion rows."""
    m, g = sizes["n_params"], sizes["n_gauge"]
    comp, pick = companion_start(synth, m, g)
    model = api.mtp_load(desc, theta)
    b = api.Batch(comp)
    nb = api.mtp_build_neighbors(model, b)
    rows = api.mtp_param_rows(model, b, nb, "fp64")
    A0 = gauge_completion(rows[torch.tensor(pick, device="cuda")].cpu().numpy(), api.mtp_gauge_directions(desc, theta))
    api.mtp_set_active_set(model, torch.tensor(A0, device="cuda"))
    _, swaps = api.mtp_maxvol(model, rows, eps=COMPANION["eps"])
    A = api.mtp_get_active_set(model).cpu().numpy()
    return A, {"kind": "maxvol", "candidates": int(rows.shape[0]), "swaps": int(swaps), "eps": COMPANION["eps"]}


def conditioning(A):
    """2-norm condition number of A, and of A with unit-norm columns (the parameter columns of
    the rows have very different scales)."""
    s = np.linalg.svd(A, compute_uv=False)
    Ae = A / np.linalg.norm(A, axis=0, keepdims=True)
    se = np.linalg.svd(Ae, compute_uv=False)
    return float(s[0] / s[-1]), float(se[0] / se[-1])


# ------------------------------------------------------------------------------------
# algorithmic work (the roofline numerators)
# ------------------------------------------------------------------------------------

def site_flops(sizes, n_atoms, n_pairs, rows):
    """Algorithmic FP operations of one per-neighborhood pass (forward + adjoint [+ rows]).

    per pair: Chebyshev T, T' (8 N_Q) + Q, Q' (6 N_Q) + f, f' (4 N_rad N_Q) + powers (6 nu_max)
              + monomials (1 each) + moment accumulation (2 per component)
              + adjoint: g_mu and h (4 per component) + gradient (6 per monomial) + radial (2 N_rad + 9)
              [+ radial block of b_i: 2 N_rad N_Q]
    per atom: forward triples (3 each) + reverse (6 each) + energy (2 N_lin).
    """
    return sum(site_flops_parts(sizes, n_atoms, n_pairs, rows).values())


def site_flops_parts(sizes, n_atoms, n_pairs, rows):
    """The same operations by kernel of the three-kernel pass (each radial function counted once,
    in the moments kernel with its derivative, which the pair-adjoint kernel recomputes)."""
    nq, nr, nu, comps = 8, sizes["n_rad"], sizes["nu_max"], sizes["n_mom_comps"]
    n_mono = (nu + 1) * (nu + 2) * (nu + 3) // 6
    moments = 8 * nq + 6 * nq + 4 * nr * nq + 6 * nu + n_mono + 2 * comps
    adjoint = 4 * comps + 6 * n_mono + 2 * nr + 9 + (2 * nr * nq if rows else 0)
    contract = 9 * sizes["n_triples"] + 2 * sizes["n_lin"]
    return {"site_moments": moments * n_pairs, "site_contract": contract * n_atoms, "site_adjoint": adjoint * n_pairs}


# ------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------

def measure_train(api, synth, torch, steps=5, warmup=2):
    """One training step of eq. 7 (loss + gradient) on a 512-configuration batch of 8-256 atoms
    (fcc/bcc/hcp, random strains and species): targets from a seeded level-8 ternary teacher,
    a level-16 ternary student, weights w_e = 1, w_f = 0.01, w_s = 0."""
    bnp = synth.training_batch(seed=3)
    def model_for(lev, seed):
        desc = api.make_desc(3, lev)
        basis = api.mtp_describe_basis(desc)
        sz = api.mtp_describe(desc)
        th = synth.draw_theta(seed, 3, sz["n_rad"], 8, [sum(n for _, n in l) for l, _ in basis],
                              [len(l) for l, _ in basis], 2.0, 5.0, 42.0)
        return api.mtp_load(desc, th)
    teacher, student = model_for(8, 33), model_for(16, 34)
    b = api.Batch(bnp)
    nb = api.mtp_build_neighbors(teacher, b)
    ref = api.mtp_energy_forces_stress(teacher, b, nb, "fp64")
    out = {"configs": int(b.n_cfg), "atoms": int(b.n_atoms), "pairs": int(nb.size()[1]), "student_params": int(student.n_params)}
    for prec in ("mixed", "fp64"):
        for _ in range(warmup):
            api.mtp_train_step(student, b, nb, ref["energy"], ref["forces"], prec=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            loss, grad = api.mtp_train_step(student, b, nb, ref["energy"], ref["forces"], prec=prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"ms_per_step": ms, "configs_per_s": b.n_cfg / (ms / 1e3), "loss": float(loss.item())}
        # the same step captured once in a CUDA graph (workspaces sized by the warm-up) and replayed
        lossb = torch.empty(1, dtype=torch.float64, device="cuda")
        gradb = torch.empty(student.n_params, dtype=torch.float64, device="cuda")
        E, F = ref["energy"].contiguous(), ref["forces"].contiguous()

        def captured():
            api._check(api.lib().mtp_train_step(student.h, api.ctypes.byref(b.c), nb.h, api._prec(prec), api._ptr(E),
                                                api._ptr(F), None, 1.0, 0.01, 0.0, api._ptr(lossb), api._ptr(gradb),
                                                api._stream()))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            captured()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            captured()
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        msg = e0.elapsed_time(e1) / steps
        out[prec]["graph_ms_per_step"] = msg
        out[prec]["graph_loss_equal"] = bool(torch.equal(lossb, loss))
    return out


def measure_peaks(api):
    out = {}
    for kind in ("fp32_fma", "fp64_fma", "tf32_mma"):
        tf, ms = api.mtp_measure_peak(kind)
        out[kind] = {"tflops": tf, "ms": ms}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2304_13144_gb300 import api, configs, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    peaks, peaks_kind = load_peaks()
    cfg = CONFIGS[args.config]
    w = configs.workload(args.config)
    steps = args.steps if args.steps is not None else cfg["steps"]
    fp64_steps = args.fp64_steps if args.fp64_steps is not None else cfg["fp64_steps"]
    grade = cfg["grade"]

    measured = measure_peaks(api) if not args.no_peaks else None
    if args.cells and args.config == "C4":
        bnp = synth.fcc_ternary(seed=w.input_seed + rank, n=args.cells)   # smaller C4 cells (profiling)
    elif args.cells and args.config == "C5":
        # the 32,768-atom liquid cube repeated cells^3 times instead of 4^3 (profiling)
        bnp = synth.liquid_rsa(seed=w.input_seed + rank, n_atoms=32768 * args.cells ** 3, tiles=args.cells)
    else:
        bnp = w.inputs(w.input_seed + rank)
    desc, theta = w.desc(), w.theta()
    sizes = api.mtp_describe(desc)
    m = sizes["n_params"]
    model = api.mtp_load(desc, theta)
    active = None
    if cfg["active"] == "maxvol":
        A, active = maxvol_active_set(api, synth, torch, desc, theta, sizes)
    elif cfg["active"] == "diag":
        A = synth.diag_dominant(cfg["a_seed"], m)
        active = {"kind": "diagonally dominant G + diag(sum|G| + 1), G ~ N(0,1)", "seed": cfg["a_seed"]}
    if active is not None:
        active["cond2"], active["cond2_unit_columns"] = conditioning(A)
        api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    batch = api.Batch(bnp)
    N = batch.n_atoms
    pos0 = batch.pos.clone()
    nb = api.Neighbors()
    out = None
    api.mtp_build_neighbors(model, batch, nb)
    api.mtp_set_mixed_pass(model, args.mixed_pass)
    if args.split_shape:
        api.mtp_set_split_shape(model, *[int(x) for x in args.split_shape.split(",")])
    # the library's autotuner picks the per-neighborhood kernel's launch shape on this workload
    # (the FP64 kernel keeps its default shape above 10^6 atoms: one FP64 pass there takes seconds)
    tuned = {}
    if not args.no_autotune:
        tuned["mixed"] = api.mtp_autotune(model, batch, nb, "mixed")
        if N <= 1_100_000:
            tuned["fp64"] = api.mtp_autotune(model, batch, nb, "fp64")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda") if cfg["flush_l2"] else None

    def set_state(k):
        # deterministic shift so that every step rebuilds its neighbor list
        batch.pos.copy_(pos0 + 1e-4 * math.sin(0.7 * k + 0.1))

    def step(k, prec):
        nonlocal out
        set_state(k)
        api.mtp_build_neighbors(model, batch, nb)
        out = api.mtp_step(model, batch, nb, prec, threshold=2.0, out=out, grade=grade)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, n_steps, warmup, profile=False):
        for k in range(warmup):
            step(k, prec)
        barrier()
        if profile:
            api.mtp_profiler_read()
            api.mtp_profiler_enable(True)
        ms = 0.0
        if flush is None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(n_steps):
                step(warmup + k, prec)
            e1.record()
            barrier()
            ms = e0.elapsed_time(e1)
        else:
            # inputs smaller than L2: each step is timed on its own, after a write of a buffer
            # larger than L2 (the flush itself is outside the timed intervals)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
            for k in range(n_steps):
                flush.zero_()
                ev[k][0].record()
                step(warmup + k, prec)
                ev[k][1].record()
            barrier()
            ms = sum(a.elapsed_time(b) for a, b in ev)
        kern = None
        if profile:
            api.mtp_profiler_enable(False)
            kern = api.mtp_profiler_read()
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, kern

    clocks = ClockSampler(local)
    # ---- mixed path (headline), kernels traced with CUDA events on the launch stream ----
    clocks.start()
    ms_mixed, kern = timed("mixed", steps, args.warmup, profile=True)
    clk = clocks.stop()
    n_pairs = nb.size()[1]
    # ---- the same step on an unchanged configuration, reusing its neighbor list: eager and
    # replayed from a CUDA graph (the rebuild reads sizes back to the host, so it is not captured)
    for _ in range(2):
        out = api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out, grade=grade)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        out = api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out, grade=grade)
    e1.record()
    barrier()
    ms_reuse = e0.elapsed_time(e1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out, grade=grade)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out, grade=grade)
    for _ in range(2):
        graph.replay()
    barrier()
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    barrier()
    ms_graph = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms_reuse, ms_graph], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_reuse, ms_graph = (float(x) for x in t.tolist())

    # ---- both precisions at one fixed state (the errors below compare them) ----
    set_state(12345)
    state_pos = batch.pos.clone()
    api.mtp_build_neighbors(model, batch, nb)
    state = {}
    for prec in ("mixed", "fp64"):
        o = api.mtp_step(model, batch, nb, prec, threshold=2.0, grade=grade)
        o.update({k: v for k, v in api.mtp_energy_forces_stress_atoms(model, batch, nb, prec).items()
                  if k in ("site_energy", "site_virial")})
        state[prec] = o
    torch.cuda.synchronize()
    mixed_out, fp64_out = state["mixed"], state["fp64"]
    bound_diag = None
    if grade:
        # the mixed grade's per-atom allowance 1e-4 max(1, gamma) + 2^-20 S_i, with
        # S_i = max_p sum_k |b_ik| |(A^-1)_kp| the sensitivity of gamma_i to componentwise relative
        # errors of b_i, on a sample of atoms (FP64 rows and A^-1 from the library)
        smp = torch.tensor(synth.sample_atoms(99, N, min(N, 8192)), device="cuda")
        B64 = api.mtp_param_rows(model, batch, nb, "fp64", atoms=smp)
        S = (B64.abs() @ api.mtp_get_active_inverse(model).abs()).amax(dim=1)
        g64s, gmxs = fp64_out["gamma"][smp], mixed_out["gamma"][smp]
        ratio = (gmxs - g64s).abs() / (1e-4 * torch.clamp(g64s, min=1.0) + 2.0 ** -20 * S)
        bound_diag = {"sample_atoms": int(smp.numel()), "max_ratio": float(ratio.max().item()),
                      "atoms_above_bound": int((ratio > 1).sum().item()),
                      "sensitivity_over_gamma_median": float((S / torch.clamp(g64s, min=1.0)).median().item())}
        del B64
    # ---- FP64 path timing ----
    out = None
    ms_fp64, _ = timed("fp64", fp64_steps, 1)
    dF = (mixed_out["forces"] - fp64_out["forces"]).abs().max().item()
    dE = (mixed_out["energy"] - fp64_out["energy"]).abs().max().item() / N
    dW = ((mixed_out["virial"] - fp64_out["virial"]).abs().max() / fp64_out["virial"].abs().max()).item()
    err_fp64 = {"max_abs_dF_eV_per_A": dF, "abs_dE_per_atom_eV": dE, "rel_dW": dW,
                "max_abs_dV_eV": (mixed_out["site_energy"] - fp64_out["site_energy"]).abs().max().item()}
    if grade:
        g64 = fp64_out["gamma"]
        rel = (mixed_out["gamma"] - g64).abs() / torch.clamp(g64, min=1.0)
        f64 = set(fp64_out["flagged"][: int(fp64_out["n_flagged"].item())].tolist())
        fmx = set(mixed_out["flagged"][: int(mixed_out["n_flagged"].item())].tolist())
        err_fp64.update({"max_rel_dgamma": rel.max().item(), "atoms_rel_dgamma_above_1e-4": int((rel > 1e-4).sum().item()),
                         "gamma_allowance": bound_diag,
                         "n_flagged_fp64": len(f64), "n_flagged_mixed": len(fmx),
                         "flag_set_differences": len(f64 ^ fmx)})
        if active is not None:
            active["flagged_fraction"] = len(f64) / N
            active["gamma_quantiles_fp64"] = {"q50": 0, "q90": 0, "q99": 0, "max": 0}
            qs = np.quantile(g64.cpu().numpy(), [0.5, 0.9, 0.99, 1.0])
            active["gamma_quantiles_fp64"] = dict(zip(("q50", "q90", "q99", "max"), (float(q) for q in qs)))

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.empty_like(getattr(batch, k), device="cpu").pin_memory()
               for k in ("atom_offset", "pos", "type", "cell", "pbc")}
        for k in pin:
            pin[k].copy_(getattr(batch, k).cpu())
        keep = ("energy", "forces", "virial", "gamma", "n_flagged")
        host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in mixed_out.items()
                    if v is not None and k in keep}
        h2d = sum(t.numel() * t.element_size() for t in pin.values())
        d2h = sum(t.numel() * t.element_size() for t in host_out.values())
        out = None

        def e2e_step(k):
            nonlocal out
            for name in ("atom_offset", "type", "cell", "pbc", "pos"):
                getattr(batch, name).copy_(pin[name], non_blocking=True)
            batch.pos.add_(1e-4 * math.sin(0.3 * k))
            api.mtp_build_neighbors(model, batch, nb)
            out = api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out, grade=grade)
            for name, t in host_out.items():
                t.copy_(out[name], non_blocking=True)

        for k in range(2):
            e2e_step(k)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(args.e2e_steps):
            e2e_step(100 + k)
        e1.record()
        barrier()
        ms_e2e = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms_e2e], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        e2e = {"value": world * N * args.e2e_steps / (ms_e2e / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (and of the others with a stated bound) ----
    per_step = {k: (v[0] / steps, v[1] / steps) for k, v in kern.items()}
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_nominal = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    if measured:
        fp32_peak, fp32_src = measured["fp32_fma"]["tflops"], "measured FP32 FMA microbenchmark (mtp_measure_peak)"
        tf32_peak, tf32_src = measured["tf32_mma"]["tflops"], "measured TF32 tcgen05.mma microbenchmark (mtp_measure_peak)"
    else:
        fp32_peak, fp32_src = fp32_nominal, f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"
        tf32_peak, tf32_src = peaks["bf16_tflops"] * 1.1 / 2.25, f"{peaks_kind} bf16 x nominal tf32/bf16"
    n_grade_rows = N if grade else 0
    parts = site_flops_parts(sizes, N, n_pairs, grade)
    work = {
        "site_efs_rows": ("alu", site_flops(sizes, N, n_pairs, True) / 1e12, fp32_peak, "TFLOP/s", fp32_src),
        "site_efs": ("alu", site_flops(sizes, N, n_pairs, False) / 1e12, fp32_peak, "TFLOP/s", fp32_src),
        "grade_tc_tf32x3": ("tensor", 2.0 * n_grade_rows * m * m / 1e12, tf32_peak, "TFLOP/s", tf32_src),
    }
    work.update({k: ("alu", v / 1e12, fp32_peak, "TFLOP/s", fp32_src) for k, v in parts.items()})
    # the three kernels of the split per-neighborhood pass are one pass of the method: the
    # roofline of the pass is its algorithmic work over their summed time
    split_names = [k for k in ("site_moments", "site_contract", "site_adjoint") if k in per_step]
    if split_names:
        per_step["site_pass"] = (sum(per_step[k][0] for k in split_names), 1.0)
        work["site_pass"] = ("alu", site_flops(sizes, N, n_pairs, grade) / 1e12, fp32_peak, "TFLOP/s", fp32_src)

    def roof_of(name):
        if name not in work:
            return None
        bound, amount, peak, unit, src = work[name]
        t = per_step[name][0] / max(per_step[name][1], 1) / 1e3
        achieved = amount / t
        return {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": measured_traffic(name, N, args.config), "peak_source": src,
                "ms_per_launch": t * 1e3}
    # the neighbor build's regions are one pass as well: HBM-bound, 28 B read per atom (positions,
    # species) and 29 B written per pair (j, image, r_ij, reverse index, scanned bin)
    nbr_names = [k for k in per_step if k.startswith("neighbors_")]
    if nbr_names:
        per_step["neighbor_build"] = (sum(per_step[k][0] for k in nbr_names), 1.0)
        hbm = peaks.get("hbm_gbs", 6800.0)
        work["neighbor_build"] = ("hbm", (28.0 * N + 29.0 * n_pairs) / 1e9, hbm, "GB/s",
                                  f"{peaks_kind} HBM copy bandwidth")
    top = {k: v for k, v in per_step.items() if k not in split_names and k not in nbr_names}
    dominant = max(top, key=lambda k: top[k][0])
    roof = roof_of(dominant)
    per_kernel_only = {k: v for k, v in per_step.items() if k not in ("site_pass", "neighbor_build")}
    total_ms = sum(v[0] for v in per_kernel_only.values())
    kernels = {k: {"ms_per_step": round(v[0], 4), "launches_per_step": v[1], "share": round(v[0] / total_ms, 4)}
               for k, v in sorted(per_kernel_only.items(), key=lambda kv: -kv[1][0])}
    launches = int(round(sum(v[1] for v in per_kernel_only.values()) * steps))

    value = world * N * steps / (ms_mixed / 1e3) / 1e6
    fp64_value = world * N * fp64_steps / (ms_fp64 / 1e3) / 1e6
    what = "neighbor rebuild + E/F/W" + (" + grade + flag" if grade else "")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.config}: {w.name} ({N} atoms), level-{w.lev_max} MTP m={m}, R_cut {w.r_cut} A; "
                               f"step = {what}",
                   "config": args.config, "n_atoms": N, "n_pairs": n_pairs,
                   "precision": "mixed (FP32 compute, FP64 sums)",
                   "l2": ("each step timed alone after writing a 256 MB buffer (inputs smaller than L2)"
                          if cfg["flush_l2"] else "inputs larger than L2 (pair list and parameter rows exceed 129 MB)"),
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU",
                   "autotuned": {p: {"warps": t[0], "ms": t[1]} for p, t in tuned.items()},
                   "launch_shape": dict(zip(("warps_mixed_kernel", "forward_schedule_in_global", "warps_generic_kernel"),
                                            api.mtp_get_launch_shape(model)))},
        "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_step": ms_fp64 / fp64_steps,
                      "steps": fp64_steps, "mixed_over_fp64": value / fp64_value},
        "errors_mixed_vs_fp64": err_fp64,
        "active_set": active,
        "reuse_neighbor_list": {"value": world * N * steps / (ms_reuse / 1e3) / 1e6, "unit": UNIT,
                                "ms_per_step": ms_reuse / steps,
                                "graph_ms_per_step": ms_graph / steps,
                                "graph_value": world * N * steps / (ms_graph / 1e3) / 1e6,
                                "note": "E/F/W [+ grade + flag] on an unchanged configuration, no rebuild; eager "
                                        "and replayed from one CUDA graph"},
        "roofline": roof,
        "roofline_kernels": {k: roof_of(k) for k in per_step if k in work and k != dominant and roof_of(k)},
        "mixed_pass": dict(zip(("setting", "in_use", "split_warps", "split_nb"), api.mtp_get_mixed_pass(model)),
                           requested=args.mixed_pass,
                           **dict(zip(("split_unroll", "split_schedule", "split_schedule_used"),
                                      api.mtp_get_split_shape(model)[2:]))),
        "measured_peaks": measured, "kernels": kernels, "gpu_launches": launches, "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_train and args.config == "C4":
        line["train_step"] = measure_train(api, synth, torch)
    if not args.no_cpu_baseline and world == 1:
        cpu, errs = oracle_leg(args, cfg, w, bnp, theta, batch, state_pos, state, model, api, torch, synth)
        line["cpu_baseline"] = cpu
        line["errors_vs_oracle"] = errs
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------
# the oracle on the host cores (timing and errors on sampled atoms of the benchmarked state)
# ------------------------------------------------------------------------------------

def _sample_with_neighbors(nbr, sample):
    need = set(int(k) for k in sample)
    for k in sample:
        need.update(nbr["j"][nbr["off"][k]:nbr["off"][k + 1]].tolist())
    return np.array(sorted(need), np.int64)


def _oracle_forces(nbr, sample, req, G):
    """F_k = sum_{p in nbh(k)} dV_k/dr_p - sum_{p: j(p) = k} dV_{c(p)}/dr_p for sampled k (the
    neighbors of k list k, the list being full)."""
    F = np.zeros((len(sample), 3))
    for q, k in enumerate(sample):
        k = int(k)
        F[q] += G[nbr["off"][k]:nbr["off"][k + 1]].sum(axis=0)
        for j in set(nbr["j"][nbr["off"][k]:nbr["off"][k + 1]].tolist()):
            for p in range(nbr["off"][j], nbr["off"][j + 1]):
                if nbr["j"][p] == k:
                    F[q] -= G[p]
    return F


def oracle_leg(args, cfg, w, bnp0, theta, batch, state_pos, state, model, api, torch, synth):
    """The oracle (FP64, OpenMP over atoms) on sampled atoms of the state both GPU paths were
    evaluated at: per-site V_i, dV_i/dr, b_i for the samples and their neighbors (so sampled
    forces are exact), the grade of the samples; timed on all host cores and on one thread."""
    from oracle import active_set as AS
    from oracle import oracle as O
    md = O.OracleModel(w.n_types, w.lev_max, w.r_min, w.r_cut)
    bnp = dict(bnp0)
    bnp["pos"] = state_pos.cpu().numpy().copy()
    N = len(bnp["type"])
    cores = O.threads()
    t0 = time.perf_counter()
    nbr = O.batch_neighbors(bnp, w.r_cut, brute=False)
    t_nbr = time.perf_counter() - t0
    sample = synth.sample_atoms(77, N, cfg["sample"]) if N > cfg["sample"] else np.arange(N, dtype=np.int64)
    req = _sample_with_neighbors(nbr, sample)
    # timed: every required site (V, dV/dr, b) on all cores, then the grade of the samples
    A = None
    if cfg["grade"]:
        if cfg["active"] == "maxvol":
            # the oracle forms its own active set by the same recipe (FP64 rows, MaxVol), and the
            # GPU grades against it below, so no input of the oracle comes from the GPU path
            D = O.gauge_directions(md, theta)
            comp, pick = companion_start(synth, md.m, len(D))
            crows = O.site_rows(md, theta, comp["type"], O.batch_neighbors(comp, w.r_cut))
            A, _, _ = AS.maxvol(gauge_completion(crows[pick], D), crows, eps=COMPANION["eps"])
        else:
            A = synth.diag_dominant(cfg["a_seed"], md.m)
    t0 = time.perf_counter()
    s = O.sites(md, theta, bnp["type"], nbr, req=req, want_dVdr=True, want_b=cfg["grade"])
    pos_of = {int(a): q for q, a in enumerate(req)}
    srow = [pos_of[int(k)] for k in sample]
    if cfg["grade"]:
        gam, am = O.grade(A, s["b"][srow])
    dt = time.perf_counter() - t0 + t_nbr * len(req) / N
    # one thread, on the first sites of the same list
    n1 = min(len(req), max(8, cfg["sample"] * 2))
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        O.sites(md, theta, bnp["type"], nbr, req=req[:n1], want_dVdr=True, want_b=cfg["grade"])
        dt1 = time.perf_counter() - t0
    finally:
        O.set_threads(cores)
    # errors of both GPU paths on the samples
    G = s["dVdr"]
    F = _oracle_forces(nbr, sample, req, G)
    V = s["V"][srow]
    Wat = np.zeros((len(sample), 3, 3))
    for q, k in enumerate(sample):
        p0, p1 = nbr["off"][k], nbr["off"][k + 1]
        Wat[q] = -(G[p0:p1, :, None] * nbr["r"][p0:p1, None, :]).sum(axis=0)
    errs = {"sample_atoms": len(sample), "sites_evaluated": len(req), "gamma_active_set": None}
    gpu_gamma = {}
    if cfg["grade"]:
        A_gpu = api.mtp_get_active_set(model).cpu().numpy()
        errs["gamma_active_set"] = {"kind": cfg["active"],
                                    "max_abs_diff_vs_library_active_set": float(np.abs(A - A_gpu).max() /
                                                                                 np.abs(A).max())}
        api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
        batch.pos.copy_(state_pos)
        nb = api.mtp_build_neighbors(model, batch)
        for prec in ("mixed", "fp64"):
            g = api.mtp_grade(model, batch, nb, prec, threshold=2.0)
            gpu_gamma[prec] = (g["gamma"].cpu().numpy()[sample], g["argmax"].cpu().numpy()[sample])
    for prec in ("mixed", "fp64"):
        o = state[prec]
        Vg = o["site_energy"].cpu().numpy()[sample]
        Fg = o["forces"].cpu().numpy()[sample]
        Wg = o["site_virial"].cpu().numpy()[sample]
        e = {"max_abs_dV_eV": float(np.abs(Vg - V).max()),
             "max_rel_dV": float(np.abs(Vg - V).max() / max(np.abs(V).max(), 1e-300)),
             "max_abs_dF_eV_per_A": float(np.abs(Fg - F).max()),
             "max_rel_dF": float(np.abs(Fg - F).max() / max(np.abs(F).max(), 1e-300)),
             "max_rel_dW_site": float(np.abs(Wg - Wat).max() / max(np.abs(Wat).max(), 1e-300))}
        if cfg["grade"]:
            dg = np.abs(gpu_gamma[prec][0] - gam) / np.maximum(1.0, gam)
            e["max_rel_dgamma"] = float(dg.max())
            e["argmax_equal"] = bool((gpu_gamma[prec][1] == am).all())
        errs[prec] = e
    if cfg["grade"]:
        errs["gamma_oracle_sample_max"] = float(gam.max())
    cpu = {"value": len(req) / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": (f"{len(req)} sites of the benchmarked state ({len(sample)} sampled atoms and their neighbors): "
                      f"V, dV/dr" + (", b_i and the grade" if cfg["grade"] else "") +
                      f"; the oracle's neighbor build over all {N} atoms ({t_nbr:.1f} s) charged per site; {dt:.1f} s"),
           "single_thread": {"value": n1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                             "sample": f"{n1} of the same sites (V, dV/dr" + (", b_i" if cfg["grade"] else "") +
                                       f"), {dt1:.1f} s, neighbor build not included"}}
    return cpu, errs


def run_reference(args):
    """The FP64 oracle alone on the host cores: each step = the neighbor build of a small
    periodic cell of the workload's structure plus V, dV/dr (and b_i and the grade) of a
    bounded sample of its atoms."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2304_13144_gb300 import configs, synth
    cfg = CONFIGS[args.config]
    w = configs.workload(args.config)
    md = O.OracleModel(w.n_types, w.lev_max, w.r_min, w.r_cut)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(w.theta_seed, w.n_types, md.n_rad, md.n_q, nu_sum, nf, w.r_min, w.r_cut, w.nbar)
    small = {"C1": lambda: synth.fcc_unary_108(seed=1), "C2": lambda: synth.b2_binary(seed=2, n=8),
             "C4": lambda: synth.fcc_ternary(seed=4, n=8),
             "C5": lambda: synth.liquid_rsa(seed=5, n_atoms=4096)}[args.config]
    bnp = small()
    n_cell = len(bnp["type"])
    A = synth.diag_dominant(8, md.m) if cfg["grade"] else None
    n_sample = min(args.ref_sample, n_cell)

    def one(k):
        nbr = O.batch_neighbors(bnp, w.r_cut)
        req = synth.sample_atoms(100 + k, n_cell, n_sample)
        s = O.sites(md, theta, bnp["type"], nbr, req=req, want_dVdr=True, want_b=cfg["grade"])
        if cfg["grade"]:
            O.grade(A, s["b"])
        return len(req)

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    done = sum(one(args.warmup + k) for k in range(args.steps))
    dt = time.perf_counter() - t0
    value = done / dt / 1e6
    cores = O.threads()
    sample = (f"{n_sample} atoms per step of a {n_cell}-atom periodic cell of the {args.config} workload's structure "
              f"(neighbor build + V, dV/dr" + (", b_i, grade" if cfg["grade"] else "") + ")")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.config}: {w.name}, level-{w.lev_max} MTP m={md.m}, R_cut {w.r_cut} A "
                               f"(oracle sample)", "config": args.config},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default per config)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="C4", choices=sorted(CONFIGS))
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-peaks", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (fixed launch sequence)")
    ap.add_argument("--split-shape", default="",
                    help="warps_pair,nb_contract[,unroll[,schedule]] of the three-kernel pass (no autotune)")
    ap.add_argument("--cells", type=int, default=0,
                    help="C4: n^3 fcc cells instead of 64^3; C5: the liquid cube repeated n^3 times instead of 4^3 (profiling)")
    ap.add_argument("--mixed-pass", default="auto", choices=["auto", "single", "split"],
                    help="mixed path: the autotuner's choice, the single kernel or the three kernels")
    ap.add_argument("--ref-sample", type=int, default=256)
    args = ap.parse_args()
    if args.impl == "reference":
        args.steps = args.steps if args.steps is not None else 10
        run_reference(args)
    else:
        args.warmup = max(args.warmup, 3)
        run_ours(args)


if __name__ == "__main__":
    main()
