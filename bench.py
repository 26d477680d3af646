#!/usr/bin/env python
"""Throughput of the MTP hot path on one GB300 (Matom*steps/s), one JSON line on stdout.

Default workload: fcc random solid solution of three species, a = 3.6 A, 64^3 conventional
cells (1,048,576 atoms), Gaussian displacements sigma = 0.1 A, level-20 ternary MTP (m = 651),
R_cut = 5 A.  One step = a real neighbor rebuild (positions are jittered each step) +
energies, forces and virial + per-atom grade gamma_i against the active set + compaction of
the atoms with gamma_i > 2, through the C ABI (mtp_build_neighbors, mtp_step).  The mixed
path (FP32 with FP64 sums) is the headline; the all-FP64 path is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent configuration (weak scaling, no
collective); rank 0 prints.  --impl reference times the FP64 CPU oracle on the host cores on
a bounded sample of the same workload.
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
TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense ratio


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the kernel on a 32^3-cell case of the same workload (131,072 atoms, inputs and outputs larger
# than L2); the traffic grows with the atom count, so a launch over N atoms moves bytes * N / atoms.
# Reported only while the kernel source is the one that was captured (same SHA-1).
MEASURED_TRAFFIC = {
    "site_efs_rows": {"source": "paper_2304_13144_gb300/csrc/site_fast.cu",
                      "sha1": "169ae7b082683549d6c43bd8e44e670cf6108e25",
                      "atoms": 131072, "bytes": 119990016 + 725012480},
    "grade_tc_tf32x3": {"source": "paper_2304_13144_gb300/csrc/grade_tc.cu",
                        "sha1": "edc8f658b225b15351d41bea8a0a3621a776d4a4",
                        "atoms": 131072, "bytes": 708309248 + 2733312},
}


def measured_traffic(kernel, n_atoms):
    rec = MEASURED_TRAFFIC.get(kernel)
    if rec is None:
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

def make_workload(api, synth, n_cells=64, seed=4):
    """The C4 workload of configs.py (fcc ternary solid solution, level 20), with the cell count
    and structure seed adjustable (replicas under torchrun use seed 4 + rank)."""
    from paper_2304_13144_gb300 import configs
    w = configs.workload("C4")
    bnp = synth.fcc_ternary(seed=seed, n=n_cells)
    desc = w.desc()
    return bnp, desc, w.theta(), api.mtp_describe(desc)


def active_set(api, synth, torch, desc, theta, sizes, companion_seed=444, n_cells=12):
    """Active set: parameter rows (FP64) of m - n_gauge atoms drawn without replacement from a
    companion snapshot (same lattice, independent displacement seed), completed by the
    n_gauge null directions of the rows (scaled to the rows' magnitude)."""
    comp = synth.fcc_ternary(seed=companion_seed, n=n_cells)
    m, g = sizes["n_params"], sizes["n_gauge"]
    model = api.mtp_load(desc, theta)
    b = api.Batch(comp)
    nb = api.mtp_build_neighbors(model, b)
    pick = torch.tensor(synth.sample_atoms(companion_seed, len(comp["type"]), m - g))
    rows = api.mtp_param_rows(model, b, nb, "fp64", pick).cpu().numpy()
    D = api.mtp_gauge_directions(desc, theta)
    A = np.vstack([rows, D / np.linalg.norm(D, axis=1, keepdims=True) * np.abs(rows).max()])
    return A


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
    nq, nr, nu, comps = 8, sizes["n_rad"], sizes["nu_max"], sizes["n_mom_comps"]
    n_mono = (nu + 1) * (nu + 2) * (nu + 3) // 6
    per_pair = 8 * nq + 6 * nq + 4 * nr * nq + 6 * nu + n_mono + 2 * comps + 4 * comps + 6 * n_mono + 2 * nr + 9
    if rows:
        per_pair += 2 * nr * nq
    per_atom = 9 * sizes["n_triples"] + 2 * sizes["n_lin"]
    return per_pair * n_pairs + per_atom * n_atoms


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


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2304_13144_gb300 import api, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    peaks, peaks_kind = load_peaks()

    bnp, desc, theta, sizes = make_workload(api, synth, n_cells=args.cells, seed=4 + rank)
    A = active_set(api, synth, torch, desc, theta, sizes)
    model = api.mtp_load(desc, theta)
    api.mtp_set_active_set(model, torch.tensor(A, device="cuda"))
    batch = api.Batch(bnp)
    N = batch.n_atoms
    pos0 = batch.pos.clone()
    nb = api.Neighbors()
    out = None
    # the library's autotuner picks the per-neighborhood kernel's launch shape on this workload
    api.mtp_build_neighbors(model, batch, nb)
    tuned = ({p: api.mtp_autotune(model, batch, nb, p) for p in ("mixed", "fp64")} if not args.no_autotune
             else {p: (0, 0.0) for p in ("mixed", "fp64")})

    def step(k, prec):
        nonlocal out
        # deterministic jitter so every step rebuilds a changed neighbor list
        batch.pos.copy_(pos0 + 1e-4 * math.sin(0.7 * k + 0.1))
        api.mtp_build_neighbors(model, batch, nb)
        out = api.mtp_step(model, batch, nb, prec, threshold=2.0, out=out)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, steps, warmup, profile=False):
        for k in range(warmup):
            step(k, prec)
        barrier()
        if profile:
            api.mtp_profiler_read()
            api.mtp_profiler_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            step(warmup + k, prec)
        e1.record()
        barrier()
        ms = e0.elapsed_time(e1)
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
    ms_mixed, kern = timed("mixed", args.steps, args.warmup, profile=True)
    clk = clocks.stop()
    mixed_out = {k: (v.clone() if v is not None else None) for k, v in out.items()}
    n_pairs = nb.size()[1]
    # ---- the same step on an unchanged configuration, reusing its neighbor list ----
    # (the list stores r_ij, so moving atoms need the rebuild that the headline step includes)
    for _ in range(2):
        out = api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        out = api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out)
    e1.record()
    barrier()
    ms_reuse = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms_reuse], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_reuse = float(t.item())
    # ---- FP64 path beside it ----
    out = None
    ms_fp64, _ = timed("fp64", args.fp64_steps, 1)
    fp64_out = out
    # errors of the mixed path against the FP64 GPU path on the same step
    dF = (mixed_out["forces"] - fp64_out["forces"]).abs().max().item()
    dE = (mixed_out["energy"] - fp64_out["energy"]).abs().max().item() / N
    dW = ((mixed_out["virial"] - fp64_out["virial"]).abs().max() / fp64_out["virial"].abs().max()).item()
    g64 = fp64_out["gamma"]
    dg = ((mixed_out["gamma"] - g64).abs() / torch.clamp(g64, min=1.0)).max().item()
    nflag = int(fp64_out["n_flagged"].item())

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.empty_like(getattr(batch, k), device="cpu").pin_memory()
               for k in ("atom_offset", "pos", "type", "cell", "pbc")}
        for k in pin:
            pin[k].copy_(getattr(batch, k).cpu())
        host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in mixed_out.items()
                    if v is not None and k in ("energy", "forces", "virial", "gamma", "n_flagged")}
        h2d = sum(t.numel() * t.element_size() for t in pin.values())
        d2h = sum(t.numel() * t.element_size() for t in host_out.values())
        out = None

        def e2e_step(k):
            nonlocal out
            pin_pos = pin["pos"]
            for name in ("atom_offset", "type", "cell", "pbc"):
                getattr(batch, name).copy_(pin[name], non_blocking=True)
            batch.pos.copy_(pin_pos, non_blocking=True)
            batch.pos.add_(1e-4 * math.sin(0.3 * k))
            api.mtp_build_neighbors(model, batch, nb)
            out = api.mtp_step(model, batch, nb, "mixed", threshold=2.0, out=out)
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
        e2e = {"value": world * N * args.e2e_steps / (ms_e2e / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ----
    per_step = {k: (v[0] / args.steps, v[1] / args.steps) for k, v in kern.items()}
    total_ms = sum(v[0] for v in per_step.values())
    dominant = max(per_step, key=lambda k: per_step[k][0])
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # FP32 FMA peak, TFLOP/s
    m = sizes["n_params"]
    work = {
        "site_efs_rows": ("alu", site_flops(sizes, N, n_pairs, True) / 1e12, alu_peak, "TFLOP/s"),
        "grade_tc_tf32x3": ("tensor", 2.0 * N * m * m / 1e12,
                            peaks["bf16_tflops"] * TF32_OVER_BF16, "TFLOP/s"),
        "grade_simt_fp32": ("alu", 2.0 * N * m * m / 1e12, alu_peak, "TFLOP/s"),
    }
    roof = None
    if dominant in work:
        bound, amount, peak, unit = work[dominant]
        t = per_step[dominant][0] / max(per_step[dominant][1], 1) / 1e3
        achieved = amount / t
        roof = {"bound": bound, "kernel": dominant, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": measured_traffic(dominant, N),
                "peak_source": (f"{peaks_kind} bf16 x nominal tf32/bf16" if bound == "tensor"
                                else f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({peaks_kind} max clock)")}
    kernels = {k: {"ms_per_step": round(v[0], 4), "launches_per_step": v[1], "share": round(v[0] / total_ms, 4)}
               for k, v in sorted(per_step.items(), key=lambda kv: -kv[1][0])}
    launches = int(round(sum(v[1] for v in per_step.values()) * args.steps))

    value = world * N * args.steps / (ms_mixed / 1e3) / 1e6
    fp64_value = world * N * args.fp64_steps / (ms_fp64 / 1e3) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"fcc ternary random solid solution {args.cells}^3 cells ({N} atoms), "
                               f"level-20 MTP m={m}, R_cut 5 A; step = neighbor rebuild + E/F/W + grade + flag",
                   "n_atoms": N, "n_pairs": n_pairs, "precision": "mixed (FP32 compute, FP64 sums)",
                   "l2": "inputs larger than L2 (pair list and parameter rows exceed 129 MB)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU",
                   "autotuned_warps_per_block": {p: w for p, (w, _) in tuned.items()},
                   "launch_shape": dict(zip(("warps_mixed_kernel", "forward_schedule_in_global", "warps_generic_kernel"),
                                            api.mtp_get_launch_shape(model)))},
        "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_step": ms_fp64 / args.fp64_steps,
                      "steps": args.fp64_steps, "mixed_over_fp64": value / fp64_value},
        "errors_mixed_vs_fp64": {"max_abs_dF_eV_per_A": dF, "abs_dE_per_atom_eV": dE, "rel_dW": dW,
                                 "max_rel_dgamma": dg, "n_flagged_fp64": nflag,
                                 "n_flagged_mixed": int(mixed_out["n_flagged"].item())},
        "reuse_neighbor_list": {"value": world * N * args.steps / (ms_reuse / 1e3) / 1e6, "unit": UNIT,
                                "ms_per_step": ms_reuse / args.steps,
                                "note": "E/F/W + grade + flag on an unchanged configuration, no rebuild"},
        "roofline": roof, "kernels": kernels, "gpu_launches": launches, "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_train:
        line["train_step"] = measure_train(api, synth, torch)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------
# the oracle on the host cores
# ------------------------------------------------------------------------------------

def oracle_sample_step(O, md, theta, bnp, nbr, A, n_sample, seed):
    """One step of the oracle on a bounded sample: sites (V, dV/dr, b) and grade of n_sample
    atoms of a periodic cell of the same workload (per-atom work is independent of the size)."""
    from paper_2304_13144_gb300 import synth
    req = synth.sample_atoms(seed, len(bnp["type"]), n_sample)
    s = O.sites(md, theta, bnp["type"], nbr, req=req, want_dVdr=True, want_b=True)
    O.grade(A, s["b"])
    return len(req)


def cpu_baseline(args, steps=1):
    from oracle import oracle as O
    from paper_2304_13144_gb300 import synth
    md = O.OracleModel(3, 20, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(44, 3, md.n_rad, 8, nu_sum, nf, 2.0, 5.0, 42.0)
    bnp = synth.fcc_ternary(seed=4, n=8)
    t0 = time.perf_counter()
    nbr = O.batch_neighbors(bnp, 5.0)
    t_nbr = (time.perf_counter() - t0) / len(bnp["type"])
    A = synth.diag_dominant(8, md.m)
    done = 0
    t0 = time.perf_counter()
    for k in range(steps):
        done += oracle_sample_step(O, md, theta, bnp, nbr, A, args.cpu_sample, 7 + k)
    dt = time.perf_counter() - t0 + t_nbr * done
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{args.cpu_sample} atoms of a 2048-atom periodic cell of the same fcc ternary "
                      f"workload per step (V, dV/dr, b_i, grade; neighbor build amortised per atom), "
                      f"{steps} step(s), {dt:.1f} s"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2304_13144_gb300 import synth
    md = O.OracleModel(3, 20, 2.0, 5.0)
    nu_sum = [sum(nu for _, nu in labs) for labs, _ in md.basis]
    nf = [len(labs) for labs, _ in md.basis]
    theta = synth.draw_theta(44, 3, md.n_rad, 8, nu_sum, nf, 2.0, 5.0, 42.0)
    bnp = synth.fcc_ternary(seed=4, n=8)
    nbr = O.batch_neighbors(bnp, 5.0)
    A = synth.diag_dominant(8, md.m)
    for k in range(args.warmup):
        oracle_sample_step(O, md, theta, bnp, nbr, A, args.ref_sample, 100 + k)
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        t1 = time.perf_counter()
        nbr = O.batch_neighbors(bnp, 5.0)
        done += oracle_sample_step(O, md, theta, bnp, nbr, A, args.ref_sample, k)
    dt = time.perf_counter() - t0
    value = done / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{args.ref_sample} atoms per step of a 2048-atom periodic cell of the fcc ternary level-20 "
              f"workload (neighbor build + V, dV/dr, b_i, grade)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"fcc ternary random solid solution, level-20 MTP m={md.m}, R_cut 5 A (oracle sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=64)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (fixed launch sequence)")
    ap.add_argument("--cpu-sample", type=int, default=1024)
    ap.add_argument("--ref-sample", type=int, default=256)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
