#!/usr/bin/env python
"""Benchmark of the mass-consistent wind solve on the 3000 x 3000 x 15 cell
terrain-following domain (about 1.44e8 nodes, 1.35e8 free unknowns).

One step = the whole hot path on one synthetic problem: assembly (2x2x2
Gauss; with the default separable operator the column and layer factors and
the finest float64 rows) + Galerkin hierarchy + coarsest inverse, then a
cold solve (load vector + float32 V-cycles inside float64 refinement, the
residual checked every 6 cycles, to a 1e-8 relative residual) + recovery of
u, then a warm-started solve for the next time step's wind (u0 perturbed by
2 %) + recovery.  value = free unknowns x V-cycles / second over the timed
steps; the line also carries the time to 1e-8 of the mixed, mixed + CG and
plain float64 forms, the per-class rooflines, the end-to-end figure with
host buffers, the 96-domain batch and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun: every rank solves its own replica of the domain
(the single-domain solve does not shard here), value sums the ranks' work
over the slowest rank's time.  --impl reference times the CPU oracle on a
bounded window of the same domain (rank 0 only).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("V-cycle unknowns/s and time-to-1e-8 residual at 3000×3000×15; "
          "HBM GB/s % of peak")
UNIT = "unknown-V-cycles/s"
CELLS = (3000, 3000, 15)
RTOL = 1e-8
SAMPLE_W = 160       # CPU baseline / reference window (cells per side)
SAMPLE_I0, SAMPLE_J0 = 1420, 1420
# Float-pair arithmetic per element of the modal element kernels (the default):
# the FP32-pipe thread instructions of their fully unrolled form, counted by ncu
# (sm__inst_executed_pipe_fma x 32 / elements) on one element-parity launch of the
# 600x600x15 case (720000 elements).  The kernels that run keep their loops rolled
# over shared memory and issue some more (selects, addressing); this count is the
# arithmetic the method needs, the `alu` roofline's numerator.
FP32_OPS_STIFFNESS = 14198.0
FP32_OPS_LOAD = 8308.0
# Center recovery in float pairs: FMA-pipe thread instructions per element of
# this build, counted by ncu on the 600x600x15 case (86 % of its instructions;
# the FMA pipe was 73 % busy), the `alu` units of the recover class.
FP32_OPS_RECOVER = 1811.0
# Separable load vector: float-pair multiply-adds per node (45 horizontal and
# 6 vertical), about 12 FP32-pipe instructions each.
FP32_OPS_LOAD_SEPARABLE = 51 * 12.0
# FP32 pipe: 128 lanes per SM x 152 SMs x 2.07 GHz maximum SM clock
FP32_PIPE_PEAK_T = 152 * 128 * 2.07e9 / 1e12
# Float64 element kernels (element_arith = ARITH_F64, the plain FP64 form):
# float64 thread instructions per element of the modal stiffness and load
# vector, counted by ncu on the 600x600x15 case (DADD + DFMA + DMUL).
FP64_OPS_STIFFNESS = 1213.0
FP64_OPS_LOAD = 665.0
# DRAM bytes (read + write) per unit of a launch, from one ncu capture of a
# smaller case of the same kernel, scaled by the units of the full launch:
# separable float32 smoother, bytes per free node of the column group
# (1200x1200x15: 189.8 MB per group launch of 5.39 M nodes).
TRAFFIC_PER_UNIT = {"smooth_fine": (35.2, "ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                          "1200x1200x15 group launch, scaled per group node",
                                    "separable")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mcwind", choices=["mcwind", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--op-form", default="separable", choices=["stored", "separable"],
                    help="float32 cycle on stored 27-point rows or on the column x layer "
                         "factors of the shift-form grid (mixed precision)")
    ap.add_argument("--cells", type=int, nargs=3, default=list(CELLS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f64-compare", action="store_true")
    ap.add_argument("--workload", default="domain", choices=["domain", "batched", "rates"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 96-domain batched workload in the default run")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--launch-summary", default=None, metavar="CSV",
                    help="print per-kernel launches, time and share from an ncu "
                         "--metrics gpu__time_duration.sum --csv log, then exit")
    return ap.parse_args()


# --------------------------------------------------------------------------
# CPU oracle on a bounded window of the same domain

def oracle_step(c, cn):
    """The oracle's own pipeline on case c: assembly + hierarchy, cold
    V-cycle solve to 1e-8 + recovery, warm solve for wind cn + recovery.
    Returns the V-cycles run."""
    import oracle
    H = oracle.Hierarchy(c)
    f = oracle.assemble_f(c)
    lam, h1 = H.solve(f, rtol=RTOL)
    oracle.recover(c, lam)
    f2 = oracle.assemble_f(c, u0=cn)
    lam2, h2 = H.solve(f2, x0=lam, rtol=RTOL)
    oracle.recover(c, lam2, u0=cn)
    return (len(h1) - 1) + (len(h2) - 1)


def sample_case(w=SAMPLE_W):
    import synth
    c = synth.full_domain_window(SAMPLE_I0, SAMPLE_J0, w, w)
    cn = synth.perturb_wind(c.u0, 0)
    return c, cn


def run_cpu_sample(steps=1, warmup=0):
    """Time the oracle on the window; returns a dict in the bench's unit."""
    c, cn = sample_case()
    for _ in range(warmup):
        oracle_step(c, cn)
    t0 = time.perf_counter()
    cycles = 0
    for _ in range(steps):
        cycles += oracle_step(c, cn)
    dt = time.perf_counter() - t0
    return {"value": c.n_free * cycles / dt, "unit": UNIT, "seconds": dt, "cycles": cycles,
            "steps": steps, "n_free": c.n_free}


def cpu_sample_subprocess(threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", "1"],
                         env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        return {"error": out.stderr[-400:]}
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_subprocess():
    """The oracle on the bounded window with all host threads (its OpenMP
    element loops; the multigrid's sparse products run in one thread), and
    again with one thread."""
    ncpu = os.cpu_count() or 1
    many = cpu_sample_subprocess(ncpu)
    one = cpu_sample_subprocess(1)
    if "error" in many:
        return many
    sample = (f"oracle (plain C with OpenMP + scipy) on cells [{SAMPLE_I0},{SAMPLE_I0 + SAMPLE_W})^2 x 15 "
              f"of the same domain ({many['n_free']} free unknowns): assembly + hierarchy, "
              f"cold + warm V-cycle solves to 1e-8, recovery; {many['cycles']} V-cycles in "
              f"{many['seconds']:.1f} s")
    return {"value": many["value"], "unit": UNIT, "cores": ncpu, "nproc": ncpu, "kind": "oracle",
            "sample": sample, "seconds": many["seconds"],
            "one_thread": ({"value": one["value"], "seconds": one["seconds"], "cores": 1}
                           if "error" not in one else one)}


def oracle_full_size(case, lam_h, u0):
    """The oracle at full size (its OpenMP element loops, all host threads):
    the load vector of Eq. 5 and the residual certificate
    ||f - K lambda_gpu|| / ||f||, each timed."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    f = oracle.assemble_f(case, u0=u0, parallel=True)
    t1 = time.perf_counter()
    r = f - oracle.apply_K(case, lam_h)
    t2 = time.perf_counter()
    free = oracle.case_free_mask(case)
    cert = float(np.linalg.norm(r[free]) / np.linalg.norm(f[free]))
    return {"kind": "oracle", "cores": os.cpu_count() or 1, "load_vector_s": t1 - t0,
            "residual_certificate_s": t2 - t1, "certificate_rel_res": cert,
            "sample": "full 3000x3000x15 domain: oracle load vector and ||f - K lambda||/||f|| "
                      "of the GPU's cold-solve lambda, both element by element in float64"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    r = run_cpu_sample(steps=max(1, args.steps), warmup=max(0, args.warmup))
    c_free = r["n_free"]
    line = {
        "impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * r["seconds"] / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"CPU oracle on a {SAMPLE_W}x{SAMPLE_W}x15-cell window of the "
                               "3000x3000x15 terrain-following domain (bounded sample)",
                   "cells": [SAMPLE_W, SAMPLE_W, 15], "n_free": c_free, "rtol": RTOL},
        "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{SAMPLE_W}x{SAMPLE_W}x15 window, {r['cycles']} V-cycles"},
        "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# whole-job aggregate over the ranks (replicas: no data-path collective)

def job_totals(dist, seconds, work, device):
    """Slowest rank's time and the summed work of all ranks (one replica of
    the domain per rank).  dist is None for one process; otherwise an
    initialized torch.distributed (nccl on the GPUs, gloo in the tests)."""
    if dist is None:
        return float(seconds), float(work)
    import torch
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], device=device, dtype=torch.float64)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


# --------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    def __init__(self, torch, dev):
        self.proc = None
        self.path = None
        try:
            uuid = str(torch.cuda.get_device_properties(dev).uuid)
            sel = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
        except Exception:
            sel = str(dev)
        fields = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                  "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", sel, f"--query-gpu={fields}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------

KINDS = ["assemble", "rap", "setup", "rhs", "outer_residual", "smooth_fine", "smooth_coarse",
         "residual_fine", "residual_coarse", "restrict", "prolong", "coarse_solve", "update",
         "recover", "krylov", "other"]


def read_profile(m, plan):
    import ctypes
    ms = (ctypes.c_double * len(KINDS))()
    n = (ctypes.c_longlong * len(KINDS))()
    m.lib().mcwind_profile_read(plan.handle, ms, n, len(KINDS), m._stream(None))
    return {k: (ms[i], n[i]) for i, k in enumerate(KINDS)}


def class_units(levels, mixed, separable, solves, nu, cpc, n_elem, n_coarse, sep_rhs=True,
                element_f64=False, with_recovery=True):
    """Algorithmic units of every kernel class over the timed region.

    levels: the plan's level descriptions (Nx, Ny, Nz, hx, hy); solves: the
    cycle counts of the timed solves (cold and warm alternating, cold first).  For each class a list of (bound, total
    units): bytes every array element the launches must read or write at
    least once ("hbm"), float64 FMAs ("fp64"), float-pair FP32-pipe operations
    ("alu").  A smoother launch of one column group reads the x values of the
    whole level (its 8 neighbours lie in the other groups), f and the
    coefficients (or the column factors) of its own nodes, and writes its own
    x; the residual reads x, f and the coefficients once and writes r (or,
    fused with the vertical restriction, the coarse right side)."""
    cs = 4 if mixed else 8
    L = len(levels)
    nodes = [d["Nx"] * d["Ny"] * d["Nz"] for d in levels]
    free = [(d["Nx"] - 2) * (d["Ny"] - 2) * (d["Nz"] - 1) for d in levels]
    fcols = [(d["Nx"] - 2) * (d["Ny"] - 2) for d in levels]
    cycles = sum(solves)
    checks = sum(c // cpc for c in solves) if mixed else cycles
    nsolve = len(solves)
    fac = 36 * 4            # float32 factor bytes per column
    U = {k: [] for k in ("smooth_fine", "smooth_coarse", "residual_fine", "residual_coarse",
                         "restrict", "prolong", "coarse_solve", "update", "outer_residual")}

    def add(key, bound, v):
        U[key].append([bound, v])

    hb = {k: 0.0 for k in U}
    fp64 = {k: 0.0 for k in U}
    for l in range(L - 1):
        sm = "smooth_fine" if l == 0 else "smooth_coarse"
        rs = "residual_fine" if l == 0 else "residual_coarse"
        g4 = free[l] / 4.0
        if separable:
            full = 4 * nodes[l] + 8 * g4 + fac * fcols[l] / 4.0
            zero = 4 * g4 + 16 * fcols[l] / 4.0 + 4 * nodes[l]
        else:
            full = 27 * cs * g4 + cs * nodes[l] + 2 * cs * g4
            zero = 2 * cs * g4 + cs * g4 + cs * nodes[l]
        n_launch = 4 * (nu[0] + nu[1])
        # first group of each pre-smoothing starts from zero on the coarse levels, and
        # on the finest level in the first cycle of each check (mixed precision)
        n_zero = cycles if l > 0 else (checks if mixed else 0)
        hb[sm] += (cycles * n_launch - n_zero) * full + n_zero * zero
        if not mixed:
            fp64[sm] += cycles * n_launch * 27 * g4
        fused = separable and not levels[l]["hx"] and not levels[l]["hy"]
        if separable:
            rb = 4 * nodes[l] + 4 * free[l] + fac * fcols[l] + (4 * nodes[l + 1] if fused else 4 * nodes[l])
        else:
            rb = 27 * cs * free[l] + cs * nodes[l] + cs * free[l] + cs * nodes[l]
        hb[rs] += cycles * rb
        if not mixed:
            fp64[rs] += cycles * 27 * free[l]
        if not fused:
            hb["restrict"] += cycles * (cs * nodes[l] + cs * nodes[l + 1])
        hb["prolong"] += cycles * (cs * nodes[l + 1] + 2 * cs * free[l])
        if not mixed:
            # float64 transfers: per fine node its n coarse taps share one
            # weight, n float64 operations; per coarse node centre + (minus +
            # plus) / 2 per direction and row, two operations each
            a, b = levels[l], levels[l + 1]
            tx = (a["Nx"] - 2) + (-(-(a["Nx"] - 2) // 2) if a["hx"] else 0)
            ty = (a["Ny"] - 2) + (-(-(a["Ny"] - 2) // 2) if a["hy"] else 0)
            tz = (a["Nz"] - 1) + (a["Nz"] - b["Nz"])
            fp64["prolong"] += cycles * float(tx) * ty * tz
            rows = (3 if a["hy"] else 1) * 3
            per_c = 2 * (rows if a["hx"] else 0) + 2 * (3 if a["hy"] else 0) + 2
            fp64["restrict"] += cycles * float(per_c) * free[l + 1]
    hb["coarse_solve"] += cycles * 8.0 * n_coarse * n_coarse
    fp64["coarse_solve"] += cycles * float(n_coarse) * n_coarse
    if mixed:
        hb["update"] += checks * 20.0 * free[0]
    # the first residual of a cold solve is r = f (x = 0): f read, r written
    n_cold = (nsolve + 1) // 2
    n_outer = checks + nsolve - n_cold
    hb["outer_residual"] += n_outer * (27 * 8 + 8 + 8 + 8) * free[0] + n_cold * 16.0 * free[0]
    fp64["outer_residual"] += n_outer * 28.0 * free[0]
    for k in U:
        if hb[k]:
            add(k, "hbm", hb[k])
        if fp64[k]:
            add(k, "fp64", fp64[k])
    # per call: load vector (one per solve), recovery (one per solve), assembly
    # (one per two solves)
    if separable and sep_rhs:
        # u0 -> split-layout float pairs (24 B in, 24 B out per node), then the
        # load vector: u0 pairs in, f out, the column factors once
        U["rhs"] = [["hbm", nsolve * (48 + 24 + 8) * nodes[0] + nsolve * 45 * 8.0 * fcols[0]],
                    ["alu", nsolve * FP32_OPS_LOAD_SEPARABLE * nodes[0]]]
    elif element_f64:
        U["rhs"] = [["fp64", nsolve * FP64_OPS_LOAD * n_elem]]
    else:
        U["rhs"] = [["alu", nsolve * FP32_OPS_LOAD * n_elem]]
    if separable:
        # the finest float64 rows expanded from the factors in float pairs: 27
        # coefficients and 1/diag written per node, the column factors read once
        U["assemble"] = [["hbm", nsolve / 2 * (28 * 8.0 * nodes[0] + 36 * 8.0 * nodes[0] / levels[0]["Nz"])]]
    elif element_f64:
        U["assemble"] = [["fp64", nsolve / 2 * FP64_OPS_STIFFNESS * n_elem]]
    else:
        # float pairs: their own FP32-pipe count, and the float64 form's work
        # (1213 FP64 instructions per element) against the FP64 rate
        U["assemble"] = [["alu", nsolve / 2 * FP32_OPS_STIFFNESS * n_elem],
                         ["fp64_equiv", nsolve / 2 * FP64_OPS_STIFFNESS * n_elem]]
    if separable:
        # lambda and u0 read, u written (the column form splits in registers)
        U["recover"] = [["hbm", nsolve * ((8 + 24) * nodes[0] + 24.0 * n_elem)]]
    else:
        U["recover"] = [["hbm", nsolve * ((8 + 24 + 24) * nodes[0] + 24.0 * n_elem)],
                        ["alu", nsolve * FP32_OPS_RECOVER * n_elem]]
    # Galerkin products per assembly: of the column factors (separable: 36 float64
    # values per column read and written per horizontal stage, and the float32
    # tiles), or of the stored rows (28 float64 values per node in and out per
    # one-direction stage)
    n_asm = nsolve / 2
    rap = 0.0
    for l in range(L - 1):
        a, b = levels[l], levels[l + 1]
        if separable:
            if a["hx"] or a["hy"]:
                cin = a["Nx"] * a["Ny"]
                cmid = b["Nx"] * a["Ny"] if (a["hx"] and a["hy"]) else 0
                cout = b["Nx"] * b["Ny"]
                rap += 36 * 8.0 * (cin + 2 * cmid + cout) + 36 * 12.0 * cout
        else:
            stages = int(a["hx"]) + int(a["hy"]) + int(b["Nz"] != a["Nz"])
            rap += stages * 28 * 8.0 * (nodes[l] + nodes[l + 1])
    U["rap"] = [["hbm", n_asm * rap]]
    # set-up per assembly: the finest rows' finalization (27 coefficients read,
    # 1/diag written) and, separable, the shift-form check (X, Y, Z read) and
    # the two float64 factor passes over the ground layer
    setup = (27 * 8 + 8) * nodes[0]
    if separable:
        setup += 24 * nodes[0] + (36 + 45) * 8 * 2.0 * fcols[0]
    elif mixed:
        setup += sum(28 * 12.0 * nn for nn in nodes)  # float32 copies
    U["setup"] = [["hbm", n_asm * setup]]
    # layout conversions and norms per solve: |f| (8 B per node), lambda out
    # (8 in, 8 out), lambda in for warm starts (8 in, 8 out); per recovery of
    # the stored form lambda and u0 split into float pairs (16 and 48 B per node)
    n_warm = nsolve - (nsolve + 1) // 2
    other = nsolve * (8 + 16) * nodes[0] + n_warm * 16.0 * nodes[0]
    if not separable and with_recovery:
        other += nsolve * 64.0 * nodes[0]
    U["other"] = [["hbm", other]]
    return {k: v for k, v in U.items() if v}


def run_batched(steps, warmup, autotune_on=True):
    """96 independent domains (horizontal cells uniform in [48, 384] per axis,
    8-20 layers, a3 in {1, 4, 10}), mixed precision with the separable
    operator, per-domain autotuned sweeps, solved together to 1e-8 by one CUDA
    graph launch per solve (a conditional loop with an IF node per domain).
    Every domain of the timed solve is certified by the oracle
    (||f - K lambda|| / ||f||, element by element in float64); the 4
    smallest are also compared element-wise with the oracle's own solve."""
    import numpy as np
    import torch

    import oracle
    import paper_2101_08453_gb300 as m
    from paper_2101_08453_gb300 import autotune
    import synth

    m.build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cases = synth.batch_domains(n=96, seed=0)
    plans, u0s = [], []
    for c in cases:
        X, Y, Z, u0 = (torch.from_numpy(a).cuda() for a in (c.X, c.Y, c.Z, c.u0))
        p = m.Plan.for_case(c, precision=m.PREC_MIXED, op_form=m.OP_SEPARABLE)
        p.assemble(X, Y, Z)
        p._keep = (X, Y, Z)
        plans.append(p)
        u0s.append(u0)
    n_free = [c.n_free for c in cases]
    t0 = time.perf_counter()
    tuned = autotune.tune_batch(plans, u0s, rtol=RTOL) if autotune_on else None
    t_tune = time.perf_counter() - t0
    batch = m.Batch(plans)
    lams = [torch.zeros(p.node_shape, dtype=torch.float64, device="cuda") for p in plans]
    for _ in range(warmup):
        batch.solve(u0s, lams, rtol=RTOL)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    dom_cycles = 0
    stats = None
    for _ in range(steps):
        for l in lams:
            l.zero_()
        _, stats = batch.solve(u0s, lams, rtol=RTOL)
        dom_cycles += sum(nf * st.cycles for nf, st in zip(n_free, stats))
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / steps
    # the oracle's certificate of every domain's timed solution
    certs = []
    for c, lam, st in zip(cases, lams, stats):
        lh = lam.cpu().numpy().ravel()
        f = oracle.assemble_f(c, parallel=True)
        free = oracle.case_free_mask(c)
        r = f - oracle.apply_K(c, lh)
        certs.append(float(np.linalg.norm(r[free]) / np.linalg.norm(f[free])))
    # the same domains one after another
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for p, u0, l in zip(plans, u0s, lams):
        l.zero_()
        m.mcwind_solve(p.handle, u0, l, RTOL, 150, 0)
    s1.record()
    torch.cuda.synchronize()
    t_seq = s0.elapsed_time(s1) / 1e3
    # element-wise against the oracle's own solve on the 4 smallest domains
    lams2, _ = batch.solve(u0s, [torch.zeros_like(l) for l in lams], rtol=1e-11, max_cycles=250)
    small = sorted(range(len(cases)), key=lambda d: n_free[d])[:4]
    errs = {}
    for d in small:
        ref = oracle.solve(cases[d])
        errs[cases[d].name] = float(np.linalg.norm(lams2[d].cpu().numpy().ravel() - ref)
                                    / np.linalg.norm(ref))
    return {
        "workload": "96 independent domains, horizontal cells U[48,384] per axis, 8-20 layers, "
                    "a3 in {1,4,10}, random hills + log-law wind, mixed precision, separable "
                    "operator, one graph launch per batch solve",
        "n_free_total": sum(n_free), "rtol": RTOL,
        "unknowns_per_s": sum(n_free) / t, "unknown_vcycles_per_s": dom_cycles / steps / t,
        "batched_s": t, "sequential_s": t_seq, "batched_speedup": t_seq / t,
        "graph_launches_per_solve": 1, "max_domain_cycles": max(st.cycles for st in stats),
        "all_converged": all(st.status == 0 for st in stats),
        "oracle_certificate_max": max(certs), "oracle_certificate_domains": len(certs),
        "max_rel_err_vs_oracle_solve_smallest4": max(errs.values()),
        "autotune_s": t_tune,
        "tuning_sweeps": sorted({b[0] for b in tuned}) if tuned else None,
    }


def bench_batched(args):
    """The batched workload alone (--workload batched)."""
    r = run_batched(args.steps, args.warmup, autotune_on=not args.no_autotune)
    line = {
        "metric": "aggregate unknowns/s, 96 batched domains to 1e-8", "unit": "unknowns/s",
        "value": r["unknowns_per_s"], "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * r["batched_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": r["workload"], "n_free_total": r["n_free_total"], "rtol": RTOL},
        "batched": r,
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_rates(args):
    """Convergence rate of the multigrid cycle (2+2 sweeps, FP64) over the
    penalty a3 and the vertical stretching, for both readings of the
    semicoarsening ratio: one 150 m hill (sigma 400 m) on 128 x 128 x 12 cells,
    ground layer 5 m, log-law wind + noise; rate = geometric mean reduction
    from cycle 3, to 1e-10."""
    import numpy as np
    import torch

    import paper_2101_08453_gb300 as m
    import synth

    m.build.build()
    rows = []
    terrain = synth.single_hill(128, 128, 12).Z[0]   # the ground surface z_s(x, y)
    for stretch in (1.0, 1.1, 1.2, 1.3):
        for a3 in (1.0, 2.0, 5.0, 10.0, 20.0):
            X, Y, Z, zeta = synth.node_grid(128, 128, 12, terrain, h0=5.0, ratio=stretch)
            u0 = synth.log_wind(128, 128, 12, zeta, 8.0, 270.0, 0.2, np.random.default_rng(0))
            Xd, Yd, Zd, U = (torch.from_numpy(v).cuda() for v in (X, Y, Z, u0))
            for rule, name in ((m.RULE_PAPER, "paper"), (m.RULE_OPERATOR, "operator")):
                p = m.Plan(128, 128, 12, (1.0, 1.0, a3), synth.DX,
                           synth.layer_thicknesses(12, 5.0, stretch), coarsen_rule=rule)
                p.assemble(Xd, Yd, Zd)
                lam, st = p.solve(U, rtol=1e-10, max_cycles=200)
                rows.append({"stretch": stretch, "a3": a3, "rule": name, "levels": p.num_levels,
                             "cycles_to_1e-10": st.cycles, "rate": st.rate, "status": st.status})
                del p
    print(json.dumps({"workload": "rate study, 128x128x12 single hill", "rows": rows}), flush=True)
    return 0


def launch_summary(path):
    """Per-kernel launches, total device time and share of an ncu launch list."""
    import collections
    import csv
    rows = list(csv.reader(open(path)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Value" in r)
    h = rows[hi]
    ki, mi, vi, ui = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    scale = {"nsecond": 1e-6, "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0,
             "ms": 1.0, "second": 1e3}
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki]
        for pre in ("void ", "mcw::", "<unnamed>::", "unnamed>::", "(anonymous namespace)::"):
            name = name.replace(pre, "")
        name = name.split("(")[0]
        tot[name] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1e-6)
        cnt[name] += 1
    total = sum(tot.values())
    print(f"| kernel | launches | total ms | share |\n|---|---:|---:|---:|")
    for k, v in sorted(tot.items(), key=lambda kv: -kv[1]):
        print(f"| `{k}` | {cnt[k]} | {v:.2f} | {100 * v / total:.1f}% |")
    print(f"| total | {sum(cnt.values())} | {total:.2f} | 100% |")
    return 0


def main():
    args = parse()
    if args.launch_summary:
        return launch_summary(args.launch_summary)
    if args.workload == "batched" and args.impl != "reference":
        return bench_batched(args)
    if args.workload == "rates" and args.impl != "reference":
        return bench_rates(args)
    if args.cpu_sample:
        print(json.dumps(run_cpu_sample(steps=1)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import ctypes

    import numpy as np
    import torch

    import paper_2101_08453_gb300 as m
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    m.build.build()
    nx, ny, nz = args.cells
    prec = m.PREC_MIXED if args.precision == "mixed" else m.PREC_F64
    t_gen = time.perf_counter()
    case = synth.full_domain(nx, ny, nz, seed=0)
    u0n_np = synth.perturb_wind(case.u0, 0)
    t_gen = time.perf_counter() - t_gen
    n_free = case.n_free

    X, Y, Z, U0, U0N = (torch.from_numpy(a).to(dev) for a in (case.X, case.Y, case.Z, case.u0, u0n_np))
    op_form = m.OP_SEPARABLE if (args.op_form == "separable" and prec == m.PREC_MIXED) else m.OP_STORED
    plan = m.Plan.for_case(case, precision=prec, op_form=op_form)
    plan_cpc = m.plan_options(plan.handle).cycles_per_check   # the interval in use
    plan_ws = plan.workspace_bytes
    plan_nu = (plan.options.nu_pre, plan.options.nu_post)
    main_levels = [plan.level(l) for l in range(plan.num_levels)]
    f64_levels, f64_solves = None, None
    lam = torch.zeros(plan.node_shape, dtype=torch.float64, device=dev)
    u_c = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev)
    u_w = torch.empty_like(u_c)
    stream = torch.cuda.current_stream()

    copy_stream = torch.cuda.Stream(device=dev)
    ev_u0, ev_u0n, ev_uc = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()

    def step(inputs=None, outputs=None, ev=None):
        # With host buffers, the winds are copied in on a copy stream while
        # the grid is assembled (the first) and the first wind is solved (the
        # second), and the first wind field is copied out while the second
        # is solved.
        if inputs is not None:
            for dst, src in zip((X, Y, Z), inputs[:3]):
                dst.copy_(src, non_blocking=True)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                U0.copy_(inputs[3], non_blocking=True)
                ev_u0.record(copy_stream)
                U0N.copy_(inputs[4], non_blocking=True)
                ev_u0n.record(copy_stream)
        if ev: ev[0].record()
        plan.assemble(X, Y, Z)
        if ev: ev[1].record()
        if inputs is not None:
            stream.wait_event(ev_u0)
        _, s1 = m.mcwind_solve(plan.handle, U0, lam, RTOL, 100, 0)
        if ev: ev[2].record()
        m.mcwind_recover(plan.handle, U0, lam, u_c)
        if outputs is not None:
            ev_uc.record(stream)
            copy_stream.wait_event(ev_uc)
            with torch.cuda.stream(copy_stream):
                outputs[0].copy_(u_c, non_blocking=True)
        if inputs is not None:
            stream.wait_event(ev_u0n)
        _, s2 = m.mcwind_solve(plan.handle, U0N, lam, RTOL, 100, m.WARM)
        if ev: ev[3].record()
        m.mcwind_recover(plan.handle, U0N, lam, u_w)
        if ev: ev[4].record()
        if outputs is not None:
            outputs[1].copy_(u_w, non_blocking=True)
        if inputs is not None or outputs is not None:
            stream.wait_stream(copy_stream)
        if s1.status != 0 or s2.status != 0:
            raise RuntimeError(f"solve did not converge: {s1.status} {s2.status}")
        return s1, s2

    for _ in range(args.warmup):
        step()
    barrier()
    # ---- timed region: K steps, inputs resident in HBM -------------------
    clocks = ClockSampler(torch, dev)
    m.lib().mcwind_profile(plan.handle, 1, m._stream(None))
    l0 = m.lib().mcwind_launch_count()
    phase_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    w0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_steps")   # lets ncu --nvtx-include select the timed steps
    e0.record()
    cycles = []
    for s in range(args.steps):
        s1, s2 = step(ev=phase_ev[s])
        cycles.append((s1.cycles, s2.cycles, s1.rel_res, s2.rel_res, s1.rate, s2.rate))
    e1.record()
    torch.cuda.nvtx.range_pop()
    barrier()
    wall = time.perf_counter() - w0
    launches = m.lib().mcwind_launch_count() - l0
    prof = read_profile(m, plan)
    m.lib().mcwind_profile(plan.handle, 0, m._stream(None))
    clk = clocks.stop()
    t_dev = e0.elapsed_time(e1) / 1e3
    work = n_free * sum(c[0] + c[1] for c in cycles)
    phases = np.array([[phase_ev[s][q].elapsed_time(phase_ev[s][q + 1]) for q in range(4)]
                       for s in range(args.steps)])
    t_dev, work_all = job_totals(dist, t_dev, work, dev)
    value = work_all / t_dev

    # one more step without the profiler (solver iterations replayed from graphs)
    u0e, u1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    u0e.record()
    step()
    u1e.record()
    barrier()
    ms_unprofiled = u0e.elapsed_time(u1e)

    # ---- end to end through the public API with host buffers ------------
    e2e = None
    if not args.no_e2e:
        # End to end through the public API with host buffers, every step
        # copying its own inputs in and both wind fields out inside the timed
        # region.  Two device sets of inputs and outputs alternate, so the
        # next step's inputs are copied in (copy stream) while this step
        # computes, once the step before released that set, and this step's
        # second wind is copied out while the next one computes.
        pin = [torch.from_numpy(a).pin_memory() for a in (case.X, case.Y, case.Z, case.u0, u0n_np)]
        outs = [torch.empty(u_c.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        sets = [(X, Y, Z, U0, U0N, u_c, u_w)]
        sets.append(tuple(torch.empty_like(t) for t in sets[0]))
        ready = [torch.cuda.Event(), torch.cuda.Event()]   # a set's inputs are in
        done = [torch.cuda.Event(), torch.cuda.Event()]    # a set's compute is over
        uc_ev = torch.cuda.Event()

        def copy_in(si, after=None):
            with torch.cuda.stream(copy_stream):
                if after is not None:
                    copy_stream.wait_event(after)
                for dst, src in zip(sets[si][:5], pin):
                    dst.copy_(src, non_blocking=True)
                ready[si].record(copy_stream)

        def e2e_steps(n):
            work = 0
            copy_stream.wait_stream(stream)
            copy_in(0)
            for s in range(n):
                si = s % 2
                Xs, Ys, Zs, U0s, U0Ns, ucs, uws = sets[si]
                if s + 1 < n:   # the next step's inputs, once step s-1 is done with its set
                    copy_in(1 - si, done[1 - si] if s >= 1 else None)
                stream.wait_event(ready[si])
                plan.assemble(Xs, Ys, Zs)
                _, s1 = m.mcwind_solve(plan.handle, U0s, lam, RTOL, 100, 0)
                m.mcwind_recover(plan.handle, U0s, lam, ucs)
                uc_ev.record(stream)
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(uc_ev)
                    outs[0].copy_(ucs, non_blocking=True)
                _, s2 = m.mcwind_solve(plan.handle, U0Ns, lam, RTOL, 100, m.WARM)
                m.mcwind_recover(plan.handle, U0Ns, lam, uws)
                done[si].record(stream)
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(done[si])
                    outs[1].copy_(uws, non_blocking=True)
                if s1.status != 0 or s2.status != 0:
                    raise RuntimeError(f"solve did not converge: {s1.status} {s2.status}")
                work += n_free * (s1.cycles + s2.cycles)
            stream.wait_stream(copy_stream)
            return work

        e2e_steps(2)   # warm-up of both sets
        torch.cuda.synchronize()
        ke = max(2, min(4, args.steps))
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        ework = e2e_steps(ke)
        a1.record()
        barrier()
        te, ework = job_totals(dist, a0.elapsed_time(a1) / 1e3, ework, dev)
        h2d = sum(p.numel() * 8 for p in pin)
        d2h = sum(o.numel() * 8 for o in outs)
        e2e = {"value": ework / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ke, "ms_per_step": 1e3 * te / ke,
               "copies": "inputs of the next step and the second wind of this one "
                         "overlap the compute (two device sets)"}
        # the plan reads the coordinates it was assembled with: restore set 0
        plan.assemble(X, Y, Z)
        del pin, outs, sets

    # ---- time to 1e-8: mixed vs plain float64 (outside the timed region) --
    def time_solve(p, u0, warm):
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        _, st = m.mcwind_solve(p.handle, u0, lam, RTOL, 100, m.WARM if warm else 0)
        b1.record()
        torch.cuda.synchronize()
        return b0.elapsed_time(b1) / 1e3, st

    lam.zero_()
    t_cold, st_cold = time_solve(plan, U0, False)
    lam_cold_h = lam.cpu().numpy().ravel() if (rank == 0 and not args.no_cpu_baseline) else None
    t_warm, st_warm = time_solve(plan, U0N, True)
    tt = {args.precision: {"cold_s": t_cold, "cold_cycles": st_cold.cycles,
                           "warm_s": t_warm, "warm_cycles": st_warm.cycles,
                           "cold_rate": st_cold.rate,
                           "form": ("float32 V-cycles (%s operator) inside float64 refinement; "
                                    "element arithmetic in float pairs" % args.op_form)
                           if prec == m.PREC_MIXED else "float64"}}
    prof_main = prof
    prof_f64 = None
    if not args.no_f64_compare and prec == m.PREC_MIXED:
        plan = None
        torch.cuda.empty_cache()
        # the same solves accelerated by conjugate gradients (one V-cycle per iteration)
        pcg = m.Plan.for_case(case, precision=m.PREC_MIXED, accel=m.ACCEL_CG, op_form=op_form)
        pcg.assemble(X, Y, Z)
        lam.zero_()
        time_solve(pcg, U0, False)
        lam.zero_()
        tcc, scc = time_solve(pcg, U0, False)
        tcw, scw = time_solve(pcg, U0N, True)
        tt["mixed_cg"] = {"cold_s": tcc, "cold_cycles": scc.cycles, "warm_s": tcw,
                          "warm_cycles": scw.cycles, "cold_rate": scc.rate}
        del pcg
        torch.cuda.empty_cache()
        # the plain float64 form: float64 element arithmetic too
        p64 = m.Plan.for_case(case, precision=m.PREC_F64, element_arith=m.ARITH_F64)
        p64.assemble(X, Y, Z)
        lam.zero_()
        time_solve(p64, U0, False)
        lam.zero_()
        m.lib().mcwind_profile(p64.handle, 1, m._stream(None))
        t64c, s64c = time_solve(p64, U0, False)
        t64w, s64w = time_solve(p64, U0N, True)
        prof_f64 = read_profile(m, p64)
        m.lib().mcwind_profile(p64.handle, 0, m._stream(None))
        f64_levels = [p64.level(l) for l in range(p64.num_levels)]
        f64_solves = [s64c.cycles, s64w.cycles]
        tt["f64"] = {"cold_s": t64c, "cold_cycles": s64c.cycles, "warm_s": t64w,
                     "warm_cycles": s64w.cycles, "cold_rate": s64c.rate,
                     "form": "plain float64: element arithmetic, stored operators and solve all "
                             "in float64 (element_arith = ARITH_F64)"}
        del p64

    # ---- roofline of the dominant kernel class ---------------------------
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    plan_dims = (nx + 1, ny + 1, nz + 1)
    n_nodes = plan_dims[0] * plan_dims[1] * plan_dims[2]
    n_elem = nx * ny * nz

    # FP64 pipe of this GB300: 2 FP64 FMA per clock per SM, measured 5.81e11 FMA/s
    FP64_PEAK_T = 0.581

    UNITS = {"hbm": ("GB/s", 1e9, hbm_peak), "fp64": ("T FP64 FMA/s", 1e12, FP64_PEAK_T),
             "alu": ("T FP32-pipe op/s", 1e12, FP32_PIPE_PEAK_T)}

    def roofs(profile, units):
        """Per class: achieved = its algorithmic units over the timed region / its
        summed device time, against each bound; the bound with the highest
        fraction of its peak is the one that binds, the others sit beside it."""
        out = {}
        for k, bounds in units.items():
            ms, n = profile.get(k, (0.0, 0))
            if n == 0 or ms <= 0.0:
                continue
            cand, info = [], {}
            for bound, total in bounds:
                # "fp64_equiv": the float64 form's work of a float-pair kernel,
                # against the FP64 rate; reported beside the bound, never as it
                unit, scale, peak = UNITS["fp64" if bound == "fp64_equiv" else bound]
                ach = total / (ms / 1e3) / scale
                if bound == "fp64_equiv":
                    info[bound] = ach / peak
                    continue
                cand.append({"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                             "frac": ach / peak})
            best = dict(max(cand, key=lambda c: c["frac"]))
            best["other_bounds"] = {c["bound"]: c["frac"] for c in cand if c["bound"] != best["bound"]}
            best["other_bounds"].update(info)
            best["ms"] = ms
            best["launches"] = n
            best["ms_per_launch"] = ms / n
            out[k] = best
        return out

    def plan_levels_of(p):
        return [p.level(l) for l in range(p.num_levels)]

    mixed = prec == m.PREC_MIXED
    cpc = plan_cpc
    timed_solves = [c for cyc in cycles for c in cyc[:2]]
    lev_main = main_levels
    nc_main = ((lev_main[-1]["Nx"] - 2) * (lev_main[-1]["Ny"] - 2) * (lev_main[-1]["Nz"] - 1))
    units_main = class_units(lev_main, mixed, op_form == m.OP_SEPARABLE, timed_solves,
                             (plan_nu[0], plan_nu[1]), cpc, n_elem, nc_main)
    roof_kernels = roofs(prof_main, units_main)
    roof_f64 = None
    if prof_f64:
        nc64 = ((f64_levels[-1]["Nx"] - 2) * (f64_levels[-1]["Ny"] - 2) * (f64_levels[-1]["Nz"] - 1))
        roof_f64 = roofs(prof_f64, class_units(f64_levels, False, False, f64_solves,
                                               (plan_nu[0], plan_nu[1]), 1, n_elem, nc64,
                                               element_f64=True, with_recovery=False))
    dom = max((k for k in prof_main if prof_main[k][1] > 0), key=lambda k: prof_main[k][0])
    dom_roof = dict(roof_kernels.get(dom, {"bound": None}))
    dom_roof["kernel"] = dom
    dom_roof["traffic"] = None
    if dom in TRAFFIC_PER_UNIT and mixed:
        per_unit, how, form = TRAFFIC_PER_UNIT[dom]
        if form == args.op_form:
            dom_roof["traffic"] = per_unit * n_free / 4.0
            dom_roof["traffic_source"] = how
    dom_roof["peak_source"] = {
        "hbm": "measured: MEASURED_PEAKS.json hbm_gbs (burst copy)",
        "fp64": "measured: FP64 FMA issue rate of this GB300, 5.81e11/s",
        "alu": "FP32 pipe: 128 lanes x 152 SMs x 2.07 GHz"}.get(dom_roof.get("bound"))

    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        plan = None
        del X, Y, Z, U0, U0N
        torch.cuda.empty_cache()
        batched = run_batched(steps=2, warmup=1, autotune_on=not args.no_autotune)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_subprocess()
        if lam_cold_h is not None:
            cpu["full_size"] = oracle_full_size(case, lam_cold_h, case.u0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == m.PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": f"{nx}x{ny}x{nz}-cell terrain-following domain (400 hills + ridge, "
                               f"u0 from a 100x100 coarse wind): assemble + hierarchy, cold solve + "
                               f"recover, 2%-perturbed warm solve + recover, to rtol {RTOL}",
                   "cells": [nx, ny, nz], "n_free": n_free, "precision": args.precision,
                   "op_form": args.op_form if prec == m.PREC_MIXED else "stored",
                   "workspace_gb": plan_ws / 1e9,
                   "rtol": RTOL, "levels": plan_levels if False else None,
                   "l2": "inputs larger than L2 (X, Y, Z, u0, u0' = %.1f GB resident)" % (
                       9 * n_nodes * 8 / 1e9),
                   "replicas": world,
                   "cycles_per_check": plan_cpc},
        "gpu_launches": int(launches),
        "cycles_per_step": {"cold": cycles[-1][0], "warm": cycles[-1][1]},
        "rel_res": {"cold": cycles[-1][2], "warm": cycles[-1][3]},
        "rate": {"cold": cycles[-1][4], "warm": cycles[-1][5]},
        "phases_ms": {"setup": float(phases[:, 0].mean()), "cold_solve": float(phases[:, 1].mean()),
                      "recover_warm_solve": float(phases[:, 2].mean()),
                      "recover": float(phases[:, 3].mean())},
        "time_to_1e-8": tt,
        "vcycle_rate": {k: n_free * v["cold_cycles"] / v["cold_s"] for k, v in tt.items()},
        "wall_s": wall,
        "ms_per_step_unprofiled_graphs": ms_unprofiled,
        "roofline": dom_roof,
        "roofline_kernels": roof_kernels,
        "roofline_kernels_f64_solve": roof_f64,
        "profile_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in prof_main.items() if v[1]},
        "profile_ms_f64_solve": ({k: {"ms": v[0], "launches": v[1]} for k, v in prof_f64.items()
                                  if v[1]} if prof_f64 else None),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "batched_96_domains": batched,
        "clocks": clk,
        "input_gen_s": t_gen,
    }
    line["config"].pop("levels")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
