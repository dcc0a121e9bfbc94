#!/usr/bin/env python
"""Benchmark: FP64 TENO-AA SSP-RK3 steps on the 3D 256^3 periodic workload.

One step = the per-problem CFL reduction (teno_cfl_dt) followed by one SSP-RK3
step (teno_rk3_step, three right-hand-side evaluations with x/y/z face sweeps
and the stage combinations), all on the device, dt kept on the device.
value = cell-updates/s over all ranks (each rank advances its own independent
256^3 problem: weak scaling, no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--scheme 8|10|12]
  python bench.py --impl reference      # the CPU oracle on the host cores

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 TENO-AA cell-updates/s, 3D 256^3"
UNIT = "cell-updates/s"
N_SM = 152
FP64_FLOP_PER_CLK_SM = 4          # 2 DFMA lanes per SM per clock (1.25 TFLOP/s at 2.07 GHz)
SM_MAX_MHZ = 2070.0
HBM_BYTES_PER_CELL_UPDATE_3D = 320.0   # 3 fused stages: 80 + 120 + 120 B (ncons = 5)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scheme", type=int, default=10, choices=[8, 10, 12])
    ap.add_argument("--n", "--size", dest="n", type=int, default=256,
                    help="cells per axis of the 3D workload (--size under torchrun, whose "
                         "own options shadow --n)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-noh", action="store_true")
    ap.add_argument("--no-teno12", action="store_true",
                    help="skip the TENO12-AA line (same workload, twelve-point scheme)")
    ap.add_argument("--no-teno8", action="store_true",
                    help="skip the TENO8-AA line (same workload, eight-point scheme)")
    ap.add_argument("--no-2d", action="store_true",
                    help="skip the 2D 1024^2 four-quadrant line")
    ap.add_argument("--2d-only", dest="quadrants_2d_only", action="store_true",
                    help="run only the 2D four-quadrant line and print its record (profiling)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched workload and print its record (profiling)")
    ap.add_argument("--batched-no-reference", action="store_true",
                    help="skip the per-problem launch loop of the batched record (profiling: "
                         "it is tens of thousands of launches)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint workload and print its record (profiling)")
    ap.add_argument("--adjoint-n", type=int, default=512)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--fd-directions", type=int, default=16,
                    help="seeded directions of the adjoint's central-difference check")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# algorithmic FP64 work (add/sub/mul/div/sqrt = 1 flop, fma = 2 flops),
# counted from the operations the method prescribes per face and per cell
# ---------------------------------------------------------------------------

def flops_per_cell_sweep(nd):
    # the plain method's per-cell work: primitive variables, sound speed,
    # enthalpy, sqrt(rho), physical flux (4 nd + 11) and the three
    # characteristic speeds |u-c|, |u+c|, |u|+c
    return 4 * nd + 11 + 3


def flops_face_fixed(nd, H):
    """The plain method's fixed FP64 work per face (Roe average,
    eigenvectors, projection of the 2H stencil cells, splitting,
    back-projection)."""
    nc = nd + 2
    roe = 6 * nd + 17
    eig = 3 * nd + 14
    proj = nc * 2 * H * 2 * (2 * nc - 1)
    split = nc * 2 * H * 6
    back = nc * (2 * nc - 1) + nc
    return roe + eig + proj + split + back


# FP64 instructions (DADD, DMUL, DFMA) of one double division and one double
# square root as the compiler expands them on sm_103a, measured with ncu from
# the instruction counts of prims_kernel (one division, two square roots per
# cell) and wave_max_kernel (one of each) minus their other operations.
KDIV = {"dadd": 0.0, "dmul": 0.0, "dfma": 5.0}
KSQRT = {"dadd": 0.0, "dmul": 3.0, "dfma": 5.0}
FP64_LANES_PER_CLK_SM = 2        # FP64 pipe: 2 lanes per SM per clock (DADD, DMUL or DFMA)


def _acc(tot, add=0.0, mul=0.0, fma=0.0, div=0.0, sqrt=0.0, w=1.0):
    tot["dadd"] += w * (add + div * KDIV["dadd"] + sqrt * KSQRT["dadd"])
    tot["dmul"] += w * (mul + div * KDIV["dmul"] + sqrt * KSQRT["dmul"])
    tot["dfma"] += w * (fma + div * KDIV["dfma"] + sqrt * KSQRT["dfma"])


def face_fp64_instructions(nd, H, hist, exact_frac, tf=32):
    """FP64 instructions the face-sweep kernel executes per face, by kind,
    following its code: staged cells formed from the stored primitives
    (flux, halving, speeds), Roe average and eigenvector rows, projection of
    the halved staged values, one fma per split value, the 2H - 1 shifted
    values the decision filter reads, each reconstruction's value formula
    for its decided outcome (hist: fractions of fallback, S3 .. S_H) or the
    whole method on the exact path (exact_frac), and the back-projection.
    The filter's own single-precision and integer work is not FP64."""
    nc, W = nd + 2, 2 * H
    nrec = 2 * nc
    t = {"dadd": 0.0, "dmul": 0.0, "dfma": 0.0}
    staged = (tf + W - 1) / tf
    _acc(t, add=5, mul=nd + 1 + 2 * nc, w=staged)                       # staged cells
    _acc(t, add=2, mul=2 * nd + 12, fma=2 * nd, div=2, sqrt=1)         # Roe state
    _acc(t, add=5, mul=5 * nd + 2)                                     # eigenvector rows
    _acc(t, mul=3 * W * 2, fma=3 * W * 2 * (nc - 1))                   # acoustic, entropy
    _acc(t, add=(nd - 1) * W * 2, mul=(nd - 1) * W * 2)                # shear fields
    _acc(t, fma=nc * 2 * W)                                            # split values
    _acc(t, add=nrec * (W - 1))                                        # shifted values
    for sel in range(5):                                               # decided values
        f = hist[sel] * nrec * (1.0 - exact_frac)
        if sel == 0:
            _acc(t, add=6, mul=8, fma=2, div=3, w=f)
        else:
            _acc(t, mul=1, fma=2 * (sel + 2) - 1, w=f)
    _acc(t, add=nc + nd + 3, mul=nc + 1, fma=(nd - 1) + 2 * nc)        # back-projection
    exact = exact_frac * nrec * sum(hist[s] * recon_flops(H, s) for s in range(5))
    return t, exact


def executed_fp64_per_face(hist, exact_frac, nd, H):
    """FP64 flops the face kernel executes per face (add/mul 1, fma 2),
    from face_fp64_instructions."""
    t, exact = face_fp64_instructions(nd, H, hist, exact_frac)
    return t["dadd"] + t["dmul"] + 2.0 * t["dfma"] + exact


def executed_fp64_instr_per_face(hist, exact_frac, nd, H):
    """FP64 instructions (thread level: DADD, DMUL, DFMA, each one slot of
    the FP64 pipe) the face kernel executes per face; the rare exact-path
    reconstructions counted as if all their flops were fmas (a lower bound)."""
    t, exact = face_fp64_instructions(nd, H, hist, exact_frac)
    return t["dadd"] + t["dmul"] + t["dfma"] + 0.5 * exact


def fp64_roofline(hist, exact_frac, nd, H, faces_per_launch, avg_launch_s, method_fpf):
    """The face kernel against the FP64 pipe: executed FP64 instructions per
    second over the pipe's 2 lanes per SM per clock (the binding resource),
    with the same work in flops against the DFMA peak, and the plain
    method's op count over the same time."""
    ipf = executed_fp64_instr_per_face(hist, exact_frac, nd, H)
    fpf = executed_fp64_per_face(hist, exact_frac, nd, H)
    peak_i = N_SM * FP64_LANES_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e9
    peak_f = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    ach_i = ipf * faces_per_launch / avg_launch_s / 1e9
    ach_f = fpf * faces_per_launch / avg_launch_s / 1e12
    ach_m = method_fpf * faces_per_launch / avg_launch_s / 1e12
    return {
        "bound": "alu", "kernel": "face_kernel (x/y/z face sweeps)",
        "achieved": ach_i, "peak": peak_i, "unit": "G FP64 instr/s", "frac": ach_i / peak_i,
        "peak_source": "derived: 152 SM x 2 FP64 lanes/clk x 2.07 GHz (DADD, DMUL and DFMA "
                       "each take one lane slot)",
        "counted": "FP64 instructions executed per face, counted from the kernel's code with "
                   "the live decision mix and exact-path fraction (div/sqrt expansions measured "
                   "with ncu); ncu counts about 3 % more (sign and absolute-value operations)",
        "fp64_instr_per_face": ipf,
        "flops": {"achieved": ach_f, "peak": peak_f, "unit": "TFLOP/s", "frac": ach_f / peak_f,
                  "fp64_flops_per_face": fpf,
                  "note": "the same work in flops (fma 2) against the all-DFMA peak"},
        "method_equivalent": {"achieved": ach_m, "frac": ach_m / peak_f, "unit": "TFLOP/s",
                              "flops_per_face": method_fpf,
                              "note": "the plain method's FP64 op count per face / the same "
                                      "time; above 1 because the certified filter takes most "
                                      "decisions in FP32"},
    }


def beta_large_flops(w):
    k = w - 1                          # non-zero shifted values
    return k + k * k + 2 * k - 1


def selection_class(flags_np, H):
    """Per decision byte: L - 2 of the selected large stencil S_L (1..4) or 0
    for the small-stencil fallback (S6 of the twelve-point scheme is written
    with bits 0-4 zero)."""
    import numpy as np
    sel = (flags_np & 3).astype(np.int64)
    if H == 6:
        sel[(flags_np & 31) == 0] = 4
    return sel


def recon_flops(H, sel):
    """Algorithmic flops of one reconstruction given its selection class."""
    base = 48 + 33 + 18 + 2            # C_T measure, small indicators, their gammas, sum
    tested = []
    for L in range(H, 2, -1):
        tested.append(L)
        if sel == L - 2:
            break
    f = base
    for L in tested:
        f += beta_large_flops(2 * L) + 8
    if sel:
        f += 2 * (2 * sel + 4) - 1     # linear scheme of S_(sel+2), width 2(sel+2)
    else:
        f += 29
    return f


def flops_per_face_from_flags(flags_np, nd, H):
    import numpy as np
    hist = np.bincount(selection_class(flags_np, H), minlength=5).astype(np.float64)
    nrec = flags_np.size
    per = {s: recon_flops(H, s) for s in range(5)}
    tot_rec = sum(hist[s] * per[s] for s in range(5))
    nfaces = nrec / ((nd + 2) * 2)
    return flops_face_fixed(nd, H) + flops_per_cell_sweep(nd) + tot_rec / nfaces, hist / nrec


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(device_index)], stdout=self.fh,
                stderr=subprocess.DEVNULL)
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
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4)
                          if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload)
# ---------------------------------------------------------------------------

def oracle_sample_rate(U, n, scheme, target_s, threads):
    """One SSP-RK3 step of the oracle on a periodic z-slab n x n x nz of the
    same field (identical per-cell work); nz chosen for ~target_s seconds."""
    import numpy as np
    import oracle
    oracle.build()
    U5 = U.reshape(5, n, n, n)
    H = scheme // 2

    def slab(nz):
        Us = np.ascontiguousarray(U5[:, :nz]).reshape(5, -1)
        p = oracle.params(3, [n, n, nz], [2 * np.pi / n] * 3, scheme=scheme, bc=0)
        return p, Us

    p, Us = slab(H)
    t0 = time.perf_counter()
    oracle.rhs(p, Us, threads=threads)
    t_rhs = time.perf_counter() - t0
    per_cell_step = 3.0 * t_rhs / (n * n * H)
    nz = int(max(H, min(n, target_s / max(per_cell_step * n * n, 1e-9))))
    p, Us = slab(nz)
    dt, _, _ = oracle.cfl_dt(p, Us, 0.4)
    t0 = time.perf_counter()
    oracle.rk3_step(p, Us, dt, threads=threads)
    t = time.perf_counter() - t0
    cells = n * n * nz
    return cells / t, "1 SSP-RK3 step of TENO%d-AA on a periodic %dx%dx%d z-slab of the same " \
        "field (%d cells), %d OpenMP threads" % (scheme, n, n, nz, cells, threads), nz


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------

def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, cells_per_rank: int, steps: int, seconds: float) -> float:
    """Cell-updates per second of the whole job: every rank advances its own
    problem of cells_per_rank cells by steps steps (weak scaling)."""
    return world * cells_per_rank * steps / seconds


def workload_desc(n, scheme):
    """The benchmark workload, the same string on both arms."""
    return ("3D Euler %d^3 periodic on [0,2pi]^3, Taylor-Green Mach 0.5 + seeded k^-5/3 "
            "solenoidal field (10%% rms), TENO%d-AA, LLF, CFL 0.4; step = CFL time step + "
            "SSP-RK3 step" % (n, scheme))


def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle
    import workloads
    oracle.build()
    n, scheme = args.n, args.scheme
    case = workloads.tgv_3d(n, scheme=scheme)
    threads = host_cores()
    H = scheme // 2
    nz = max(H, 8)
    U5 = case["U"].reshape(5, n, n, n)
    Us = np.ascontiguousarray(U5[:, :nz]).reshape(5, -1)
    p = oracle.params(3, [n, n, nz], [2 * np.pi / n] * 3, scheme=scheme, bc=0)
    for _ in range(args.warmup):
        dt, _, _ = oracle.cfl_dt(p, Us, 0.4)
        Us, _ = oracle.rk3_step(p, Us, dt, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dt, _, _ = oracle.cfl_dt(p, Us, 0.4)
        Us, _ = oracle.rk3_step(p, Us, dt, threads=threads)
    t = time.perf_counter() - t0
    cells = n * n * nz
    value = cells * args.steps / t
    sample = ("per step: CFL dt + 1 SSP-RK3 step of TENO%d-AA on a periodic %dx%dx%d z-slab "
              "of the 256^3 field, %d OpenMP threads" % (scheme, n, n, nz, threads))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(n, scheme), "scheme": scheme, "cells": n ** 3,
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_batched(args, dev, stream):
    """Batched 1D workload (4096 seeded Riemann problems, N ~ U{64..4096},
    schemes 8|10, 10 % near vacuum with the limiter): persistent kernels with
    the step captured in a CUDA graph (autotuned) vs one teno_cfl_dt +
    teno_rk3_step per problem, from the same state; states compared bitwise."""
    import numpy as np
    import torch

    import paper_2109_14340_gb300 as T
    import workloads
    cases = workloads.batched_1d(count=args.batch_count)
    sizes = [c["n"][0] for c in cases]
    offs, total = T.pack_offsets(sizes)
    U = np.zeros(total)
    probs = []
    for c, o in zip(cases, offs):
        n = c["n"][0]
        U[o:o + 3 * n] = c["U"].ravel()
        probs.append(dict(n=n, offset=o, dx=c["dx"][0], scheme=c["scheme"],
                          limiter=c.get("limiter", 0), bc_lo=c["bc_lo"][0], bc_hi=c["bc_hi"][0]))
    cells = int(sum(sizes))
    common = T.teno_params_init(gamma=1.4)
    B = T.Batch(common, probs, dev)
    scratch = torch.from_numpy(U.copy()).to(dev)
    tile, bps = B.autotune(scratch)
    del scratch

    def timed(mode, k, Ud):
        B.steps(Ud, 1, 0.4, mode, stream)            # warm-up (captures the graph)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.steps(Ud, k, 0.4, mode, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e-3

    k_b = max(3, args.steps)
    clocks = ClockSampler(dev.index)
    t_b = timed(T.TENO_BATCH_GRAPH, k_b, torch.from_numpy(U.copy()).to(dev))
    clk = clocks.stop()
    v_b = cells * k_b / t_b
    if args.batched_no_reference:
        t_p = v_p = same = None
    else:
        t_p = timed(T.TENO_BATCH_PER_PROBLEM, 1, torch.from_numpy(U.copy()).to(dev))
        Ua = torch.from_numpy(U.copy()).to(dev)
        Ub = torch.from_numpy(U.copy()).to(dev)
        B.steps(Ua, 2, 0.4, T.TENO_BATCH_GRAPH, stream)
        B.steps(Ub, 2, 0.4, T.TENO_BATCH_PER_PROBLEM, stream)
        torch.cuda.synchronize(dev)
        same = bool(torch.equal(Ua, Ub))
        v_p = cells * 1 / t_p
    # FP64 roofline of the step's face sweeps against the whole step's time
    # (the kernels inside one CUDA graph are not timed apart); every
    # reconstruction counted at its cheapest outcome, the largest stencil's
    # value, so the figure is a lower bound of the work done
    flops = instr = 0.0
    for scheme in (8, 10):
        H = scheme // 2
        hist = [0.0] * 5
        hist[H - 2] = 1.0
        ti, _ = face_fp64_instructions(1, H, hist, 0.0, tf=tile)
        nf = 3 * sum(c["n"][0] + 1 for c in cases if c["scheme"] == scheme)
        flops += nf * (ti["dadd"] + ti["dmul"] + 2.0 * ti["dfma"])
        instr += nf * (ti["dadd"] + ti["dmul"] + ti["dfma"])
    peak = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak_i = N_SM * FP64_LANES_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e9
    achieved = flops / (t_b / k_b) / 1e12
    achieved_i = instr / (t_b / k_b) / 1e9
    return {"workload": "%d independent 1D Riemann problems, N ~ U{64..4096} (%d cells), "
                        "TENO8|10 50/50, 10%% near vacuum with limiter, per-problem CFL 0.4"
                        % (len(probs), cells),
            "value": v_b, "unit": UNIT, "ms_per_step": 1e3 * t_b / k_b,
            "per_problem_value": v_p,
            "per_problem_ms_per_step": None if t_p is None else 1e3 * t_p,
            "speedup": None if v_p is None else v_b / v_p, "identical_states": same,
            "autotuned": {"tile_faces": tile, "warps_per_tile": tile // 32,
                          "blocks_per_sm": bps},
            "clocks": clk,
            "roofline": {"bound": "alu", "kernel": "batch_face_kernel (3 per step) + small "
                                                  "kernels, one CUDA graph",
                         "achieved": achieved_i, "peak": peak_i, "unit": "G FP64 instr/s",
                         "frac": achieved_i / peak_i,
                         "flops": {"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                   "frac": achieved / peak},
                         "counted": "FP64 instructions the three persistent face sweeps of a "
                                    "step execute (largest-stencil value for every "
                                    "reconstruction, primitives read from the stored rows), over "
                                    "the whole step's time: a lower bound"},
            "mode": "persistent (problem, tile) work list, step captured in a CUDA graph"}


def run_adjoint(args, dev, stream):
    """2D 512^2 TENO8-AA, Mach-2 oblique-shock flow with seeded entropy /
    vortex perturbations, 200 RK3 steps at the dt of the initial state,
    checkpoints every 20; loss = 1/2 ||rho(T) - rho_target||^2 with the
    target from a seeded 1e-3 perturbation of the initial state.  Reports
    backward (incl. recompute) / forward time and central differences of the
    frozen-decision map along seeded directions against the gradient."""
    import torch

    import paper_2109_14340_gb300 as T
    import workloads
    n, nsteps, every = args.adjoint_n, args.adjoint_steps, 20
    c = workloads.adjoint_2d(n)
    p = T.teno_params_init(ndim=2, n=c["n"], dx=c["dx"], scheme=8, bc_lo=c["bc_lo"],
                           bc_hi=c["bc_hi"])
    s = T.Solver(p, dev)
    U0 = torch.from_numpy(c["U"]).to(dev)
    dt = float(s.cfl_dt(U0, 0.4).item())
    rho_t = T.rollout(p, torch.from_numpy(c["U_target_ic"]).to(dev), dt, nsteps, every)[0].detach()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # warm-up (module load) on a short horizon
    Uw = U0.clone().requires_grad_(True)
    (0.5 * ((T.rollout(p, Uw, dt, 2, 1)[0] - rho_t) ** 2).sum()).backward()
    torch.cuda.synchronize(dev)
    U0g = U0.clone().requires_grad_(True)
    e0, e1, e2 = ev(), ev(), ev()
    e0.record(stream)
    UT = T.rollout(p, U0g, dt, nsteps, every)
    loss = 0.5 * ((UT[0] - rho_t) ** 2).sum()
    e1.record(stream)
    loss.backward()
    e2.record(stream)
    torch.cuda.synchronize(dev)
    t_f = e0.elapsed_time(e1) * 1e-3
    t_b = e1.elapsed_time(e2) * 1e-3
    grad = U0g.grad
    # the recompute share: the same number of recorded steps on their own
    fws = T.aligned_workspace(T.teno_workspace_bytes(p), dev)
    flb = T.teno_flags_bytes(p)
    U = U0.clone()
    fls = []
    e3, e4 = ev(), ev()
    e3.record(stream)
    for _ in range(nsteps):
        U1, U2 = torch.empty_like(U), torch.empty_like(U)
        fl = torch.empty(3 * flb, dtype=torch.uint8, device=dev)
        T.teno_rk3_step_record_sel(p, U, dt, U1, U2, fl, fws)
        fls.append(fl)
        del U1, U2
    e4.record(stream)
    torch.cuda.synchronize(dev)
    t_rec = e3.elapsed_time(e4) * 1e-3

    def frozen(Ustart):
        Uf = Ustart.clone()
        for fl in fls:
            T.teno_rk3_step_frozen(p, Uf, dt, fl, fws)
        return 0.5 * float(((Uf[0] - rho_t) ** 2).sum())

    scale = U0.abs().amax(dim=1, keepdim=True)
    errs = []
    for seed in range(5003, 5003 + args.fd_directions):
        v = torch.from_numpy(workloads.smooth_field((4, n, n), seed).reshape(4, -1)).to(dev) * scale
        h = 1e-6
        fd = (frozen(U0 + h * v) - frozen(U0 - h * v)) / (2 * h)
        ad = float((grad * v).sum())
        errs.append(abs(fd - ad) / abs(ad))
    del fls
    return {"workload": "2D Euler %dx%d TENO8-AA, Mach-2 oblique shock + entropy/vortex, "
                        "transmissive x / periodic y, %d steps at fixed dt, checkpoints every %d"
                        % (n, n, nsteps, every),
            "forward_s": t_f, "backward_s": t_b, "cost_ratio": t_b / t_f,
            "cost_ratio_excluding_recompute": (t_b - t_rec) / t_f,
            "fd_frozen_decisions_max_rel_err": max(errs),
            "fd_frozen_decisions_median_rel_err": float(sorted(errs)[len(errs) // 2]),
            "fd_directions": len(errs),
            "vjp_face_kernel_fp64_pipe_busy": read_adjoint_fp64_busy(),
            "vjp_face_kernel_fp64_pipe_busy_source": "ncu, profiles/adjoint_2d.md (512^2, the "
                                                     "two reverse face sweeps averaged)",
            "loss": float(loss.detach())}


def run_noh(args, dev, stream, n=64, scheme=10, t_end=0.6):
    """3D Noh implosion (Sec. 5.5) at 64^3 to t = 0.6: symmetry walls, inflow
    faces as Dirichlet states with the analytic density, updated every step
    from the host; Rusanov, limiter on.  Reports the rate of the whole loop
    (CFL reduction read back for the host-side time, boundary states copied
    in, RK3 step) and the solution against Eq. density_noh."""
    import numpy as np
    import torch

    import paper_2109_14340_gb300 as T
    import workloads
    c = workloads.noh_3d(n, scheme=scheme)
    st = [torch.from_numpy(a).to(dev) for a in workloads.noh_inflow_states(c, 0.0)]
    p = T.teno_params_init(ndim=3, n=c["n"], dx=c["dx"], scheme=scheme, gamma=c["gamma"],
                           bc_lo=c["bc_lo"], bc_hi=c["bc_hi"], flux_split=c["split"],
                           limiter=c["limiter"], bc_state_hi=st)
    S = T.Solver(p, dev)
    U = torch.from_numpy(c["U"]).to(dev)
    torch.cuda.synchronize(dev)
    t, steps = 0.0, 0
    t0 = time.perf_counter()
    while t < t_end - 1e-12:
        for d, a in enumerate(workloads.noh_inflow_states(c, t)):
            st[d].copy_(torch.from_numpy(a))
        dt = min(float(S.cfl_dt(U, 0.4).item()), t_end - t)
        S.step(U, dt=dt)
        t += dt
        steps += 1
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    nonphys = S.status()
    # diagnostics of the final state from one right-hand side with the
    # decision record: selections, C_T exponents, faces where the limiter bound
    _, rec = S.rhs(U, dt, flags=True)
    d0, d1, l0, _ = T.record_layout(p)
    rec = rec.cpu().numpy()
    _, hist = flops_per_face_from_flags(rec[:d1], 3, scheme // 2)
    diag = {"selection_mix": selection_mix(hist, scheme),
            "ct_exponent_mix": ct_exponent_hist(rec[:d1]),
            "limiter_faces_frac": float(rec[l0:].mean())}
    S.status()
    L = c["L"]
    dx = L / n
    cc = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(cc, cc, cc, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z).ravel()
    rho = U[0].cpu().numpy()
    R = t / 3.0
    shell = np.floor(r / dx).astype(int)
    k = np.arange(int(L / dx))
    prof = np.array([rho[shell == i].mean() for i in k])
    rc = np.array([r[shell == i].mean() for i in k])
    ex = workloads.noh_density(rc, t)
    r40 = float(rc[int(np.argmax((prof < 40.0) & (rc > 0.5 * R)))])
    pre = rc > R + 6 * dx
    post = (rc > 0.4 * R) & (rc < R - 4 * dx)
    cell_pre = r > R + 6 * dx
    exc = workloads.noh_density(r[cell_pre], t)
    return {"workload": "3D Noh implosion %d^3 on [0,0.256]^3, gamma 5/3, TENO%d-AA, Rusanov, "
                        "limiter, symmetry walls + Dirichlet inflow, to t = %.1f" % (n, scheme, t_end),
            "steps": steps, "seconds": el, "value": n ** 3 * steps / el, "unit": "cell-updates/s",
            "nonphysical": nonphys, "shock_radius": r40, "shock_radius_exact": R,
            "pre_shock_shell_err_max": float((np.abs(prof[pre] - ex[pre]) / ex[pre]).max()),
            "post_shock_mean_density": float(prof[post].mean()), "post_shock_exact": 64.0,
            "pre_shock_cell_scatter_p99": float(np.percentile(np.abs(rho[cell_pre] - exc) / exc, 99)),
            "final_state_decisions": diag}


def ct_exponent_hist(flags_np):
    """Fractions of reconstructions per C_T exponent [beta] = 7 .. 14 (bits
    5-7 of each decision byte hold [beta] - 7)."""
    import numpy as np
    h = np.bincount((flags_np >> 5).astype(np.int64), minlength=8).astype(np.float64)
    h /= max(1, flags_np.size)
    return {str(7 + k): float(h[k]) for k in range(8)}


def selection_mix(hist, scheme):
    mix = {"fallback": hist[0], "S3": hist[1], "S4": hist[2]}
    for L in range(5, scheme // 2 + 1):
        mix["S%d" % L] = hist[L - 2]
    return mix


def run_scheme_leg(args, dev, stream, scheme, n=256, steps=3):
    """The same 256^3 workload with another scheme width (the eight-point
    TENO8-AA of the 3D configuration, the twelve-point TENO12-AA): time per
    step, rate and the face kernel's FP64 roofline fraction (executed flops
    per face / live average launch time)."""
    import torch

    import paper_2109_14340_gb300 as T
    import workloads
    case = workloads.tgv_3d(n, seed=3001, scheme=scheme)
    p = T.teno_params_init(ndim=3, n=[n, n, n], dx=case["dx"], scheme=scheme,
                           bc_lo=[0, 0, 0], bc_hi=[0, 0, 0])
    solver = T.Solver(p, dev)
    U = torch.from_numpy(case["U"]).to(dev)

    def step():
        solver.cfl_dt(U)
        solver.step(U)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    _, flags = solver.rhs(U, flags=True)
    fl_np = flags.cpu().numpy()[:T.record_layout(p)[1]]      # decision bytes
    fpf, hist = flops_per_face_from_flags(fl_np, 3, scheme // 2)
    ct_hist = ct_exponent_hist(fl_np)
    del flags, fl_np
    clocks = ClockSampler(dev.index)
    T.teno_profile_enable(True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    face_ms, face_launches, face_faces, face_exact = T.teno_profile_read()
    T.teno_profile_enable(False)
    clk = clocks.stop()
    peak = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    avg_launch_s = face_ms * 1e-3 / max(face_launches, 1)
    faces_per_launch = face_faces / max(face_launches, 1)
    exact_frac = face_exact / max(face_faces * 2 * 5, 1)
    traffic_pf = read_traffic_per_face(scheme)
    roof = fp64_roofline(hist, exact_frac, 3, scheme // 2, faces_per_launch, avg_launch_s, fpf)
    roof.update({"exact_path_fraction": exact_frac, "avg_launch_ms": avg_launch_s * 1e3,
                 "traffic": (traffic_pf * faces_per_launch) if traffic_pf else None,
                 "face_kernel_share": face_ms / ms if ms > 0 else None,
                 "selection_mix": selection_mix(hist, scheme), "ct_exponent_mix": ct_hist})
    return {
        "workload": "the same 256^3 Taylor-Green + k^-5/3 field with TENO%d-AA, LLF, CFL 0.4"
                    % scheme,
        "steps": steps, "ms_per_step": ms / steps, "value": n ** 3 / (ms / steps * 1e-3),
        "unit": UNIT, "nonphysical": solver.status(), "clocks": clk, "roofline": roof,
    }


def run_2d_leg(args, dev, stream, scheme=10, n=1024, warm=45, steps=20):
    """The 2D four-quadrant Riemann problem at 1024^2 (TENO10-AA,
    transmissive sides, CFL 0.4), timed after `warm` steps, when rounding
    noise has spread over its constant states (the decisions there follow
    the noise, which the decision filter must still certify): rate, the
    share of reconstructions that reached the exact FP64 path, and the face
    kernel's FP64 roofline fraction."""
    import torch

    import paper_2109_14340_gb300 as T
    import workloads
    case = workloads.quadrants_2d(n, scheme=scheme)
    p = T.teno_params_init(ndim=2, n=case["n"], dx=case["dx"], scheme=scheme,
                           bc_lo=case["bc_lo"], bc_hi=case["bc_hi"])
    solver = T.Solver(p, dev)
    U = torch.from_numpy(case["U"]).to(dev)

    def step():
        solver.cfl_dt(U)
        solver.step(U)

    for _ in range(warm):
        step()
    torch.cuda.synchronize(dev)
    _, flags = solver.rhs(U, flags=True)
    fl_np = flags.cpu().numpy()[:T.record_layout(p)[1]]      # decision bytes
    fpf, hist = flops_per_face_from_flags(fl_np, 2, scheme // 2)
    del flags, fl_np
    clocks = ClockSampler(dev.index)
    T.teno_profile_enable(True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    face_ms, face_launches, face_faces, face_exact = T.teno_profile_read()
    T.teno_profile_enable(False)
    clk = clocks.stop()
    avg_launch_s = face_ms * 1e-3 / max(face_launches, 1)
    faces_per_launch = face_faces / max(face_launches, 1)
    exact_frac = face_exact / max(face_faces * 2 * 4, 1)
    roof = fp64_roofline(hist, exact_frac, 2, scheme // 2, faces_per_launch, avg_launch_s, fpf)
    roof.update({"exact_path_fraction": exact_frac, "avg_launch_ms": avg_launch_s * 1e3,
                 "traffic": None, "face_kernel_share": face_ms / ms if ms > 0 else None,
                 "selection_mix": selection_mix(hist, scheme)})
    return {
        "workload": "2D Euler %dx%d four-quadrant Riemann problem + entropy wave, TENO%d-AA, "
                    "LLF, transmissive sides, CFL 0.4, timed after %d steps" % (n, n, scheme, warm),
        "steps": steps, "ms_per_step": ms / steps, "value": n * n / (ms / steps * 1e-3),
        "unit": UNIT, "nonphysical": solver.status(), "clocks": clk, "roofline": roof,
    }


def measured_hbm_peak():
    """HBM copy bandwidth from MEASURED_PEAKS.json (measured on this machine's
    GB300s), else the profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def read_adjoint_fp64_busy():
    """The reverse face kernel's FP64-pipe busy fraction from the committed
    ncu summary (a line 'fp64_pipe_busy[adj_face_kernel]: <value>')."""
    path = os.path.join(ROOT, "profiles", "adjoint_2d.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"fp64_pipe_busy\[adj_face_kernel\]:\s*([0-9.eE+-]+)", open(path).read())
    return float(m.group(1)) if m else None


def read_traffic_per_face(scheme):
    """Measured DRAM bytes per face of the face sweep, from the committed ncu
    summary (a line 'traffic_bytes_per_face[TENO<s>]: <value>')."""
    path = os.path.join(ROOT, "profiles", "face_sweep_3d.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"traffic_bytes_per_face\[TENO%d\]:\s*([0-9.eE+-]+)" % scheme, open(path).read())
    return float(m.group(1)) if m else None


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2109_14340_gb300 as T
    import workloads
    from paper_2109_14340_gb300 import _build
    _build.build()
    T.load()

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    n, scheme = args.n, args.scheme
    case = workloads.tgv_3d(n, seed=3001 + rank, scheme=scheme)
    p = T.teno_params_init(ndim=3, n=[n, n, n], dx=case["dx"], scheme=scheme,
                           bc_lo=[0, 0, 0], bc_hi=[0, 0, 0])
    solver = T.Solver(p, dev)
    U = torch.from_numpy(case["U"]).to(dev)
    cells = n ** 3
    stream = torch.cuda.current_stream(dev)

    def step():
        solver.cfl_dt(U)
        solver.step(U)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    U_w = U.clone()          # the state the timed steps start from (also the e2e's)

    # decision histogram of the current state (untimed) -> algorithmic flops
    _, flags = solver.rhs(U, flags=True)
    fl_np = flags.cpu().numpy()[:T.record_layout(p)[1]]      # decision bytes only
    fpf, hist = flops_per_face_from_flags(fl_np, 3, scheme // 2)
    ct_hist = ct_exponent_hist(fl_np)
    del flags, fl_np

    clocks = ClockSampler(local_rank)
    T.teno_profile_enable(True)
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1)
    face_ms, face_launches, face_faces, face_exact = T.teno_profile_read()
    T.teno_profile_enable(False)
    clk = clocks.stop()
    nonphys = solver.status()

    t_max = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(world, cells, args.steps, t_max * 1e-3)

    # e2e: host buffers through teno_advance_host, one step per call
    # (H2D of the state, CFL + RK3 step, D2H of the state, every step), from
    # the state the timed steps started from (the first steps of the field
    # cost more: its initial small scales take more fallbacks)
    Uh = U_w.cpu().pin_memory()
    Ud2 = torch.empty_like(U_w)
    ws2 = torch.zeros_like(solver.ws)
    T.teno_advance_host(p, Uh, Ud2, 1, 0.4, ws2)         # warm
    k_e2e = max(1, min(args.steps, 3))
    e2e_clocks = ClockSampler(local_rank)
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        T.teno_advance_host(p, Uh, Ud2, 1, 0.4, ws2)
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_clk = e2e_clocks.stop()
    e2e_value = whole_job_rate(world, cells, k_e2e, t_e2e)
    # context: the same step with every decision evaluated in FP64 (filter
    # off), and one step from the same state both ways compared bitwise
    Ua, Ub = U.clone(), U.clone()
    solver.cfl_dt(Ua)
    solver.step(Ua)
    T.teno_set_decision_filter(False)
    try:
        solver.cfl_dt(Ub)
        solver.step(Ub)
        step()
        torch.cuda.synchronize(dev)
        k_off = 2
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k_off):
            step()
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms_off = f0.elapsed_time(f1) / k_off
    finally:
        T.teno_set_decision_filter(True)
    filter_off = {"ms_per_step": ms_off, "value": cells / (ms_off * 1e-3),
                  "identical_step": bool(torch.equal(Ua, Ub)),
                  "note": "same step with the single-precision decision filter off (every "
                          "decision evaluated in FP64); outputs are identical either way"}
    del Ua, Ub

    state_bytes = 5 * cells * 8

    # FP64 probe (context): measured DFMA rate on this GPU
    probe = None
    try:
        import ctypes
        plib = ctypes.CDLL(_build.build_probe())
        plib.teno_probe_dfma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
        blocks = N_SM * 8
        sink = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
        pms = ctypes.c_double()
        ptot = ctypes.c_int64()
        rc = plib.teno_probe_dfma(blocks, 20000, ctypes.c_void_p(sink.data_ptr()),
                                  ctypes.byref(pms), ctypes.byref(ptot),
                                  ctypes.c_void_p(stream.cuda_stream))
        if rc == 0:
            probe = 2.0 * ptot.value / (pms.value * 1e-3) / 1e12
    except Exception:
        probe = None

    peak = N_SM * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    avg_launch_s = face_ms * 1e-3 / max(face_launches, 1)
    faces_per_launch = face_faces / max(face_launches, 1)
    exact_frac = face_exact / max(face_faces * 2 * 5, 1)
    traffic_pf = read_traffic_per_face(scheme)
    roof = fp64_roofline(hist, exact_frac, 3, scheme // 2, faces_per_launch, avg_launch_s, fpf)
    roof.update({"peak_probe_measured_tflops": probe,
                 "traffic": (traffic_pf * faces_per_launch) if traffic_pf else None,
                 "exact_path_fraction": exact_frac, "faces_per_launch": faces_per_launch,
                 "avg_launch_ms": avg_launch_s * 1e3,
                 "face_kernel_share": face_ms / ms if ms > 0 else None,
                 "selection_mix": selection_mix(hist, scheme), "ct_exponent_mix": ct_hist})
    launches_per_step = 3 + 3 * (2 + 3)       # CFL (2), primitives; per stage prepare, 3 sweeps, combine
    hbm_peak, hbm_src = measured_hbm_peak()
    batched = None
    if not args.no_batched:
        batched = run_batched(args, dev, stream)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(args, dev, stream)
    noh = None
    if not args.no_noh:
        noh = run_noh(args, dev, stream)
    teno12 = None
    if not args.no_teno12 and scheme != 12:
        teno12 = run_scheme_leg(args, dev, stream, 12, n=n)
    teno8 = None
    if not args.no_teno8 and scheme != 8:
        teno8 = run_scheme_leg(args, dev, stream, 8, n=n)
    quad2d = None
    if not args.no_2d:
        quad2d = run_2d_leg(args, dev, stream)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        threads = host_cores()
        rate, sample, _ = oracle_sample_rate(case["U"], n, scheme, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {
            "workload": workload_desc(n, scheme),
            "scheme": scheme, "cells": cells, "parallelism": "independent problem per GPU",
            "l2": "state 671 MB > 129 MB L2 (no flush needed)"},
        "roofline": roof,
        "roofline_hbm": {
            "bound": "hbm", "achieved": value * HBM_BYTES_PER_CELL_UPDATE_3D / 1e9,
            "peak": hbm_peak, "unit": "GB/s",
            "frac": value * HBM_BYTES_PER_CELL_UPDATE_3D / 1e9 / hbm_peak,
            "peak_source": hbm_src,
            "note": "algorithmic 320 B per cell-update; the path is FP64-ALU bound"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes + 8,
                "call": "teno_advance_host(nsteps=1) from pinned host memory, measured right "
                        "after the timed region", "clocks": e2e_clk},
        "gpu_launches": launches_per_step * args.steps,
        "decision_filter_off": filter_off,
        "nonphysical": nonphys,
        "clocks": clk,
        "cpu_baseline": cpu,
        "batched": batched,
        "adjoint": adjoint,
        "noh": noh,
        "teno12": teno12,
        "teno8": teno8,
        "quadrants_2d": quad2d,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.batched_only:
        import torch
        from paper_2109_14340_gb300 import _build
        _build.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        print(json.dumps(run_batched(args, dev, torch.cuda.current_stream(dev))), flush=True)
        return
    if args.adjoint_only or args.quadrants_2d_only:
        import torch
        from paper_2109_14340_gb300 import _build
        _build.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        run = run_adjoint if args.adjoint_only else run_2d_leg
        print(json.dumps(run(args, dev, torch.cuda.current_stream(dev))), flush=True)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
