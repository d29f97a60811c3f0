#!/usr/bin/env python
"""Benchmark: unknowns solved per second at relative residual 1e-8.

Workload (default ``layered_1024_m64``): the axisymmetric equation on a
1024 x 1024 grid (r x z), 64 right-hand sides (Gaussian point sources), kappa in
8 z-layers times an elliptical x5 inclusion, q proportional to kappa.  One
"step" is one complete solve of all 64 right-hand sides to an FP64 true
relative residual of 1e-8 with the chosen form (FP32 PCG inside FP64
iterative refinement), inputs resident in HBM.  The plain FP64 PCG on the
same GPU is timed beside it.  Under torchrun each rank solves its own replica
(weak scaling, no data-path collective).

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "unknowns solved/s at rel. residual 1e-8"
UNIT = "unknowns/s"
TOL = 1e-8

# Algorithmic bytes per grid unknown of one launch (FP32 working precision),
# M = right-hand sides sharing the coefficient tables.
#   stencil (p = z + beta p, q = A p): read z, p_old; write p, q  -> 16 B, + CR, CZ, W (12 B / M)
#   FFT forward transform (x += a p, r -= a q, rhat = S r): read x, p, r, q; write x, r, rhat -> 28 B
#   update pass (x += a p, r -= a q) ahead of the tensor-core transform: read x, p, r, q; write x, r
#     and r split into BF16 halves (the transform's operand) -> 28 B
#   tensor-core forward transform (rhat = S r): read split r, write rhat -> 8 B
#   mode solves: read rhat, write yhat -> 8 B, + IP (4 B / M)
#   FFT inverse transform (z = S yhat, (r, z)): read yhat, r; write z -> 12 B
#   tensor-core inverse transform (z = S yhat; (r, z) comes from the mode solves): read split
#     yhat, write z -> 8 B
#   true residual (r = phi - A x, x and phi as FP32 pairs): read x, phi (16 B); write r (4 B) -> 20 B,
#     + coefficients and their low parts 24 B / M
ALG_BYTES = {"stencil": (16.0, 12.0), "dst_forward": (28.0, 0.0), "mode_solve": (8.0, 4.0),
             "dst_inverse": (12.0, 0.0), "outer_residual": (20.0, 24.0), "pcg_update": (28.0, 0.0)}
ALG_BYTES_TC = dict(ALG_BYTES, dst_forward=(8.0, 0.0), dst_inverse=(8.0, 0.0))
# Fused tensor-core iteration of the mixed PCG (nr <= 4096): the inverse
# transform's epilogue forms p = z + beta p and x += alpha p_old, so
#   stencil (q = A p): read p, write q -> 8 B, + CR, CZ, W (12 B / M)
#   update pass (r -= a q): read r, q; write r and its split -> 16 B
#   inverse transform: read split yhat, p_old, x; write p_new, x -> 20 B
ALG_BYTES_FUSED = dict(ALG_BYTES_TC, stencil=(8.0, 12.0), pcg_update=(16.0, 0.0), dst_inverse=(20.0, 0.0))
# Tensor-core transform: multiply-adds per row = products x n^2 / 2 (even / odd
# halves), 2 flops each.
TC_CLASSES = ("dst_forward", "dst_inverse")


# Source of each kernel class whose change invalidates its ncu traffic figure:
# (file, __global__ function or None for the whole file), plus the shared
# device helpers.
KERNEL_SOURCES = {"stencil": [("ax_stencil.cu", "stencil_kernel")],
                  "dst_forward": [("ax_dst_impl.cuh", None)],
                  "dst_inverse": [("ax_dst_impl.cuh", None)],
                  "dst_forward_tc": [("ax_dst_gemm.cu", None)],
                  "dst_inverse_tc": [("ax_dst_gemm.cu", None)],
                  "mode_solve": [("ax_tridiag.cu", "tridiag_reg_kernel")],
                  "mode_solve_scaled": [("ax_tridiag.cu", "tridiag_reg2_kernel")],
                  "mode_solve_reuse": [("ax_tridiag.cu", "tridiag_reg3_kernel")],
                  "mode_solve_pipe": [("ax_tridiag.cu", "tridiag_pipe_kernel")],
                  "mode_solve_modemajor": [("ax_tridiag.cu", "tridiag_tr_kernel")],
                  "mode_solve_tall": [("ax_tridiag.cu", "tridiag_kernel")],
                  "outer_residual": [("ax_stencil.cu", "residual_df_kernel")],
                  "pcg_update": [("ax_solver.cu", "pcg_update")]}
TRAFFIC_TABLE = os.path.join(ROOT, "profiles", "traffic_per_unknown.json")


def _function_text(src: str, name: str) -> str:
    """The text of the __global__ function `name`: from its declaration line
    to the first line that closes it at column 0."""
    lines = src.splitlines()
    for i, line in enumerate(lines):
        if "__global__" in line and (name + "(") in " ".join(lines[i:i + 2]):
            for j in range(i, len(lines)):
                if lines[j] == "}":
                    return "\n".join(lines[i:j + 1])
    return src


def _code_only(text: str) -> str:
    """`text` without its comments and blank lines: what decides the compiled
    kernel (a comment edit keeps a traffic figure valid)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def source_hash(kernel: str, read=None) -> str:
    """Hash of the code (comments dropped) of the sources of kernel class
    `kernel`; read(name) returns a file's text (default: the csrc file)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1002_3094_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(csrc, name)) as fh:
                return fh.read()
    for f, fn in KERNEL_SOURCES.get(kernel, []) + [("ax_common.cuh", None)]:
        text = read(f)
        h.update(_code_only(text if fn is None else _function_text(text, fn)).encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, units_per_launch: float):
    """DRAM bytes (read + write) per launch of `kernel`, scaled from the ncu
    capture recorded in profiles/traffic_per_unknown.json (bytes per grid
    unknown of the captured launch), or None when no capture matches the
    current source of the kernel."""
    try:
        with open(TRAFFIC_TABLE) as fh:
            entries = json.load(fh)["entries"]
    except (OSError, ValueError, KeyError):
        return None
    want = source_hash(kernel)
    for e in entries:
        if e.get("class") == kernel and e.get("source_sha") == want:
            return float(e["dram_bytes_per_unknown"]) * units_per_launch
    return None


MODE_CLASSES = {1: "mode_solve", 9: "mode_solve_scaled", 12: "mode_solve_scaled", 10: "mode_solve_reuse",
                11: "mode_solve_reuse", 14: "mode_solve_modemajor"}


def kernel_class(top: str, tc_path: bool, mode_eff: int) -> str:
    """The KERNEL_SOURCES class of profiled kernel group `top` as the solve
    ran it (transform form, mode-solve kernel id)."""
    if top in TC_CLASSES and tc_path:
        return top + "_tc"
    if top == "mode_solve":
        if mode_eff == 0:
            return "mode_solve_tall"
        return MODE_CLASSES.get(mode_eff, "mode_solve_pipe")
    return top


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="layered_1024_m64")
    ap.add_argument("--method", default="pcg_mixed", choices=["pcg_mixed", "cheb_mixed", "pcg64", "cheb64"])
    ap.add_argument("--plain-steps", type=int, default=1, help="timed solves of the plain FP64 comparator")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rhs", type=int, default=0, help="override the number of right-hand sides (profiling)")
    ap.add_argument("--train", type=int, default=4096, help="guess_256: training seeds")
    ap.add_argument("--eval", type=int, default=512, help="guess_256: held-out seeds")
    ap.add_argument("--epochs", type=int, default=8, help="guess_256: training epochs")
    ap.add_argument("--batch", type=int, default=16, help="guess_256: batch size")
    ap.add_argument("--lr", type=float, default=1e-3, help="guess_256: Adam learning rate")
    ap.add_argument("--save", default="", help="guess_256: write the trained weights here")
    ap.add_argument("--h1", type=float, default=10.0, help="guess_256: weight of the loss's lattice-edge term")
    ap.add_argument("--no-pre", action="store_true", help="guess_256: raw f / s feature instead of B^-1 (r f)")
    ap.add_argument("--train-media", type=int, default=24,
                    help="large_4096_m16_guess: training media (16 right-hand sides each)")
    ap.add_argument("--eval-media", type=int, default=2, help="large_4096_m16_guess: held-out media")
    ap.add_argument("--bc-z", type=int, default=0, choices=[0, 1],
                    help="z boundary: 0 = u = 0 (sine transform), 1 = the paper's zero flux (cosine pair)")
    ap.add_argument("--dst-tensor", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="FP32 path transform along z: -1 the library's choice, 0 FFT, 1 tensor-core GEMM "
                         "by S_hi + S_lo, 2 tensor-core GEMM by S_hi (option dst_tensor)")
    ap.add_argument("--harmonics", type=int, default=2000, help="laguerre_chain: number of harmonics")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default transform and mode-solve kernel (no ax_autotune)")
    ap.add_argument("--mode-kernel", type=int, default=0,
                    help="FP32 mode-solve kernel variant (option mode_kernel; 0 the library's choice)")
    ap.add_argument("--option", action="append", default=[], metavar="NAME=VALUE",
                    help="ax_set_option on the operator before the run (repeatable)")
    ap.add_argument("--replace-delta", type=float, default=0.0,
                    help="mixed PCG: residual reduction between FP64 residual replacements (0: the library's)")
    return ap.parse_args()


def workload(name: str, instance: int = 0, rhs: int = 0):
    from workloads import layered_inclusion_medium, large_medium, bumps_medium
    if name == "layered_1024_m64":
        return 1024, 1024, layered_inclusion_medium(rhs or 64, 1024, instance=instance)
    if name == "large_4096_m16":
        return 4096, 4096, large_medium(rhs or 16, 4096, instance=instance)
    if name == "bumps_64":
        return 64, 64, bumps_medium(instance)
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, one right-hand side per process
# ---------------------------------------------------------------------------
# Above this many unknowns per solve the oracle is timed on its parts and
# extrapolated (a full 4096^2 solve takes many minutes on one core).
ORACLE_FULL_MAX = 1 << 21
# FP64 PCG iteration counts (max over right-hand sides) of the large workloads,
# as measured by the library's FP64 PCG (the oracle's algorithm, same count to
# +-1), for the extrapolation when no GPU count is at hand (reference arm).
ORACLE_ITERS_HINT = {"large_4096_m16": 87}


def _oracle_one(args):
    """Oracle PCG solves by one worker: right-hand sides (or, for single-source
    workloads, seeded instances) j, j + stride, ... until min_s seconds have
    passed (at least one).  Large grids: one operator set-up, one A y and one
    B^-1 v are timed, and the solve time is extrapolated to `iters_hint`
    iterations (each one A p and one B^-1 r, plus the initial pair)."""
    name, j, stride, min_s, bc_z, iters_hint = args
    import numpy as np
    import oracle as O
    nr, nz, med = workload(name)
    single = med.n_rhs == 1
    if nr * nz > ORACLE_FULL_MAX:
        g = O.Grid(nr, nz, bc_z=bc_z)
        kr, kz, q, f = O.sample_medium(med, g, rhs_index=[j % med.n_rhs])
        t0 = time.perf_counter()
        op = O.Operator(kr, kz, q, g)
        t1 = time.perf_counter()
        y = op.apply_A(f[0])
        t2 = time.perf_counter()
        z = op.apply_Binv(y)
        t3 = time.perf_counter()
        assert np.isfinite(z).all()
        est = (t1 - t0) + (iters_hint + 1) * ((t2 - t1) + (t3 - t2))
        return {"unknowns": nr * nz, "iters": [iters_hint], "solves": 1, "est_s": est,
                "parts_s": [t1 - t0, t2 - t1, t3 - t2]}
    t0 = time.perf_counter()
    unknowns, iters, solves, k = 0, [], 0, j
    while True:
        if single:
            nr, nz, med = workload(name, instance=k)
        g = O.Grid(nr, nz, bc_z=bc_z)
        kr, kz, q, f = O.sample_medium(med, g, rhs_index=[0 if single else k % med.n_rhs])
        op = O.Operator(kr, kz, q, g)
        _, info = op.solve(f[0], TOL)
        unknowns += nr * nz
        iters.append(info.iters)
        solves += 1
        k += stride
        if time.perf_counter() - t0 >= min_s:
            break
    return {"unknowns": unknowns, "iters": iters, "solves": solves}


def oracle_check(name: str, bc_z: int, idx, u_gpu):
    """The FP64 oracle's view of sampled GPU answers (right-hand sides idx,
    solutions u_gpu [len(idx)][nr][nz]): the true relative residual
    ||phi - A u|| / ||phi|| with the oracle's assembled operator, and, where
    the oracle can solve the grid (nr nz <= ORACLE_FULL_MAX), the relative
    difference to the oracle's own PCG solution at 1e-10 (at most 400
    iterations: the FP64 true residual of a 1024^2 grid stops falling between
    1e-11 and 1e-12)."""
    import numpy as np
    import oracle as O
    nr, nz, med = workload(name)
    g = O.Grid(nr, nz, bc_z=bc_z)
    kr, kz, q, f = O.sample_medium(med, g, rhs_index=list(idx))
    op = O.Operator(kr, kz, q, g)
    res, diff = [], []
    for j in range(len(idx)):
        phi = op.phi(f[j])
        res.append(float(np.linalg.norm(phi - op.apply_A(u_gpu[j])) / np.linalg.norm(phi)))
        if nr * nz <= ORACLE_FULL_MAX:
            uo, _ = op.solve(f[j], 1e-10, max_iter=400)
            diff.append(float(np.linalg.norm(u_gpu[j] - uo) / np.linalg.norm(uo)))
    out = {"rhs": [int(i) for i in idx], "true_rel_residual": res, "max_true_rel_residual": max(res)}
    if diff:
        out["rel_diff_to_oracle_solution"] = diff
    return out


def oracle_pool(cores: int):
    import multiprocessing as mp
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    for k in env_keys:
        os.environ[k] = "1"  # inherited by the spawned workers before they import numpy
    return mp.get_context("spawn").Pool(cores)


def cpu_baseline(name: str, cores: int, pool=None, bc_z: int = 0, iters_hint: int = 0):
    """Solves `cores` right-hand sides of the workload, one per core, with the
    oracle's PCG; returns unknowns solved per second of wall time."""
    own = pool is None
    pool = pool or oracle_pool(cores)
    try:
        t0 = time.perf_counter()
        res = pool.map(_oracle_one, [(name, j, cores, 2.0, bc_z, iters_hint) for j in range(cores)])
        wall = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    unknowns = sum(r["unknowns"] for r in res)
    solves = sum(r["solves"] for r in res)
    its = [i for r in res for i in r["iters"]]
    if "est_s" in res[0]:
        est = max(r["est_s"] for r in res)
        parts = res[0]["parts_s"]
        return {"value": unknowns / est, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"extrapolated: {cores} right-hand sides of {name}, one per host core; each core timed "
                          f"its operator set-up ({parts[0]:.1f} s), one A y ({parts[1]:.2f} s) and one B^-1 v "
                          f"({parts[2]:.1f} s) and the solve was taken as set-up + {iters_hint + 1} x (A + B^-1), "
                          f"{iters_hint} being the GPU FP64 PCG iteration count; sample wall {wall:.1f} s",
                "wall_s": est, "unknowns": unknowns, "extrapolated": True}
    return {"value": unknowns / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{solves} solves of {name} ({solves // cores}+ per host core, one process each), FP64 "
                      f"oracle PCG to {TOL:g} (set-up included), wall {wall:.1f} s, iterations "
                      f"{min(its)}..{max(its)}",
            "wall_s": wall, "unknowns": unknowns}


def _reference_laguerre(args):
    """Reference arm of laguerre_chain: the oracle's chain (direct sums, FP64
    PCG to the same tolerance, warm start from the previous harmonic) over the
    first 12 harmonics of the workload on one host core (the chain is
    sequential, so a window has to start at harmonic 0); the operator set-up
    runs once, outside the timed steps, as on the GPU arm.  value = harmonics
    nr nz / wall time; per_iteration = unknowns x PCG iterations / wall time,
    which does not depend on how many iterations the harmonics of the window
    need (the first ones have right-hand sides ~1e-10 of the largest)."""
    import numpy as np
    import oracle as O
    from oracle import laguerre as OL
    from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs
    from workloads.laguerre import ALPHA, H_LAG, fault_medium, wavelet_coefficients
    nr = nz = 1024
    lr = lz = 2048.0
    k = 12
    med = fault_medium(lr, lz)
    kr, kz, q = sample_operator_inputs(med, nr, nz, lr, lz, bc_z=1)
    src = sample_rhs(med, nr, nz, lr, lz, bc_z=1)[0]
    fm = wavelet_coefficients(args.harmonics, ALPHA, H_LAG)
    fm = fm / np.abs(fm).max()
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz, lr, lz, bc_z=1))
    times, iters = [], []

    def solve(rhs, prev):
        y, info = ora.solve(rhs, TOL, y0=prev)
        its.append(info.iters)
        return y

    for step in range(args.warmup + args.steps):
        its = []
        t0 = time.perf_counter()
        OL.chain(solve, 4.0 * q, src, fm[:k], ALPHA)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
            iters.append(its)
    total = sum(times)
    value = k * nr * nz * args.steps / total
    per_it = sum(sum(i) for i in iters) * nr * nz / total
    sample = (f"harmonics 0..{k - 1} of laguerre_chain ({nr}^2), FP64 oracle PCG to {TOL:g}, warm start, "
              f"operator set-up outside the timed steps; iterations per harmonic {iters[-1]}")
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference", "config": {"workload": "laguerre_chain", "harmonics_per_step": k,
                                                      "nr": nr, "nz": nz, "tol": TOL, "bc_z": 1},
                      "iters_per_harmonic": iters[-1],
                      "per_iteration": {"value": per_it, "unit": "unknown-iterations/s"},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"each step: {sample}"},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def arm_config(args, nr: int, nz: int, m: int, world: int) -> dict:
    """The config of a single-operator workload's line (the same on both arms)."""
    # working set of the mixed solve: f and u (FP64), the double-float x and
    # phi, six FP32 vectors and the split operand, about 64 B per unknown
    unknowns = nr * nz * m
    ws_mb = (unknowns * 64) >> 20
    l2_note = ("inputs larger than L2 (f is %d MB, solver working set ~%d MB)" % ((unknowns * 8) >> 20, ws_mb)
               if ws_mb > 129 else
               "working set ~%d MB fits in L2, no flush between steps (a solve this small is launch-bound)"
               % max(ws_mb, 1))
    return {"workload": args.workload, "nr": nr, "nz": nz, "rhs": m, "tol": TOL, "bc_z": args.bc_z,
            "method": args.method, "parallelism": f"replicas x{world}", "l2": l2_note, "options": args.option}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "laguerre_chain":
        _reference_laguerre(args)
        return
    cores = os.cpu_count() or 1
    pool = oracle_pool(cores)
    try:
        # warm-up steps: a 64 x 64 solve per core (pool start-up, imports)
        for _ in range(args.warmup):
            pool.map(_oracle_one, [("bumps_64", 0, 1, 0.0, 0, 0)] * cores)
        times, units = [], 0
        for _ in range(args.steps):
            r = cpu_baseline(args.workload, cores, pool, args.bc_z, ORACLE_ITERS_HINT.get(args.workload, 0))
            times.append(r["wall_s"])
            units += r["unknowns"]
        total = sum(times)
        value = units / total
        # the GPU arm's config of this workload (each step here solves a
        # bounded sample of it: cpu_baseline.sample says which)
        if args.workload in ("layered_1024_m64", "large_4096_m16", "bumps_64"):
            nr, nz, med = workload(args.workload, rhs=args.rhs)
            config = arm_config(args, nr, nz, med.n_rhs, args.gpus)
        else:
            config = {"workload": args.workload, "tol": TOL, "bc_z": args.bc_z}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": config,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"each step: {r['sample']}"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
    finally:
        pool.close()
        pool.join()


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_batched(args):
    """Workload batched_256: 256 independent instances, nr and nz drawn from
    {127, 255, 511, 1023, 2047}, one right-hand side each, solved together by
    the batched entry point (instances of one grid shape share each launch;
    shapes run concurrently).  value = all unknowns / wall time of one batched
    solve; latency = per-instance time to its group's completion."""
    import numpy as np
    import torch
    import paper_1002_3094_gb300 as P
    from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs
    from workloads import batched_instances
    count = args.rhs or 256
    dev = torch.device("cuda", 0)
    P.build()
    P.load_library()
    ops, fs, us, unknowns, nr_nz = [], [], [], 0, []
    for nr, nz, med in batched_instances(count):
        nr_nz.append((nr, nz))
        kr, kz, q = sample_operator_inputs(med, nr, nz, bc_z=args.bc_z)
        ops.append(P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz, bc_z=args.bc_z))
        fs.append(torch.from_numpy(sample_rhs(med, nr, nz, bc_z=args.bc_z)[0]).to(dev))
        us.append(torch.zeros((nr, nz), dtype=torch.float64, device=dev))
        unknowns += nr * nz
    for op in ops:
        if args.dst_tensor >= 0:
            P.ax_set_option(op, "dst_tensor", args.dst_tensor)
        if args.replace_delta > 0:
            P.ax_set_option(op, "replace_delta", args.replace_delta)
        for kv in args.option:  # every instance (a shape group takes its first member's solver options)
            name, value = kv.split("=", 1)
            P.ax_set_option(op, name, float(value))
    batch = P.ax_batch_create(ops)
    method = P.METHODS[args.method]
    stream = torch.cuda.current_stream()
    tune_s = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        P.ax_batch_autotune(batch, 5, stream=stream)
        tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        st, info = P.ax_batch_solve(batch, fs, us, TOL, 20000, method, stream=stream, raise_on_error=False)
        if st != P.AX_OK:
            bad = [(j, nr_nz[j], i) for j, i in enumerate(info) if i["status"] != P.AX_OK]
            print(json.dumps({"error": P.ax_status_string(st), "failed": bad[:10], "n_failed": len(bad)}))
            for u_ in us:
                u_.zero_()
            st2, info2 = P.ax_batch_solve(batch, fs, us, TOL, 20000, method, P.AX_FLAG_SERIAL_GROUPS, stream=stream,
                                          raise_on_error=False)
            bad2 = [(j, nr_nz[j], i) for j, i in enumerate(info2) if i["status"] != P.AX_OK]
            print(json.dumps({"serial_groups_status": P.ax_status_string(st2), "n_failed": len(bad2),
                              "failed": bad2[:5]}))
            for j, (nr, nz), _ in bad[:3]:  # the same instance alone
                u1 = torch.zeros_like(us[j])
                st1, i1 = P.ax_solve(ops[j], fs[j], u1, 1, TOL, 20000, method, raise_on_error=False)
                st2, i2 = P.ax_solve(ops[j], fs[j], u1, 1, TOL, 20000, P.AX_PCG_FP64, raise_on_error=False)
                print(json.dumps({"instance": j, "shape": [nr, nz], "alone": i1[0], "alone_fp64": i2[0]}))
            return
    torch.cuda.synchronize()
    launches0 = P.ax_kernel_launches()
    clocks = ClockSampler(0)
    lats = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        st, info = P.ax_batch_solve(batch, fs, us, TOL, 20000, method, stream=stream)
        lat, groups = P.ax_batch_latency(batch, len(ops))
        lats += lat
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    value = unknowns * args.steps / (ms / 1e3)
    launches = P.ax_kernel_launches() - launches0
    # the plain FP64 PCG on the same batch (the comparator of the metric)
    plain = None
    if args.plain_steps > 0 and method != P.AX_PCG_FP64:
        u64 = [torch.zeros_like(u_) for u_ in us]
        P.ax_batch_solve(batch, fs, u64, TOL, 20000, P.AX_PCG_FP64, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.plain_steps):
            _, pinfo = P.ax_batch_solve(batch, fs, u64, TOL, 20000, P.AX_PCG_FP64, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / args.plain_steps
        plat, _ = P.ax_batch_latency(batch, len(ops))
        diff = max(float(torch.linalg.vector_norm(a - b_) / torch.linalg.vector_norm(b_)) for a, b_ in zip(us, u64))
        plain = {"value": unknowns / (pms / 1e3), "ms_per_step": pms,
                 "iters_max": max(i["iters"] for i in pinfo),
                 "latency_ms": {"p50": float(np.percentile(plat, 50)), "p99": float(np.percentile(plat, 99))},
                 "max_rel_diff_to_chosen": diff}
        del u64
    tuned = [P.ax_batch_config(batch, g) for g in range(groups)]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner / f64 refinement" if "mixed" in args.method else "f64",
            "data": "synthetic",
            "config": {"workload": "batched_256", "instances": len(ops), "unknowns": unknowns, "groups": groups,
                       "bc_z": args.bc_z,
                       "method": args.method, "tol": TOL, "autotuned": not args.no_autotune,
                       "options": list(args.option)},
            "latency_ms": {"p50": float(np.percentile(lats, 50)), "p99": float(np.percentile(lats, 99)),
                           "max": float(max(lats)), "min": float(min(lats)),
                           "meaning": "per instance: batch start to the graph replay in which it converged"},
            "iters": {"max": max(i["iters"] for i in info), "min": min(i["iters"] for i in info),
                      "mean": float(np.mean([i["iters"] for i in info])),
                      "p90": float(np.percentile([i["iters"] for i in info], 90)),
                      "slowest": sorted(([i["iters"], j, list(nr_nz[j])] for j, i in enumerate(info)),
                                        reverse=True)[:3]},
            "max_rel_res": max(i["rel_res"] for i in info),
            "plain_fp64": plain, "vs_plain_fp64": (value / plain["value"]) if plain else None,
            "autotune_s": tune_s, "tuned_groups": tuned,
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line))
    P.ax_batch_destroy(batch)
    for op in ops:
        P.ax_destroy_operator(op)


def run_laguerre(args):
    """Workload laguerre_chain (Section 4.1): the harmonics Q_0 .. Q_{n-1} of the
    Laguerre expansion in time (n = --harmonics, default 2000, alpha = 5,
    h = 300 as in the paper) on a 1024 x 1024 grid of a 2048 m x 2048 m layered
    medium with a fault, zero-flux z boundary, point source at the origin.  One
    step = the whole sequential chain; value = n nr nz / time.  The source
    coefficients are scaled by 1 / max |f_m| (the problem is linear)."""
    import numpy as np
    import torch
    import paper_1002_3094_gb300 as P
    from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs
    from paper_1002_3094_gb300.laguerre import solve_chain
    from workloads.laguerre import ALPHA, H_LAG, fault_medium, wavelet_coefficients
    nr = nz = 1024
    lr = lz = 2048.0
    n = args.harmonics
    dev = torch.device("cuda", 0)
    P.build()
    P.load_library()
    med = fault_medium(lr, lz)
    kr, kz, q = sample_operator_inputs(med, nr, nz, lr, lz, bc_z=1)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz, lr, lz, bc_z=1)
    if args.replace_delta > 0:
        P.ax_set_option(op, "replace_delta", args.replace_delta)
    src = torch.from_numpy(sample_rhs(med, nr, nz, lr, lz, bc_z=1)[0]).to(dev)
    c2 = torch.from_numpy(4.0 * q).to(dev)
    fm = wavelet_coefficients(n, ALPHA, H_LAG)
    fm = fm / np.abs(fm).max()
    method = P.METHODS[args.method]
    stream = torch.cuda.current_stream()
    qf = torch.zeros((1, nr, nz), dtype=torch.float64, device=dev)
    work = torch.zeros((3, nr, nz), dtype=torch.float64, device=dev)

    def chain():
        return solve_chain(op, c2, src, fm, ALPHA, TOL, qf, work, method=method, stream=stream)

    for _ in range(args.warmup):
        chain()
    torch.cuda.synchronize()
    launches0 = P.ax_kernel_launches()
    clocks = ClockSampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        infos = chain()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    iters = [i["iters"] for i in infos]
    line = {"metric": METRIC, "value": n * nr * nz * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 refinement" if "mixed" in args.method else "f64", "data": "synthetic",
            "config": {"workload": "laguerre_chain", "nr": nr, "nz": nz, "lr_m": lr, "lz_m": lz, "harmonics": n,
                       "alpha": ALPHA, "h": H_LAG, "bc_z": 1, "method": args.method, "tol": TOL,
                       "warm_start": "previous harmonic (gated)"},
            "ms_per_harmonic": ms / args.steps / n,
            "iters": {"mean": float(np.mean(iters)), "max": max(iters), "min": min(iters),
                      "preconditioner_applications": int(sum(iters)), "first_12": iters[:12]},
            "per_iteration": {"value": float(sum(iters)) * nr * nz * args.steps / (ms / 1e3),
                              "unit": "unknown-iterations/s"},
            "max_rel_res": max(i["rel_res"] for i in infos),
            "gpu_launches": P.ax_kernel_launches() - launches0, "clocks": clk}
    print(json.dumps(line))
    P.ax_destroy_operator(op)


def run_guess(args):
    """Workload guess_256 (random-field media on 256 x 256): solve
    `--train` seeds with the batched solver, train the guess network on the
    (features, u / s) pairs on the GPU, then solve `--eval` held-out seeds from
    zero and from the network's guess (inference time included, residual gate
    on) at 1e-8."""
    import numpy as np
    import torch
    import paper_1002_3094_gb300 as P
    from paper_1002_3094_gb300 import guess as GS
    from workloads import grf_spec
    dev = torch.device("cuda", 0)
    P.build()
    P.load_library()
    n = hw = 256
    t0 = time.perf_counter()
    pre = not args.no_pre
    train = GS.make_dataset([grf_spec(i, "train") for i in range(args.train)], n, n, hw, TOL, dev, pre=pre)
    t_data = time.perf_counter() - t0
    GS.release(train)
    net = P.ax_guessnet_create(hw, None, batch_capacity=args.batch, seed=1)
    P.ax_guessnet_set_loss(net, args.h1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = GS.train(net, train, args.epochs, args.batch, args.lr, log=lambda m: print(m, file=sys.stderr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    ev = GS.make_dataset([grf_spec(i, "eval") for i in range(args.eval)], n, n, hw, TOL, dev,
                         target_scale=train["tscale"], pre=pre)
    rows = GS.evaluate(net, ev, hw, n, n, TOL)
    GS.release(ev)
    # inference time alone (batch 1), CUDA events
    x = torch.zeros((1, 3, hw, hw), dtype=torch.float32, device=dev)
    y = torch.zeros((1, hw, hw), dtype=torch.float32, device=dev)
    for _ in range(3):
        P.ax_guessnet_forward(net, x, y, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        P.ax_guessnet_forward(net, x, y, 1)
    e1.record()
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / 10
    gflop = 2.0 * sum(9 * a * b for a, b in [(3, 24), (24, 24), (48, 24), (24, 24)]) * hw * hw / 1e9
    gflop += 2.0 * sum(9 * a * b for a, b in [(24, 48), (48, 48), (96, 48), (48, 48)]) * (hw // 2) ** 2 / 1e9
    gflop += 2.0 * sum(9 * a * b for a, b in [(48, 96), (96, 96), (192, 96), (96, 96)]) * (hw // 4) ** 2 / 1e9
    gflop += 2.0 * sum(9 * a * b for a, b in [(96, 192), (192, 192)]) * (hw // 8) ** 2 / 1e9
    it0 = np.array([r["iters_zero"] for r in rows])
    itg = np.array([r["iters_guess"] for r in rows])
    line = {"metric": "PCG iterations and wall time at rel. residual 1e-8, from the learned guess vs from zero",
            "workload": "guess_256", "train_samples": args.train, "eval_samples": args.eval,
            "epochs": args.epochs, "batch": args.batch, "params": P.ax_guessnet_num_params(net),
            "h1_weight": args.h1, "feature": "B^-1 (r f) / s" if pre else "f / s",
            "data_s": t_data, "train_s": t_train, "train_samples_per_s": args.train * args.epochs / t_train,
            "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
            "iters_zero_mean": float(it0.mean()), "iters_guess_mean": float(itg.mean()),
            "iters_saved_frac": float(1 - itg.mean() / it0.mean()),
            "ms_zero_mean": float(np.mean([r["ms_zero"] for r in rows])),
            "ms_guess_mean": float(np.mean([r["ms_guess"] for r in rows])),
            "accepted_frac": float(np.mean([r["accepted"] for r in rows])),
            "energy_ratio_median": float(np.median([r["energy_ratio"] for r in rows])),
            "max_rel_res_guess": float(max(r["res_guess"] for r in rows)),
            "inference_ms": infer_ms, "inference_gflop": gflop, "inference_tflops": gflop / infer_ms}
    print(json.dumps(line))
    if args.save:
        P.ax_guessnet_save(net, args.save)
    P.ax_guessnet_destroy(net)


def run_guess_large(args):
    """Workload large_4096_m16_guess: mixed PCG at 4096^2 x 16 right-hand sides
    with the learned guess, the network at 512^2 with bilinear lift.  Solves
    `--train-media` media of the large layered kind (disjoint seed stream),
    trains the network on the GPU on (features with B^-1 (r f), cell averages
    of u / s), then solves `--eval-media` held-out media from zero and from
    the network's guess (features, inference and lift inside the timed
    region; residual gate on) to 1e-8."""
    import numpy as np
    import torch
    import paper_1002_3094_gb300 as P
    from paper_1002_3094_gb300 import guess as GS
    from workloads import large_spec
    dev = torch.device("cuda", 0)
    P.build()
    P.load_library()
    n, hw, m = 4096, 512, 16
    t0 = time.perf_counter()
    train = GS.make_dataset_large([large_spec(i, m, n, split="train") for i in range(args.train_media)], n, n, hw,
                                  TOL, dev)
    t_data = time.perf_counter() - t0
    net = P.ax_guessnet_create(hw, None, batch_capacity=max(args.batch, m), seed=1)
    P.ax_guessnet_set_loss(net, args.h1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = GS.train(net, train, args.epochs, args.batch, args.lr, log=lambda s_: print(s_, file=sys.stderr))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    n_train = int(train["x"].shape[0])
    tscale = train["tscale"]
    del train
    ev = GS.make_dataset_large([large_spec(i, m, n, split="eval") for i in range(args.eval_media)], n, n, hw, TOL,
                               dev, target_scale=tscale, keep_ops=True)
    rows = []
    for med in ev["media"]:
        op, f = med["op"], med["f"]
        u = torch.zeros_like(f)
        P.ax_solve(op, f, u, m, TOL, 20000, P.AX_PCG_MIXED)  # warm the graphs
        torch.cuda.synchronize()
        u.zero_()
        a0 = time.perf_counter()
        _, i0 = P.ax_solve(op, f, u, m, TOL, 20000, P.AX_PCG_MIXED)
        torch.cuda.synchronize()
        a1 = time.perf_counter()
        u0 = GS.guess_large(net, med, hw, n, n, tscale)
        _, ig = P.ax_solve(op, f, u0, m, TOL, 20000, P.AX_PCG_MIXED, P.AX_FLAG_USE_GUESS | P.AX_FLAG_CHECK_GUESS)
        torch.cuda.synchronize()
        a2 = time.perf_counter()
        g1 = GS.guess_large(net, med, hw, n, n, tscale)
        ratios = [GS.energy_ratio(op, f[j:j + 1], g1[j:j + 1]) for j in range(m)]
        eratios = [GS.energy_error_ratio(op, med["u"][j], g1[j]) for j in range(m)]
        rows.append({"iters_zero": [i["iters"] for i in i0], "iters_guess": [i["iters"] for i in ig],
                     "ms_zero": 1e3 * (a1 - a0), "ms_guess": 1e3 * (a2 - a1),
                     "accepted": [i["guess_accepted"] for i in ig], "energy_ratio": ratios,
                     "energy_error_ratio": eratios,
                     "max_rel_res_guess": max(i["rel_res"] for i in ig)})
        del u, u0, g1
    med0 = ev["media"][0]
    bounds = GS.lattice_bounds(med0["op"], med0["f"], med0["u"], hw)
    for med in ev["media"]:
        P.ax_destroy_operator(med["op"])
    it0 = np.array([x for r in rows for x in r["iters_zero"]])
    itg = np.array([x for r in rows for x in r["iters_guess"]])
    er = np.array([x for r in rows for x in r["energy_ratio"]])
    ee = np.array([x for r in rows for x in r["energy_error_ratio"]])
    line = {"metric": "PCG iterations and wall time at rel. residual 1e-8, from the learned guess vs from zero",
            "workload": "large_4096_m16_guess", "grid": [n, n], "rhs_per_solve": m, "network_lattice": hw,
            "lift": "bilinear", "method": "pcg_mixed", "train_media": args.train_media, "train_samples": n_train,
            "eval_media": args.eval_media, "eval_samples": int(it0.size), "epochs": args.epochs,
            "batch": args.batch, "h1_weight": args.h1, "feature": "B^-1 (r f) / s",
            "data_s": t_data, "train_s": t_train, "train_samples_per_s": n_train * args.epochs / t_train,
            "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
            "iters_zero_mean": float(it0.mean()), "iters_guess_mean": float(itg.mean()),
            "iters_zero_max": int(it0.max()), "iters_guess_max": int(itg.max()),
            "iters_saved_frac": float(1 - itg.mean() / it0.mean()),
            "ms_zero_per_solve": float(np.mean([r["ms_zero"] for r in rows])),
            "ms_guess_per_solve": float(np.mean([r["ms_guess"] for r in rows])),
            "accepted_frac": float(np.mean([a for r in rows for a in r["accepted"]])),
            "energy_ratio_median": float(np.median(er)), "energy_ratio_min": float(er.min()),
            "energy_error_ratio_median": float(np.median(ee)), "energy_error_ratio_min": float(ee.min()),
            "energy_ratio_meaning": "sqrt((r0, B^-1 r0) / (phi, B^-1 phi)) of the guess (the gate's test)",
            "energy_error_ratio_meaning": "||u0 - u||_A / ||u||_A against the converged solution",
            "max_rel_res_guess": max(r["max_rel_res_guess"] for r in rows),
            "lattice_bounds_median": {k: float(np.median(v)) for k, v in bounds.items()},
            "lattice_bounds_meaning": "energy-norm error ratio of the first held-out medium's 16 right-hand "
                                      "sides: lattice = lift of u's own 512^2 cell averages; one_step = a B^-1 (r f) "
                                      "with the A-optimal a; one_step_plus_lattice = that plus the lift of the cell "
                                      "averages of the remainder",
            "data": "synthetic"}
    print(json.dumps(line))
    P.ax_guessnet_destroy(net)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "guess_256":
        run_guess(args)
        return
    if args.workload == "large_4096_m16_guess":
        run_guess_large(args)
        return
    if args.workload == "laguerre_chain":
        run_laguerre(args)
        return
    if args.workload == "batched_256":
        run_batched(args)
        return
    # The oracle pool must start before the first CUDA call (spawned workers).
    from paper_1002_3094_gb300 import replicas as RP
    world, rank, local_rank = RP.rank_env()
    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = oracle_pool(cores)

    import numpy as np
    import torch
    import paper_1002_3094_gb300 as P
    from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    P.build()
    P.load_library()

    nr, nz, med = workload(args.workload, instance=RP.replica_instance(rank), rhs=args.rhs)
    m = med.n_rhs
    kr, kz, q = sample_operator_inputs(med, nr, nz, bc_z=args.bc_z)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz, bc_z=args.bc_z)
    if args.dst_tensor >= 0:
        P.ax_set_option(op, "dst_tensor", args.dst_tensor)
    if args.replace_delta > 0:
        P.ax_set_option(op, "replace_delta", args.replace_delta)
    if args.mode_kernel > 0:
        P.ax_set_option(op, "mode_kernel", args.mode_kernel)
    for kv in args.option:
        name, value = kv.split("=", 1)
        P.ax_set_option(op, name, float(value))
    tuned = None
    if not args.no_autotune and args.dst_tensor < 0 and args.mode_kernel == 0 and "mixed" in args.method:
        t0 = time.perf_counter()
        P.ax_autotune(op, m, 5)
        tuned = {"dst_tensor": int(P.ax_get_option(op, "dst_tensor")),
                 "mode_kernel": int(P.ax_get_option(op, "mode_kernel")), "autotune_s": time.perf_counter() - t0}
    mode_eff = int(P.ax_get_option(op, "mode_kernel_effective"))
    f_host = sample_rhs(med, nr, nz, bc_z=args.bc_z)
    f = torch.from_numpy(f_host).to(dev)
    u = torch.zeros_like(f)
    method = P.METHODS[args.method]
    stream = torch.cuda.current_stream()

    def solve(meth=method, ff=f, uu=u, flags=0):
        st, info = P.ax_solve(op, ff, uu, m, TOL, 20000, meth, flags, stream=stream)
        if st != P.AX_OK:
            raise RuntimeError(f"solve failed: {P.ax_status_string(st)} {info[:2]}")
        return info

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return RP.max_over_ranks(x, dist, dev)

    for _ in range(args.warmup):
        info = solve()
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    launches0 = P.ax_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        info = solve()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = P.ax_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    unknowns_step = nr * nz * m
    value = RP.aggregate_rate(unknowns_step * args.steps, ms_max / 1000.0, dist, dev)
    iters = [i["iters"] for i in info]
    outer = [i["outer"] for i in info]
    rel = max(i["rel_res"] for i in info)
    # two sampled answers for the oracle's check (first and last right-hand side)
    sample_idx = sorted({0, m - 1})
    u_sample = u[sample_idx].cpu().numpy()

    # ---- plain FP64 PCG on the same GPU (the comparator named by the metric) ----
    plain = None
    if args.plain_steps > 0 and method != P.AX_PCG_FP64:
        u64 = torch.zeros_like(f)
        solve(P.AX_PCG_FP64, f, u64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.plain_steps):
            pinfo = solve(P.AX_PCG_FP64, f, u64)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(e0.elapsed_time(e1)) / args.plain_steps
        pval = RP.aggregate_rate(unknowns_step, pms / 1000.0, dist, dev)
        diff = float(torch.linalg.vector_norm(u - u64) / torch.linalg.vector_norm(u64))
        plain = {"value": pval, "ms_per_step": pms, "iters_max": max(i["iters"] for i in pinfo),
                 "rel_diff_to_chosen": diff}
        del u64

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(f_host).pin_memory()
        uh = torch.zeros_like(fh).pin_memory()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.ax_solve(op, fh, uh, m, TOL, 20000, method, P.AX_FLAG_HOST_BUFFERS, stream=stream)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0)
        nbytes = f_host.nbytes
        e2e = {"value": RP.aggregate_rate(unknowns_step * args.steps, el, dist, dev), "unit": UNIT,
               "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}

    # ---- per-kernel times with CUDA events (one profiled solve) ----
    P.ax_set_option(op, "profile", 1)
    solve()
    torch.cuda.synchronize()
    prof = {k: P.ax_profile_read(op, k) for k in P.PROFILE_KINDS}
    P.ax_set_option(op, "profile", 0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # the transform runs inside a seconds-long solve: the sustained tensor figure
    tc_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    tc_path = prof.get("pcg_update", {}).get("launches", 0) > 0  # the tensor-core transform is in use
    products = 2 if args.dst_tensor == 2 else 3
    fused = tc_path and args.method == "pcg_mixed" and nr <= 4096
    alg = ALG_BYTES_FUSED if fused else (ALG_BYTES_TC if tc_path else ALG_BYTES)
    roof = None
    cand = {k: v for k, v in prof.items() if k in alg and v["launches"] > 0}
    if cand:
        top = max(cand, key=lambda k: cand[k]["ms"])
        p = cand[top]
        per_u, per_m = alg[top]
        units_per_launch = p["units"] / p["launches"]
        rhs_per_launch = units_per_launch / (nr * nz)
        bytes_per_launch = units_per_launch * per_u + (nr * nz) * per_m
        avg_s = p["ms"] / p["launches"] / 1000.0
        achieved = bytes_per_launch / avg_s / 1e9
        variant = kernel_class(top, tc_path, mode_eff)
        traffic = measured_traffic(variant, units_per_launch)
        roof = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_s * 1e3,
                "rhs_per_launch": rhs_per_launch}
        if tc_path and top in TC_CLASSES:
            # the GEMM's binding resource is whichever of the two limits is longer
            flops = (units_per_launch / nz) * products * float(nz) * nz
            if flops / (tc_peak * 1e12) > bytes_per_launch / (hbm_peak * 1e9):
                tflops = flops / avg_s / 1e12
                roof.update({"bound": "tensor", "achieved": tflops, "peak": tc_peak, "unit": "TFLOP/s",
                             "frac": tflops / tc_peak, "flops_per_launch": flops,
                             "peak_source": "measured" if "bf16_tflops_sustained" in peaks else "fallback"})
    kernel_ms = {k: {"ms": round(v["ms"], 3), "launches": int(v["launches"])} for k, v in prof.items()}

    cpu = None
    oracle_err = None
    if pool is not None:
        try:
            hint = plain["iters_max"] if plain else ORACLE_ITERS_HINT.get(args.workload, max(iters))
            cpu = cpu_baseline(args.workload, cores, pool, args.bc_z, hint)
            cpu.pop("wall_s", None)
            cpu.pop("unknowns", None)
            oracle_err = oracle_check(args.workload, args.bc_z, sample_idx, u_sample)
        finally:
            pool.close()
            pool.join()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 refinement" if "mixed" in args.method else "f64",
            "data": "synthetic",
            "config": arm_config(args, nr, nz, m, world),
            "iters": {"max": max(iters), "min": min(iters), "outer_max": max(outer)},
            "max_rel_res": rel,
            "plain_fp64": plain,
            "vs_plain_fp64": (value / plain["value"]) if plain else None,
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "roofline": roof, "autotuned": tuned,
            "kernel_ms_profiled_solve": kernel_ms, "cpu_baseline": cpu,
            "error_vs_oracle": oracle_err,
        }
        print(json.dumps(line))
    P.ax_destroy_operator(op)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
