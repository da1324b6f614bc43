"""Benchmark: time to CG relative residual 1e-2 on the precision workload.

Workload (one "step"): N = 65,536 standardised Gaussian points in d = 8, RBF
kernel (l = 1, a^2 = 1, sigma^2 = 0.05), B = [y, 16 Rademacher probes]
(17 right-hand sides), rank-100 pivoted-Cholesky preconditioner, then the
stable CG (Alg. 2) with FP16 tensor-core MVMs until every column's
relative residual, recomputed with an FP32 MVM, is <= 1e-2 less a margin for
that check's rounding; the residual is verified in FP64 over all rows
(untimed).  The step is the
whole hot path: operand preparation, preconditioner factor + core, every MVM,
Woodbury apply, LSE scalars, re-orthogonalisation, residual checks.

Printed: one JSON line (rank 0).  `value` = seconds per solve (lower is
better), device-timed with CUDA events, inputs resident in HBM, L2 flushed
between steps.  `e2e` = the same through the public API with pinned host
buffers (X, B uploaded and U downloaded inside the timed region).  The FP32
comparator (plain Alg. 1, SIMT FP32 MVM) and the BF16 arm are timed on the
same inputs and reported under "arms".

The headline MVM schedule is relaxed (--schedule relaxed, the default): the
FP16 MVM with the kernel tile and the inputs as hi + lo while the residual is
large, the single-rounded FP16 MVM once every column's recursive relative
residual is at most 30 x the tolerance (--schedule single: single-rounded
throughout, also timed as an arm).

--impl reference times the FP64 CPU oracle's own preconditioned CG (C, all
host cores) on the same inputs: each step is one full iteration (a
65,536-row matrix-free MVM, the Woodbury apply, the vector updates), and the
time to the residual is that per-iteration time times the iteration count of
the GPU's FP32 CG (flagged as extrapolated).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time_to_cg_relresid_1e-2"
UNIT = "s"
TOL = 1e-2
MAX_ITER = 1000
FP32_ITERS_NOTE = "iterations of the FP32 stable CG on this workload"
# Margin under the tolerance for the solver's stopping test.  The FP32 check MVM
# that recomputes r = K x - b near the solution errs by about u_32 kappa / sqrt(n)
# in units of ||b||: u_32 = 2^-24, kappa = || |K| |x| || / ||b|| the cancellation
# factor (1.5e4 on this workload), n = 65,536 independently rounded terms per
# row; that is 3.4e-6 (3.8e-6 measured against the full FP64 residual), and the
# margin 1e-4 = 1 % of the tolerance is thirty times it.
STOP_MARGIN = 0.01
# Relaxed MVM schedule of the headline solve: the FP16 MVM with the kernel tile
# and the inputs as hi + lo while any column's recursive relative residual is
# above RELAX_RESID, the single-rounded FP16 MVM after that.  The rounding of an
# MVM moves the true residual away from the recursive one in proportion to the
# residual at that step (the relaxation argument for inexact Krylov methods),
# so the accurate MVM is needed while the residual is large; 30 x the tolerance
# is where the iteration count stops growing on this workload (switch points
# 0.8 / 0.45 / 0.3 / 0.03: 198 / 182 / 162 / 159 iterations).
RELAX_RESID = 30.0 * TOL
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one kmvm_tp_kernel launch,
# keyed by the launch it was captured on (kernel, precision, N, R, flags); the
# roofline reports it only for that exact launch and null otherwise.
KMVM_TRAFFIC_BYTES = {("rbf", "fp16", 65536, 17, 0): 12.793088e6 + 12.288256e6,
                      ("rbf", "fp16", 65536, 17, 0x8000 | 0x200): 16.880896e6 + 11.435264e6}   # PSPLIT | XSPLIT


def _peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int = 0):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if "Active" in r[4 + i]
                          and "Not" not in r[4 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def solve_config(N: int, R: int, kernel: str, world: int) -> dict:
    """The `config` of the solve workload, shared by both arms."""
    return {"workload": f"precision: N={N} d=8 {kernel} l=1 a2=1 sigma2=0.05, 1+16 RHS (y + Rademacher), "
                        "rank-100 pivoted Cholesky, stable CG (Alg. 2) to rel. resid 1e-2 with FP32 residual checks",
            "global_batch": R, "seq_len": N, "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "flushed between steps (256 MB write)"}


def max_over_ranks(x: float, device=None) -> float:
    """The largest x over all ranks of the initialised process group (x itself
    when there is none).  Replicas are timed by their slowest member."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------

def _fp64_cpu_solver(w, kernel_name):
    """Inputs of the oracle's FP64 CG on the host: X, B (N x R), hyperparameters
    and the FP64 rank-k pivoted-Cholesky factor (Sec. 4.2), with the time the
    factor took."""
    import oracle as O
    B = w.rhs().T.astype(np.float64)
    hyp = O.Hyp(kernel_name, w.lengthscale, w.outputscale, w.noise)
    t0 = time.perf_counter()
    L, _ = O.pivoted_cholesky(w.X, hyp, w.rank)
    return B, hyp, L, time.perf_counter() - t0


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    from oracle import cfp64 as C
    from paper_2207_06856_gb300 import workloads
    w = workloads.precision(kernel={"rbf": workloads.RBF, "matern32": workloads.MATERN32}[args.kernel])
    B, hyp, L, t_pc = _fp64_cpu_solver(w, args.kernel)
    C.build()
    rows = np.arange(256)
    for _ in range(args.warmup):
        C.kmvm(w.X, B, hyp, rows=rows)   # threads up, caches warm
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, it, _, _ = C.pcg(w.X, B, hyp, L=L, tol=TOL, max_iter=1)   # set-up + one iteration
        ts.append(time.perf_counter() - t0)
    t_iter = float(np.mean(ts))
    value = t_pc + t_iter * args.ref_iters
    cores = C.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_iter, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": solve_config(w.N, B.shape[1], args.kernel, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"FP64 preconditioned CG (Alg. 1, C + OpenMP, {cores} threads) on the full "
                                   f"workload: {args.steps} timed iterations of {t_iter:.2f} s (each a "
                                   f"{w.N}-row matrix-free MVM with {B.shape[1]} right-hand sides, Woodbury "
                                   f"apply, updates), + the rank-{w.rank} FP64 pivoted Cholesky ({t_pc:.2f} s); "
                                   f"extrapolated to {args.ref_iters} iterations ({FP32_ITERS_NOTE})",
                         "extrapolated": True},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    rank, world, local_rank = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_2207_06856_gb300 import gpk, workloads
    w = workloads.precision(kernel=gpk.KERNELS[args.kernel])
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    ctx = gpk.Context(local_rank)
    Xh = torch.from_numpy(w.X).pin_memory()
    Bh = torch.from_numpy(w.rhs()).pin_memory()
    X = Xh.to(dev)
    B = Bh.to(dev)
    R, N = B.shape
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def solve(prec, alg, reorth, Xd, Bd, refine=None, refine_resid=0.0):
        pc = gpk.pivchol(ctx, hyp, Xd, w.rank)
        U, st, info = gpk.cg_solve(ctx, hyp, Xd, Bd, pc, tol=TOL * (1.0 - args.stop_margin), max_iter=MAX_ITER,
                                   precision=prec, algorithm=alg, reorth=reorth, U=None, refine_precision=refine,
                                   refine_resid=refine_resid)
        if st != gpk.GP_OK:
            raise RuntimeError(f"solve did not converge: status {st}, residuals {info['rel_resid']}")
        return U, info

    def timed(prec, alg, reorth, steps, warmup, refine=None, refine_resid=0.0):
        for _ in range(warmup):
            solve(prec, alg, reorth, X, B, refine, refine_resid)
        torch.cuda.synchronize()
        times, infos = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            U, info = solve(prec, alg, reorth, X, B, refine, refine_resid)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            infos.append(info)
        return times, infos, U

    # --- headline arm: stable CG with the relaxed FP16 MVM schedule ----------------------
    split = gpk.PRECISIONS[args.precision] | gpk.MVM_PSPLIT | gpk.MVM_XSPLIT
    if args.schedule == "relaxed" and args.precision != "fp32":
        head = (split, "stable", "pinv", args.precision, RELAX_RESID)
    else:
        head = (args.precision, "stable", "pinv", None, 0.0)
    ctx.profile(False)
    sampler = ClockSampler(local_rank)
    launches0 = ctx.launches
    ctx.profile(True)
    sampler.start()
    times, infos, U = timed(head[0], head[1], head[2], args.steps, args.warmup, head[3], head[4])
    clocks = sampler.stop()
    prof_ms, prof_n = ctx.profile_read()
    ctx.profile(False)
    gpu_launches = ctx.launches - launches0
    # launches inside the timed steps only (warm-up solves launch the same number)
    gpu_launches = int(round(gpu_launches * args.steps / (args.steps + args.warmup)))
    t_step = max_over_ranks(float(np.mean(times)), dev)

    # --- residual recomputed in FP64 over all rows (verification, untimed) ---------------
    resid = None
    if rank == 0 and not args.skip_verify:
        import oracle as O
        from oracle import cfp64 as C
        oh = O.Hyp(workloads.KERNEL_NAMES[w.kernel], w.lengthscale, w.outputscale, w.noise)
        t0 = time.perf_counter()
        resid = C.relative_residual(w.X, U.cpu().numpy().T, w.rhs().T, oh)
        t_verify = time.perf_counter() - t0
        if args.measure_kappa:
            # cancellation factor || |Ktilde| |u| || / ||b|| per column (kernel values are positive)
            Ua = np.abs(U.cpu().numpy().T.astype(np.float64))
            kappa = np.linalg.norm(C.kmvm(w.X, Ua, oh), axis=0) / np.linalg.norm(w.rhs().T.astype(np.float64), axis=0)

    # --- roofline of the dominant kernel (tensor-core MVM) ------------------------------
    pairs_per_launch = float(N) * float(N)
    avg_launch_s = (prof_ms / 1e3 / prof_n) if prof_n else float("nan")
    achieved = pairs_per_launch / avg_launch_s / 1e9       # Gpairs/s
    peaks = ctx.measure_peaks()
    mufu_per_pair = 1 if w.kernel == gpk.RBF else 2
    peak_meas = peaks["ex2_per_s"] / mufu_per_pair / 1e9 if w.kernel == gpk.RBF else \
        1.0 / (1.0 / peaks["ex2_per_s"] + 1.0 / peaks["sqrt_per_s"]) / 1e9
    # FP16 RBF: each pair also needs half an FP32 -> FP16x2 conversion on the same unit
    mix_peak = peaks.get("fp16_epilogue_values_per_s", float("nan")) / 1e9
    # the two launch configurations of the schedule, timed alone (20 launches each)
    variants = {}
    for vname, vflags in (("fp16_single", 0), ("fp16_hi_lo_tile_and_inputs", gpk.MVM_PSPLIT | gpk.MVM_XSPLIT)):
        if args.precision == "fp32":
            break
        out_v = torch.empty_like(B)
        for _ in range(3):
            gpk.kmvm(ctx, hyp, X, B, precision=args.precision, add_noise=True, out=out_v, flags=vflags)
        torch.cuda.synchronize()
        ctx.profile(True)
        for _ in range(20):
            gpk.kmvm(ctx, hyp, X, B, precision=args.precision, add_noise=True, out=out_v, flags=vflags)
        torch.cuda.synchronize()
        v_ms, v_n = ctx.profile_read()
        ctx.profile(False)
        v_ach = pairs_per_launch / (v_ms / 1e3 / max(v_n, 1)) / 1e9
        variants[vname] = {"avg_launch_ms": v_ms / max(v_n, 1), "achieved": v_ach, "frac": v_ach / peak_meas,
                           "traffic": KMVM_TRAFFIC_BYTES.get((args.kernel, args.precision, N, R, vflags))}
    mixed = head[3] is not None
    traffic = KMVM_TRAFFIC_BYTES.get((args.kernel, args.precision, N, R, 0))
    launch_mix = None
    if mixed:
        # launches of each configuration in a timed solve: the hi + lo MVM up to the first
        # iterate whose largest recursive residual is <= RELAX_RESID, the single-rounded one after
        rh = np.max(infos[-1]["resid_hist"], axis=1)
        n_it = int(infos[-1]["iters"])
        below = np.nonzero(rh[:n_it + 1] <= RELAX_RESID)[0]
        k_sw = int(below[0]) if below.size else n_it
        launch_mix = {"hi_lo": k_sw, "single": n_it - k_sw}
        t_hl = KMVM_TRAFFIC_BYTES.get((args.kernel, args.precision, N, R, gpk.MVM_PSPLIT | gpk.MVM_XSPLIT))
        traffic = None if (traffic is None or t_hl is None or n_it == 0) else \
            (k_sw * t_hl + (n_it - k_sw) * traffic) / n_it
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_meas, "unit": "Gpairs/s",
                "frac": achieved / peak_meas,
                # mixed schedule: the launch-weighted mean of the two configurations' ncu bytes
                "traffic": traffic, "launch_mix": launch_mix,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "kernel": "kmvm_tp_kernel (tcgen05 S = X_i X_j^T and transposed value product "
                          "O^T = Vt_j P^T over row-tile pairs; kernel function on the SFU)"
                          + (": every launch of the timed solves, hi + lo and single-rounded FP16 tiles"
                             if mixed else ""),
                "variants": variants,
                "peak_source": "measured special-function-unit ex2 rate on this GPU (gp_measure_peaks), "
                               f"{mufu_per_pair} SFU op(s) per kernel pair",
                "frac_of_sfu_ex2_plus_fp16_pack": (achieved / mix_peak) if (w.kernel == gpk.RBF and mix_peak > 0) else None,
                "units_per_launch": pairs_per_launch, "avg_launch_ms": avg_launch_s * 1e3,
                "launches_timed": prof_n, "measured_unit_peaks": peaks}

    # --- comparison arms (same inputs, same preconditioner) ------------------------------
    arms = {}
    if not args.no_arms:
        split = gpk.FP16 | gpk.MVM_PSPLIT | gpk.MVM_XSPLIT
        for name, prec, alg, ro, ref in [("fp32_plain_alg1", "fp32", "standard", "none", None),
                                         ("bf16_hi_lo_stable_alg2", "bf16", "stable", "pinv", None),
                                         ("fp16_single_stable_alg2", "fp16", "stable", "pinv", None),
                                         ("fp16_split_tile_and_inputs_stable_alg2", split, "stable", "pinv", None),
                                         ("fp16_half_exp_stable_alg2", gpk.FP16 | gpk.MVM_HALF_EXP, "stable", "pinv",
                                          None),
                                         ("fp32_stable_alg2", "fp32", "stable", "pinv", None)]:
            if args.arms and name not in args.arms.split(","):
                continue
            ts, inf, _ = timed(prec, alg, ro, max(1, min(args.steps, 2)), 1, ref)
            arms[name] = {"s_per_solve": float(np.mean(ts)), "iters": int(inf[-1]["iters"]),
                          "restarts": int(inf[-1]["restarts"]),
                          "first_run_iters": int(np.max(inf[-1]["lanczos_len"]))}
        # preconditioned MINRES on the single-rounded FP16 MVM, to the same 2-norm target
        if not args.arms or "minres_fp16_single" in args.arms.split(","):
            def solve_mr():
                pc = gpk.pivchol(ctx, hyp, X, w.rank)
                return gpk.minres_solve(ctx, hyp, X, B, pc, tol=TOL * (1.0 - args.stop_margin), max_iter=MAX_ITER,
                                        precision=args.precision, restarts=8, norm="2")
            solve_mr()
            ts_mr = []
            for _ in range(max(1, min(args.steps, 2))):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, st_mr, inf_mr = solve_mr()
                e1.record(stream)
                torch.cuda.synchronize()
                ts_mr.append(e0.elapsed_time(e1) / 1e3)
            arms["minres_fp16_single"] = {"s_per_solve": float(np.mean(ts_mr)), "iters": int(inf_mr["iters"]),
                                          "restarts": int(inf_mr["restarts"]), "status": int(st_mr),
                                          "rel_resid_max": float(np.max(inf_mr["rel_resid"]))}

    # --- end to end through the public API with host buffers ----------------------------
    e2e_times = []
    Uh = torch.empty((R, N), dtype=torch.float32).pin_memory()
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Xd = Xh.to(dev, non_blocking=True)
        Bd = Bh.to(dev, non_blocking=True)
        Ud, _ = solve(head[0], head[1], head[2], Xd, Bd, head[3], head[4])
        Uh.copy_(Ud, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(e0.elapsed_time(e1) / 1e3)
    h2d = Xh.numel() * 4 + Bh.numel() * 4
    d2h = Uh.numel() * 4

    # --- CPU baseline: the oracle's FP64 CG on the host cores (rank 0, N = 1 only) ------
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        from oracle import cfp64 as C
        Bt, oh, Lpc, t_pc = _fp64_cpu_solver(w, workloads.KERNEL_NAMES[w.kernel])
        C.build()
        _, it_done, rel_cpu, t_iter = C.pcg(w.X, Bt, oh, L=Lpc, tol=TOL, max_iter=MAX_ITER,
                                            time_limit_s=args.cpu_seconds)
        converged = bool(np.all(rel_cpu <= TOL))
        iters = it_done if converged else arms.get("fp32_stable_alg2", {}).get("iters", infos[-1]["iters"])
        cpu_val = t_pc + t_iter * iters
        cpu = {"value": cpu_val, "unit": UNIT, "cores": C.threads(), "kind": "oracle",
               "sample": f"FP64 preconditioned CG (Alg. 1, C + OpenMP) on the full workload (N = {N}, {R} RHS, "
                         f"rank-{w.rank} FP64 pivoted Cholesky in {t_pc:.2f} s): {it_done} iterations timed at "
                         f"{t_iter:.2f} s each in a {args.cpu_seconds:.0f} s budget"
                         + ("" if converged else f", extrapolated to {iters} iterations ({FP32_ITERS_NOTE})"),
               "extrapolated": not converged, "iters_timed": it_done, "s_per_iter": t_iter}

    # --- the other workloads on the same GPU, reduced counts (rank 0, N = 1 only) -----
    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = {}
        t0 = time.perf_counter()
        d = diff_measure(args, args.extra_diff_steps)
        extras["differentiation"] = {k: d[k] for k in ("value", "unit", "steps", "config", "loss_first", "loss_last",
                                                       "subsample_exact_nll_initial", "subsample_exact_nll_final",
                                                       "cg_iters", "backward", "clocks")}
        sc = scale_measure(args)
        extras["scale"] = {k: sc[k] for k in ("value", "unit", "config", "mll", "cg_iters", "rel_resid_y_reported",
                                              "rel_resid_y_fp64_sampled_512_rows", "pairs_per_mvm", "clocks")}
        sv = serve_measure(args, args.extra_serve_requests, n_calib=32)
        extras["serving"] = {k: sv[k] for k in ("p50_ms", "p99_ms", "mean_ms", "solves_per_s",
                                                "saturated_solves_per_s", "offered_rate_per_s", "all_ok",
                                                "rel_resid_max", "max_inflight", "config", "clocks")}
        extras["serving"]["requests"] = args.extra_serve_requests
        extras["wall_s"] = time.perf_counter() - t0

    if rank == 0:
        inf = infos[-1]
        line = {
            "metric": METRIC, "value": t_step, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": solve_config(N, R, args.kernel, world),
            "solves_per_s": world / t_step,
            "mvm_schedule": (f"FP16 tensor-core MVM, kernel tile and inputs as hi + lo until every column's "
                             f"recursive relative residual is <= {RELAX_RESID:g}, single-rounded after")
            if head[3] is not None else f"{args.precision} tensor-core MVM throughout",
            "iters": int(inf["iters"]), "restarts": int(inf["restarts"]),
            "final_rel_resid_max": float(np.max(inf["rel_resid"])),
            "stop_tol": TOL * (1.0 - args.stop_margin),
            "fp64_rel_resid_max": None if resid is None else float(np.max(resid)),
            "cancellation_factor_max": float(np.max(kappa)) if args.measure_kappa and resid is not None else None,
            "fp32_check_minus_fp64": None if resid is None else
            float(np.max(np.abs(np.asarray(inf["rel_resid"]) - resid))),
            "fp64_rel_resid_check": None if resid is None else
            f"all {N} rows, FP64 oracle (C + OpenMP), {t_verify:.1f} s, untimed",
            "kmvm_pairs_per_s": achieved * 1e9,
            "arms": arms,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": float(np.mean(e2e_times)), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "adam_step_s": None if extras is None else extras["differentiation"]["value"],
            "scale_mll_grad_step_s": None if extras is None else extras["scale"]["value"],
            "serve_p50_ms": None if extras is None else extras["serving"]["p50_ms"],
            "serve_p99_ms": None if extras is None else extras["serving"]["p99_ms"],
            "serve_solves_per_s": None if extras is None else extras["serving"]["solves_per_s"],
            "other_workloads": extras,
            "peaks_file": {k: _peaks_file().get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_kmvm(args):
    """MVM launches only, at the workload's shape (N = 65,536, 17 RHS): used for
    kernel-level ncu captures with a small device footprint."""
    import torch
    from paper_2207_06856_gb300 import gpk, workloads
    w = workloads.precision(kernel=gpk.KERNELS[args.kernel])
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    ctx = gpk.Context(0)
    X = torch.from_numpy(w.X).cuda()
    B = torch.from_numpy(w.rhs()[:args.nrhs] if args.nrhs else w.rhs()).cuda().contiguous()
    out = torch.empty_like(B)
    fl = (gpk.MVM_ONE_TILE if args.one_tile else 0) | (gpk.MVM_PSPLIT if args.psplit else 0) | \
        (gpk.MVM_HALF_EXP if args.half_exp else 0) | (gpk.MVM_SKIP_TILES if args.skip_tiles else 0) | \
        (gpk.MVM_SYMMETRIC if args.symmetric else 0) | (gpk.MVM_XSPLIT if args.xsplit else 0) | \
        (gpk.MVM_FP32_PV if args.fp32_pv else 0)
    if args.clustered:
        # compact-support case: 16 clusters of 4,096 points (d = 8, within-cluster std 0.3 lengthscales,
        # centres 20 lengthscales apart), stored cluster by cluster
        rng = np.random.default_rng(9)
        cen = rng.standard_normal((16, 8)) * 20.0
        Xc = np.concatenate([c + 0.3 * rng.standard_normal((4096, 8)) for c in cen]).astype(np.float32)
        X = torch.from_numpy(Xc).cuda()
    for _ in range(args.warmup):
        gpk.kmvm(ctx, hyp, X, B, precision=args.precision, add_noise=True, out=out, flags=fl)
    torch.cuda.synchronize()
    ctx.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        gpk.kmvm(ctx, hyp, X, B, precision=args.precision, add_noise=True, out=out, flags=fl)
    e1.record()
    torch.cuda.synchronize()
    ms, n = ctx.profile_read()
    if n == 0:   # the SIMT engine is not event-profiled: time the whole calls
        ms, n = e0.elapsed_time(e1), args.steps
    ctx.check()
    pairs = float(w.N) ** 2
    if args.skip_tiles:
        ev, tot = gpk.kmvm_tile_count(ctx, hyp, X, precision=args.precision, flags=fl)
    else:
        ev, tot = (w.N + 1, 2 * w.N) if args.symmetric else (1, 1)   # symmetric: N (N + 1) / 2 of N^2 pairs
    print(json.dumps({"mode": "kmvm", "precision": args.precision, "kernel": args.kernel, "rhs": int(B.shape[0]),
                      "inputs": "clustered (16 clusters)" if args.clustered else "precision workload",
                      "skip_tiles": bool(args.skip_tiles), "symmetric": bool(args.symmetric),
                      "evaluated_fraction": ev / tot,
                      "evaluated_pairs_per_s": pairs * ev / tot / (ms / max(n, 1) / 1e3),
                      "engine": "one-tile" if args.one_tile else "pair", "psplit": bool(args.psplit),
                      "half_exp": bool(args.half_exp), "xsplit": bool(args.xsplit), "fp32_pv": bool(args.fp32_pv),
                      "launches": n,
                      "avg_launch_ms": ms / max(n, 1), "pairs_per_s": pairs / (ms / max(n, 1) / 1e3)}), flush=True)


def run_minres(args):
    """Preconditioned MINRES (gp_minres_solve) on the precision workload
    (N = 65,536, d = 8, RBF, 1 + 16 right-hand sides, rank-100 pivoted
    Cholesky): time to a relative 2-norm residual of 1e-2 at the FP32
    true-residual checks (MINRES minimises the P^-1 norm; its recurrence target
    follows the two norms' ratio after each check), for the single-rounded
    and the hi + lo FP16 MVM, against CG on the same inputs; both residual norms
    of every solution recomputed in FP64 over all rows by the oracle (untimed)."""
    import torch
    import oracle as O
    from oracle import cfp64 as C
    from paper_2207_06856_gb300 import gpk, workloads
    w = workloads.precision(kernel=gpk.KERNELS[args.kernel])
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    ctx = gpk.Context(0)
    X = torch.from_numpy(w.X).cuda()
    Bh = w.rhs()
    B = torch.from_numpy(Bh).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    oh = O.Hyp(workloads.KERNEL_NAMES[w.kernel], w.lengthscale, w.outputscale, w.noise)
    L64, _ = O.pivoted_cholesky(w.X, oh, w.rank)
    C.build()
    split = gpk.FP16 | gpk.MVM_PSPLIT | gpk.MVM_XSPLIT

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return float(np.mean(ts)), out

    def verify(U):
        Ut = U.cpu().numpy().T.astype(np.float64)
        res = C.kmvm(w.X, Ut, oh, add_noise=True) - Bh.T.astype(np.float64)
        Bt = Bh.T.astype(np.float64)
        rel2 = np.linalg.norm(res, axis=0) / np.linalg.norm(Bt, axis=0)
        relp = np.sqrt(np.sum(res * O.precond_apply(L64, w.noise, res), axis=0) /
                       np.sum(Bt * O.precond_apply(L64, w.noise, Bt), axis=0))
        return float(rel2.max()), float(relp.max())

    out = {}
    for name, prec, ref in (("minres_fp16_single", "fp16", None), ("minres_fp16_hi_lo", split, None),
                            ("minres_relaxed", split, "fp16"), ("minres_fp32", "fp32", None)):
        def solve_m(prec=prec, ref=ref):
            pc = gpk.pivchol(ctx, hyp, X, w.rank)
            return gpk.minres_solve(ctx, hyp, X, B, pc, tol=TOL * (1.0 - args.stop_margin), max_iter=MAX_ITER,
                                    precision=prec, restarts=8, norm="2", refine_precision=ref,
                                    refine_resid=RELAX_RESID if ref else 0.0)
        t, (U, st, info) = timed(solve_m)
        r2, rp = verify(U)
        out[name] = {"s_per_solve": t, "status": int(st), "iters": int(info["iters"]),
                     "restarts": int(info["restarts"]), "fp64_rel_resid_p_max": rp, "fp64_rel_resid_2_max": r2}
    for name, prec, ref, rr in (("cg_relaxed", split, "fp16", RELAX_RESID), ("cg_fp16_single", "fp16", None, 0.0)):
        def solve_c(prec=prec, ref=ref, rr=rr):
            pc = gpk.pivchol(ctx, hyp, X, w.rank)
            return gpk.cg_solve(ctx, hyp, X, B, pc, tol=TOL * (1.0 - args.stop_margin), max_iter=MAX_ITER,
                                precision=prec, refine_precision=ref, refine_resid=rr)
        t, (U, st, info) = timed(solve_c)
        r2, rp = verify(U)
        out[name] = {"s_per_solve": t, "status": int(st), "iters": int(info["iters"]),
                     "restarts": int(info["restarts"]), "fp64_rel_resid_p_max": rp, "fp64_rel_resid_2_max": r2}
    print(json.dumps({"mode": "minres", "workload": solve_config(w.N, Bh.shape[0], args.kernel, 1)["workload"],
                      "tol": TOL * (1.0 - args.stop_margin), "steps": args.steps, "warmup": args.warmup,
                      "note": "both stop on the 2-norm residual of the FP32 check; MINRES's recurrence on the "
                              "P^-1 norm (target rescaled at each check)",
                      "results": out}), flush=True)


def run_sumstudy(args):
    """Summation-variant study (Sec. 4.1, Fig. 4b; App. B, Fig. A.1a) on inputs
    shaped like the scale workload (N = 65,536 drawn from its distribution,
    d = 11, Matern-3/2 ARD), one right-hand side y: the CUDA-core FP16 MVM with
    each accumulation scheme and the tensor-core FP16 MVM, time and relative
    error on 512 sampled rows against the FP64 oracle."""
    import torch
    import oracle as O
    from oracle import cfp64 as C
    from paper_2207_06856_gb300 import gpk, workloads
    w = workloads.scale(N=args.study_n)
    N = w.X.shape[0]
    ctx = gpk.Context(0)
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = torch.from_numpy(w.X).cuda()
    V = torch.from_numpy(w.y[None, :].astype(np.float32)).cuda()
    rows = np.sort(np.random.default_rng(4).choice(N, 512, replace=False))
    oh = O.Hyp(workloads.KERNEL_NAMES[w.kernel], w.lengthscale.astype(np.float64), w.outputscale, w.noise)
    ref = C.kmvm(w.X, w.y.astype(np.float64)[:, None], oh, rows=rows)[:, 0]
    res = {}
    names = {0: "tensor_core_fp32_acc", 1: "simt_fp16_fp32_acc", 2: "simt_fp16_half_acc",
             3: "simt_fp16_block_sums", 4: "simt_fp16_kahan"}
    for s_ in (0, 1, 2, 3, 4):
        fl = gpk.MVM_SUM(s_) if s_ else 0
        out = gpk.kmvm(ctx, hyp, X, V, precision="fp16", add_noise=True, flags=fl)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            gpk.kmvm(ctx, hyp, X, V, precision="fp16", add_noise=True, flags=fl, out=out)
        e1.record()
        torch.cuda.synchronize()
        got = out[0].cpu().numpy().astype(np.float64)[rows]
        res[names[s_]] = {"ms": e0.elapsed_time(e1) / args.steps,
                          "rel_err": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
    ctx.check()
    print(json.dumps({"mode": "sumstudy", "N": N, "d": int(w.X.shape[1]), "kernel": "matern32", "R": 1,
                      "variants": res}), flush=True)


def vjp_timing(ctx, w, steps: int, precisions=("fp16", "fp32")) -> dict:
    """CUDA-event time of the MVM backward on workload w (17 columns, gradient in
    X too), per precision, with pairs/s = N^2 / time."""
    import torch
    from paper_2207_06856_gb300 import gpk
    N = w.X.shape[0]
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = torch.from_numpy(w.X).cuda()
    rng = np.random.default_rng(5)
    U = torch.from_numpy(rng.standard_normal((17, N)).astype(np.float32)).cuda()
    W = torch.from_numpy(rng.standard_normal((17, N)).astype(np.float32)).cuda()
    res = {}
    for prec in precisions:
        for _ in range(2):
            gpk.kmvm_vjp(ctx, hyp, X, U, W, want_X=True, precision=prec)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            gpk.kmvm_vjp(ctx, hyp, X, U, W, want_X=True, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[prec] = {"ms_per_backward": ms, "pairs_per_s": float(N) ** 2 / (ms * 1e-3)}
    if "fp16" in precisions:
        ctx.profile(True)
        gpk.kmvm_vjp(ctx, hyp, X, U, W, want_X=True, precision="fp16")
        kms, kn = ctx.profile_read()
        ctx.profile(False)
        peaks = ctx.measure_peaks()
        kpairs = float(N) ** 2 / (kms / max(kn, 1) * 1e-3)
        res["fp16"].update({"kernel_ms": kms / max(kn, 1), "kernel_pairs_per_s": kpairs,
                            "roofline": {"bound": "alu", "achieved": kpairs / 1e9, "peak": peaks["ex2_per_s"] / 1e9,
                                         "unit": "Gpairs/s", "frac": kpairs / peaks["ex2_per_s"],
                                         "peak_source": "measured ex2 rate on this GPU, one ex2 per pair (RBF)",
                                         "kernel": "kvjp_tc_kernel"}})
    ctx.check()
    return res


def run_vjp(args):
    """The backward of the kernel MVM alone on the differentiation workload
    (N = 262,144, d = 18, ARD RBF, 17 columns): the tensor-core FP16 backward
    and the CUDA-core FP32 one, CUDA-event timed; pairs/s = N^2 / time."""
    from paper_2207_06856_gb300 import gpk, workloads
    w = workloads.differentiation(N=args.diff_n)
    ctx = gpk.Context(0)
    precs = ("fp16",) if args.vjp_fp16_only else ("fp16", "fp32")
    res = vjp_timing(ctx, w, args.steps, precs)
    print(json.dumps({"mode": "vjp", "N": int(w.X.shape[0]), "d": int(w.X.shape[1]), "R": 17, **res}), flush=True)


def run_serve(args):
    print(json.dumps(serve_measure(args, args.serve_requests)), flush=True)


def serve_measure(args, n_requests, n_calib=None):
    """Serving workload: 512 posterior-mean requests (N log-uniform in [1k, 200k],
    d in {4, 8, 16}, RBF / Matern-3/2, 1024 test points each), FP16 MVM + CG to
    1e-2 with a rank-20 preconditioner.  First the saturated throughput is
    measured (a batch of requests submitted at once), then all requests are
    replayed with Poisson arrivals at 0.7x that rate; p50 / p99 latency
    (submit -> result on the host) and completed solves/s are reported."""
    import torch
    from paper_2207_06856_gb300 import gpk, workloads
    torch.cuda.set_device(0)
    reqs = workloads.serving(n_requests=512, rate_per_s=1.0, seed=1)[:n_requests]
    pin = gpk.Server.pinned
    inputs = [(gpk.Hyper(r.kernel, r.lengthscale, r.outputscale, r.noise), pin(r.X), pin(r.y), pin(r.Xstar))
              for r in reqs]
    sprec = gpk.FP16 | gpk.MVM_XSPLIT | (gpk.MVM_FP32_PV if args.serve_schedule == "fp32pv" else gpk.MVM_PSPLIT)
    srv = gpk.Server(0, arena_bytes=int(args.serve_arena_gb * (1 << 30)), max_slots=args.serve_slots, rank=20,
                     precision=sprec, mean_precision="fp32", tol=TOL,
                     max_iter=1000, restarts=4,
                     refine_precision="fp16" if args.serve_schedule == "relaxed" else None,
                     refine_resid=RELAX_RESID if args.serve_schedule == "relaxed" else 0.0,
                     large_n=args.serve_large_n, large_reserve=args.serve_large_reserve)
    small = workloads.serving(n_requests=3, rate_per_s=1.0, seed=2, n_min=1000, n_max=2000)
    for r in small:   # warm-up
        srv.submit(gpk.Hyper(r.kernel, r.lengthscale, r.outputscale, r.noise), r.X, r.y, r.Xstar).result()
    # saturated throughput: a random subset submitted at once
    n_calib = args.serve_calib if n_calib is None else n_calib
    cal = np.random.default_rng(3).choice(len(inputs), min(n_calib, len(inputs)), replace=False)
    t0 = time.perf_counter()
    futs = [srv.submit(*inputs[i]) for i in cal]
    for f in futs:
        f.result()
    sat = len(cal) / (time.perf_counter() - t0)
    rate = args.serve_load * sat
    sampler = ClockSampler(0)
    launches0 = srv.stats()["launches"]
    sampler.start()
    futs = []
    t_start = time.perf_counter()
    for r, inp in zip(reqs, inputs):
        due = t_start + r.arrival_s / rate
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        futs.append(srv.submit(*inp))
    res = [f.result() for f in futs]
    t_end = time.perf_counter()
    clocks = sampler.stop()
    st = srv.stats()
    lat = np.array([s["latency_ms"] for _, s in res])
    iters = np.array([s["iters"] for _, s in res])
    status = [s["status"] for _, s in res]
    rel = np.array([s["rel_resid"] for _, s in res])
    # spot check against the FP64 oracle on the smallest requests (untimed)
    import oracle as O
    check = []
    for i in np.argsort([r.X.shape[0] for r in reqs])[:3]:
        r = reqs[i]
        oh = O.Hyp(workloads.KERNEL_NAMES[r.kernel], r.lengthscale.astype(np.float64), r.outputscale, r.noise)
        ref = O.kernel_matrix(r.Xstar, r.X, oh) @ O.cholesky_solve(r.X, oh, r.y.astype(np.float64))
        check.append(float(np.linalg.norm(res[i][0] - ref) / np.linalg.norm(ref)))
    srv.close()
    wall = t_end - t_start
    line = {
        "metric": "serve_latency_p99", "value": float(np.percentile(lat, 99)), "unit": "ms", "n_gpus": 1,
        "steps": len(reqs), "warmup": len(small), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16", "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} posterior-mean requests (the first {len(reqs)} of the 512-request "
                               f"trace), Poisson arrivals at "
                               f"{args.serve_load:.2f}x saturated rate, N log-uniform [1k, 200k], d in {{4,8,16}}, "
                               "RBF/Matern-3/2, 1024 test points, FP16 tensor-core MVM ("
                               + {"relaxed": "kernel tile and inputs as hi + lo until every residual is <= 30 x tol, "
                                             "single-rounded after",
                                  "split": "kernel tile and inputs as hi + lo",
                                  "fp32pv": "inputs as hi + lo, FP32 kernel values and value product"}[
                                   args.serve_schedule] + ") + stable CG to 1e-2, rank 20",
                   "slots": args.serve_slots, "arena_gb": args.serve_arena_gb,
                   "large_n": args.serve_large_n, "large_reserve_sms": args.serve_large_reserve},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "solves_per_s": len(reqs) / wall, "saturated_solves_per_s": sat,
        "offered_rate_per_s": rate, "iters_p50": float(np.median(iters)), "iters_max": int(iters.max()),
        "all_ok": all(s == gpk.GP_OK for s in status), "rel_resid_max": float(rel.max()),
        "max_inflight": st["max_inflight"], "arena_peak_gb": st["peak_bytes"] / 2 ** 30,
        "oracle_mean_relerr_smallest3": check, "gpu_launches": int(st["launches"] - launches0),
        "clocks": clocks,
    }
    return line


def run_diff(args):
    print(json.dumps(diff_measure(args, args.diff_steps)), flush=True)


def diff_measure(args, n_steps):
    """Differentiation workload: N = 262,144, d = 18 (ARD RBF, Gaussian-mixture
    inputs, random-feature targets), the training loop of the paper: Adam on the
    hyperparameters, each step one MLL + gradient (CG to 1.0 with 10 iterations
    at least and 50 at most, 16 P-distributed probes, SLQ log-determinant,
    rank-100 preconditioner, FP16 tensor-core MVM, hand-written backward)."""
    import torch
    from paper_2207_06856_gb300 import autograd, gpk, workloads
    torch.cuda.set_device(0)
    w = workloads.differentiation(N=args.diff_n)
    ctx = gpk.Context(0)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    step_s = []
    t_last = [None]

    def cb(step, rec):
        torch.cuda.synchronize()
        t = time.perf_counter()
        step_s.append(t - t_last[0])
        t_last[0] = t

    launches0 = ctx.launches
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    t_last[0] = time.perf_counter()
    hist = autograd.fit(ctx, X, y, w.kernel, w.lengthscale, w.outputscale, w.noise, steps=n_steps, lr=0.05,
                        M=16, rank=w.rank, tol=args.diff_tol, max_iter=args.diff_max_iter, min_iter=10,
                        precision=args.precision, callback=cb)
    clocks = sampler.stop()
    timed = step_s[1:] if len(step_s) > 1 else step_s   # the first step also builds the workspace
    iters = [int(h[4]["iters"]) for h in hist]
    # progress check with the FP64 oracle: exact negative log marginal likelihood of a
    # random 3,000-point subsample at the initial and the final hyperparameters
    import oracle as O
    sub = np.sort(np.random.default_rng(11).choice(w.X.shape[0], 3000, replace=False))
    Xs, ys = w.X[sub], w.y[sub]
    kn = workloads.KERNEL_NAMES[w.kernel]
    nll0 = O.mll_exact(Xs, ys, O.Hyp(kn, w.lengthscale.astype(np.float64), w.outputscale, w.noise))
    nll1 = O.mll_exact(Xs, ys, O.Hyp(kn, np.asarray(hist[-1][1], np.float64), hist[-1][2], hist[-1][3]))
    line = {
        "metric": "adam_step_time", "value": float(np.mean(timed)), "unit": "s", "n_gpus": 1,
        "steps": len(timed), "warmup": len(step_s) - len(timed), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"differentiation: N={w.X.shape[0]} d=18 ARD RBF, 8-component Gaussian mixture, "
                               "random-feature GP targets + noise 0.1, 16 P-distributed probes, SLQ log-det, rank 100, "
                               f"CG tol {args.diff_tol} (10..{args.diff_max_iter} iterations), Adam lr 0.05 on "
                               "softplus parameters"},
        "loss_first": hist[0][0], "loss_last": hist[-1][0],
        "subsample_exact_nll_initial": nll0, "subsample_exact_nll_final": nll1,
        "lengthscale_last": [float(v) for v in hist[-1][1]], "outputscale_last": hist[-1][2],
        "noise_last": hist[-1][3], "cg_iters": iters, "total_s": float(np.sum(step_s)),
        "gpu_launches": int(ctx.launches - launches0), "clocks": clocks,
        "backward": vjp_timing(ctx, w, 3, ("fp16",)),
    }
    ctx.close()
    return line


def run_scale(args):
    print(json.dumps(scale_measure(args)), flush=True)


def scale_measure(args):
    """Scale workload: N = 1,843,200, d = 11, Matern-3/2 ARD: one full MLL +
    gradient step (rank-100 pivoted Cholesky, 1 + 16 right-hand sides with
    P-distributed probes, CG to 1.0 with 10..50 iterations, SLQ log-det, FP16
    tensor-core MVM, hand-written backward).  Checks the solves on sampled rows
    with the FP64 oracle."""
    import torch
    from paper_2207_06856_gb300 import gpk, workloads
    torch.cuda.set_device(0)
    w = workloads.scale(N=args.scale_n)
    N, d = w.X.shape
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    ctx = gpk.Context(0)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    rng = np.random.default_rng(7)
    Z = torch.from_numpy(rng.standard_normal((16, N)).astype(np.float32)).cuda()
    E = torch.from_numpy(rng.standard_normal((16, w.rank)).astype(np.float32)).cuda()
    sampler = ClockSampler(0)
    launches0 = ctx.launches
    sampler.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pc = gpk.pivchol(ctx, hyp, X, w.rank)
    mll, g, _, U, info = gpk.mll_and_grad(ctx, hyp, X, y, Z, precond=pc, E=E, precond_probes=True, want_logdet=True,
                                          tol=w.tol, min_iter=10, max_iter=w.max_iter, precision=args.precision,
                                          return_U=True)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t = e0.elapsed_time(e1) / 1e3
    # sampled FP64 check of the y-solve: residual of column 0 on 512 rows
    import oracle as O
    from oracle import cfp64 as C
    rows = np.sort(np.random.default_rng(3).choice(N, 512, replace=False))
    oh = O.Hyp(workloads.KERNEL_NAMES[w.kernel], w.lengthscale, w.outputscale, w.noise)
    u0 = U[0].cpu().numpy().astype(np.float64)
    r = C.kmvm(w.X, u0[:, None], oh, rows=rows)[:, 0] - w.y[rows].astype(np.float64)
    est = float(np.sqrt(N / len(rows) * np.sum(r * r)) / np.linalg.norm(w.y.astype(np.float64)))
    line = {
        "metric": "mll_gradient_step_time", "value": t, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": f"scale: N={N} d=11 Matern-3/2 ARD, 16-component anisotropic Gaussian mixture, "
                               "rank-100 pivoted Cholesky, 1+16 RHS (P-distributed probes), CG tol 1.0 "
                               "(10..50 iterations), SLQ log-det"},
        "mll": mll, "grad": [float(v) for v in g], "cg_iters": int(info["iters"]),
        "rel_resid_y_reported": float(info["rel_resid"][0]), "rel_resid_y_fp64_sampled_512_rows": est,
        "pairs_per_mvm": float(N) * float(N), "gpu_launches": int(ctx.launches - launches0), "clocks": clocks,
    }
    ctx.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "fp32"])
    ap.add_argument("--schedule", default="relaxed", choices=["relaxed", "single"],
                    help="headline MVM schedule: hi + lo tile and inputs until the residual is 30 x tol, "
                         "then single-rounded (relaxed), or the single-rounded MVM throughout")
    ap.add_argument("--kernel", default="rbf", choices=["rbf", "matern32"])
    ap.add_argument("--no-arms", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-verify", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--stop-margin", type=float, default=STOP_MARGIN)
    ap.add_argument("--measure-kappa", action="store_true", help="also report the cancellation factor")
    ap.add_argument("--no-extras", action="store_true", help="skip the differentiation / scale / serving runs")
    ap.add_argument("--extra-diff-steps", type=int, default=4)
    ap.add_argument("--extra-serve-requests", type=int, default=96)
    ap.add_argument("--ref-iters", type=int, default=152)
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "kmvm", "serve", "diff", "scale", "vjp", "sumstudy", "minres"])
    ap.add_argument("--diff-steps", type=int, default=20)
    ap.add_argument("--diff-n", type=int, default=262144)
    ap.add_argument("--diff-tol", type=float, default=1.0)
    ap.add_argument("--diff-max-iter", type=int, default=50)
    ap.add_argument("--scale-n", type=int, default=1843200)
    ap.add_argument("--study-n", type=int, default=65536)
    ap.add_argument("--vjp-fp16-only", action="store_true")
    ap.add_argument("--one-tile", action="store_true", help="kmvm mode: the one-row-tile tensor-core engine")
    ap.add_argument("--psplit", action="store_true", help="kmvm mode: FP16 kernel tile as hi + lo")
    ap.add_argument("--half-exp", action="store_true", help="kmvm mode: FP16 exp2 argument and exponential")
    ap.add_argument("--skip-tiles", action="store_true", help="kmvm mode: compact-support tile skipping")
    ap.add_argument("--clustered", action="store_true", help="kmvm mode: clustered inputs (16 far-apart clusters)")
    ap.add_argument("--symmetric", action="store_true", help="kmvm mode: FP32 symmetric half-work MVM")
    ap.add_argument("--xsplit", action="store_true", help="kmvm mode: inputs carried as hi + lo")
    ap.add_argument("--fp32-pv", action="store_true", help="kmvm mode: FP32 value product (1 to 4 right-hand sides)")
    ap.add_argument("--serve-schedule", default="fp32pv", choices=["relaxed", "split", "fp32pv"],
                    help="serving CG MVM: FP32 kernel values and value product with hi + lo inputs (fp32pv, the "
                         "default), hi + lo tile and inputs throughout (split), or hi + lo until the residual is "
                         "30 x tol then single-rounded (relaxed; fails on low-noise requests)")
    ap.add_argument("--serve-large-n", type=int, default=32768,
                    help="serving: requests with N >= this leave --serve-large-reserve SMs to smaller ones")
    ap.add_argument("--serve-large-reserve", type=int, default=16, help="serving: 0 = every request on all SMs")
    ap.add_argument("--arms", default="", help="comma-separated subset of the comparison arms (default: all)")
    ap.add_argument("--nrhs", type=int, default=0, help="kmvm mode: use the first NRHS right-hand sides (0: all 17)")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-arena-gb", type=float, default=48.0)
    ap.add_argument("--serve-calib", type=int, default=64)
    ap.add_argument("--serve-load", type=float, default=0.7)
    args = ap.parse_args()
    if args.mode == "kmvm":
        run_kmvm(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "diff":
        run_diff(args)
    elif args.mode == "scale":
        run_scale(args)
    elif args.mode == "vjp":
        run_vjp(args)
    elif args.mode == "sumstudy":
        run_sumstudy(args)
    elif args.mode == "minres":
        run_minres(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
