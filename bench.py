#!/usr/bin/env python
"""Benchmark: seconds per CP-ALS-QR sweep (ALS-QR-BRE: restructured dimension
tree + customised extrapolation) on the 400 x 400 x 400 rank-32 workload.

A step is one sweep (every mode updated once: TTM chain, Khatri-Rao QR,
V = Y_(n) Q0, R0^{-T} solve, normalisation, factor QR, fit) on a seeded
synthetic tensor resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec split|fp64] [--quick]

N > 1 (torchrun): independent replicas, one per GPU (the solver has no
cross-GPU exchange in this build); value = max-over-ranks time / sweeps of all
ranks.  --impl reference times the FP64 CPU oracle on the host cores instead.
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

METRIC = "sec/CP-ALS-QR sweep & time-to-fit 1e-6 (mixed+learned vs FP64 GPU); TTM %peak"
WORKLOAD = "cube400_r32_c09"
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of the current kernels
# on this workload (the same launch shapes through bench.py --kernel); None where a kernel changed
# after its capture
TTM_TC_TRAFFIC = 270.4e6    # ttm_tc_kernel<0, 0, 32>, 1 x 400 x 160000 -> R = 32 (256.1 MB read + 14.3 MB written)
TTM_DEEP_TRAFFIC = 20.6e6   # ttm_tc_kernel<1, 0, 32>, 12800 x 400 x 1 -> R = 32 (20.6 MB read, output left in L2)
# whole-GPU FP64 DFMA rate measured by a probe on the GB300s (TFLOP/s)
FP64_PEAK_TFLOPS = 1.20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sweep_times(prob, tree, sweeps):
    """Wall time of each oracle sweep on the host cores (FP64 numpy/BLAS)."""
    from oracle import cpqr_oracle as o
    stamps = [time.perf_counter()]
    o.cp_als_qr(prob.X, prob.R, prob.A0, tree=tree, extrapolate=True, max_sweeps=sweeps,
                on_sweep=lambda k, f: stamps.append(time.perf_counter()))
    return np.diff(stamps)


def run_reference(args, rank):
    if rank != 0:
        return None
    from oracle import cpqr_oracle as o
    from paper_2503_18759_gb300 import inputs
    prob = inputs.workload(WORKLOAD, seed=0)
    t = oracle_sweep_times(prob, o.TREE_RESTRUCTURED, args.warmup + args.steps)
    per = float(np.mean(t[args.warmup:])) if args.steps > 0 else float("nan")
    cores = os.cpu_count()
    return {"metric": METRIC, "value": per, "unit": "s/sweep", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "dims": prob.dims, "rank": prob.R, "tree": "restructured",
                       "extrapolation": "paper rule", "l2": "no flush; 512 MB FP64 tensor > L2"},
            "cpu_baseline": {"value": per, "unit": "s/sweep", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full-size oracle sweeps after {args.warmup} warm-up sweeps"},
            "e2e": {"value": per, "unit": "s/sweep", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _guard(st, args):
    """How the Gram-route QRs of the run (warm-up, timed and timing sweeps) were finished when their
    first Cholesky pass was not accurate enough: by a second Cholesky pass or by the Householder QR."""
    return {"second_cholesky_pass": int(st.qr_second_pass), "householder": int(st.qr_fallbacks),
            "sweeps": int(args.warmup + 2 * args.steps)}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2503_18759_gb300 import binding as b
    from paper_2503_18759_gb300 import build, inputs

    build.build()
    b.lib()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = b.PREC_SPLIT_BF16 if args.prec == "split" else b.PREC_FP64
    wname = args.workload
    if wname == WORKLOAD:
        prob = inputs.workload(wname, seed=rank)
        X = torch.from_numpy(prob.X).to(dev)
    else:  # the other named workloads (timing and buckets only), generated on the GPU
        cfg = dict(inputs.WORKLOADS[wname])
        prob = inputs.make_problem_device(wname, cfg.pop("dims"), cfg.pop("R"), seed=rank, c=cfg.get("c"),
                                          eta=cfg.get("eta", 0.0), device=str(dev))
        X = prob.X
    tree = {"standard": b.TREE_STANDARD, "none": b.TREE_NONE}.get(args.tree, b.TREE_RESTRUCTURED)
    xbytes = X.numel() * X.element_size()
    opts = b.make_options(tree=tree, prec=prec, extrap=b.EXTRAP_PAPER)
    clocks = ClockSampler(local_rank)
    clocks.start()
    dec = b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts)
    dec.sweep(args.warmup)
    launches0 = dec.stats().launches

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_range:
        torch.cuda.profiler.start()
    e0.record()
    fits = dec.sweep(args.steps)
    e1.record()
    if args.profile_range:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    barrier()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    launches = dec.stats().launches - launches0
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # per-kernel device time over the same number of sweeps (CUDA events around each launch)
    dec.set_timing(True)
    dec.sweep(args.steps)
    st = dec.stats()
    dec.set_timing(False)
    buckets = {name: st.ms_bucket[i] / max(args.steps, 1) for i, name in enumerate(b.BUCKETS)}
    n_full = st.n_bucket[0]
    full_ms = st.ms_bucket[0] / max(n_full, 1)
    n_deep = st.n_bucket[1]
    deep_ms = st.ms_bucket[1] / max(n_deep, 1)
    out = None
    if rank == 0 and wname != WORKLOAD:
        out = {"metric": METRIC, "value": ms * 1e-3 / world, "unit": "s/sweep", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "bf16x3+f32+f64" if prec == b.PREC_SPLIT_BF16 else "f64",
               "data": "synthetic", "config": {"workload": wname, "dims": prob.dims, "rank": prob.R,
                                               "tree": args.tree, "precision": args.prec},
               "buckets_ms_per_sweep": buckets, "launches_per_bucket_per_sweep":
                   {name: st.n_bucket[i] / max(args.steps, 1) for i, name in enumerate(b.BUCKETS)},
               "ttm_flops_per_sweep": st.ttm_flops / (args.warmup + 2 * args.steps), "gpu_launches": int(launches),
               "fit_last": float(fits[-1]) if len(fits) else None,
               "qr_guard": _guard(st, args),
               "note": "extra workload: not the bench line (no roofline, e2e or CPU baseline)"}
    elif rank == 0:
        hbm, peak_kind = _peaks()
        # first-level TTM, algorithmic bytes: X once (FP32, or bf16 hi + lo: 4 B/element) + output (FP32/FP64)
        out_elems = prob.X.size // prob.dims[0] * prob.R  # every full TTM here shrinks one side of 400 to R
        ob = 4 if prec == b.PREC_SPLIT_BF16 else 8
        alg_bytes = xbytes + out_elems * ob
        achieved = alg_bytes / (full_ms * 1e-3) / 1e9 if n_full else None
        roof_ttm = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": (achieved / hbm) if achieved else None,
                    "traffic": TTM_TC_TRAFFIC if prec == b.PREC_SPLIT_BF16 else None,
                    "kernel": "ttm_tc_kernel (first-level TTM, full tensor)",
                    "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                    "note": "persistent grid on all SMs; the previous sweep's lagged explicit residual streams X "
                            "beside it; alone the same launch takes ~54 us (ncu)",
                    "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": full_ms, "launches": int(n_full)}
        # deeper TTMs (every one on this workload contracts a 400 x 400 x 32 node to 400 x 32 x 32):
        # node read once (4 B per element: FP32, or bf16 hi + lo) + result written once (4 B per element)
        deep_in, deep_out = 400 * 400 * prob.R, 400 * prob.R * prob.R
        deep_bytes = (deep_in + deep_out) * (4 if prec == b.PREC_SPLIT_BF16 else 8)
        roof_deep = {"bound": "hbm", "achieved": deep_bytes / (deep_ms * 1e-3) / 1e9 if n_deep else None,
                     "peak": hbm, "unit": "GB/s", "traffic": TTM_DEEP_TRAFFIC if prec == b.PREC_SPLIT_BF16 else None,
                     "kernel": "ttm_tc_kernel (deeper tree levels, MN- and K-major)",
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)", "alg_bytes_per_launch": deep_bytes,
                     "avg_launch_ms": deep_ms, "launches": int(n_deep),
                     "note": "launches run beside the Khatri-Rao QR on another stream; the 20.5 MB node can be L2-resident"}
        roof_deep["frac"] = roof_deep["achieved"] / hbm if n_deep else None
        if prec == b.PREC_FP64:
            flops = 2 * prob.X.size * prob.R
            roof_ttm.update({"bound": "alu", "achieved": flops / (full_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "kernel": "ttm_kernel<float,double,double> (first-level TTM, FP64)",
                             "peak_kind": "FP64 DFMA rate measured by a probe", "alg_flops_per_launch": flops})
            roof_ttm["frac"] = roof_ttm["achieved"] / roof_ttm["peak"]
        # the mode update after V (Alg. 3 lines 8-10: eq. 19, the R0^{-T} solve, normalisation and the
        # factor QR by the guarded Gram route): FP64 and float-float, bound by the latency of its
        # serial parts (the 32-step back substitution, the 32-step Cholesky), not by a roof
        n_qr = st.n_bucket[4]
        qr_ms = st.ms_bucket[4] / max(n_qr, 1)
        I, R = prob.dims[0], prob.R
        # solve I R^2, Gram I R^2, Cholesky R^3 / 3, substitution I R^2, E I R^2, correction I R^2
        qr_flops = 5 * I * R * R + R ** 3 // 3
        roof_qr = {"bound": "alu", "achieved": qr_flops / (qr_ms * 1e-3) / 1e12 if n_qr else None,
                   "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "traffic": None,
                   "kernel": "finish_prep_kernel, fg_chol_kernel, fg_q1_kernel, kg_e_kernel, kg_q0_kernel "
                             "(eq. 19, R0^{-T} solve, normalise, Gram-route factor QR; the Householder finish "
                             "launched after them returns at once unless the guard trips)",
                   "peak_kind": "FP64 DFMA rate of the whole GPU measured by a probe; the chain is bound by the "
                                "latency of its serial 32-step solve and Cholesky",
                   "alg_flops_per_launch": qr_flops, "avg_launch_ms": qr_ms, "launches": int(n_qr)}
        roof_qr["frac"] = roof_qr["achieved"] / roof_qr["peak"] if n_qr else None
        # the dominant kernel by device time: the first-level TTM (one launch per sweep reads all of X)
        roof = roof_ttm
        roof["share_of_sweep"] = (st.ms_bucket[0] / max(args.steps, 1)) / ms if ms > 0 else None
        out = {"metric": METRIC, "value": ms * 1e-3 / world, "unit": "s/sweep", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None,
               "dtype": "bf16x3+f32+f64" if prec == b.PREC_SPLIT_BF16 else "f64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "dims": prob.dims, "rank": prob.R, "tree": "restructured",
                          "extrapolation": "paper rule", "precision": args.prec,
                          "l2": "no flush; inputs larger than L2 (256 MB tensor, 512 MB bf16 split)",
                          "replicas": world},
               "roofline": roof,
               "roofline_ttm_deep": roof_deep,
               "roofline_factor_qr": roof_qr,
               "buckets_ms_per_sweep": buckets,
               "gpu_launches": int(launches),
               "fit_last": float(fits[-1]) if len(fits) else None,
               "qr_guard": _guard(st, args)}
    if args.metrics_jsonl and rank == 0:
        dec.write_history_jsonl(args.metrics_jsonl, workload=wname, ms_per_sweep_timed_avg=ms)
    dec.close()
    if rank == 0 and not args.quick and wname == WORKLOAD:
        out.update(extras(args, prob, X, dev, b))
    out_clocks = clocks.stop()
    if out is not None:
        out["clocks"] = out_clocks
        if not args.quick and wname == WORKLOAD:
            out["cpu_baseline"] = cpu_baseline(prob)
    return out


def _run_to_target(b, prob, X, opts, target, max_sweeps, chunk=25):
    """Sweeps in chunks (fits may come one sweep late inside a chunk) until the fit reaches
    target or max_sweeps; returns the history, the wall time per chunk and the final exact fit."""
    import torch
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, opts) as d:
        fits, walls = [], []
        torch.cuda.synchronize()
        while len(fits) < max_sweeps:
            n = min(chunk, max_sweeps - len(fits))
            t0 = time.perf_counter()
            f = d.sweep(n)
            torch.cuda.synchronize()
            walls.append((n, time.perf_counter() - t0))
            fits.extend(float(v) for v in f)
            if target is not None and max(fits) >= target:
                break
        st = d.stats()
        return np.array(fits), walls, d.fit_exact(), st


def _seconds_to(fits, walls, target):
    """First sweep whose fit reaches target, and the wall time up to it (within-chunk time
    prorated by sweeps)."""
    hit = np.nonzero(fits >= target)[0]
    if not len(hit):
        return None, None
    k = int(hit[0]) + 1
    t, done = 0.0, 0
    for n, w in walls:
        if done + n >= k:
            return k, t + w * (k - done) / n
        t += w
        done += n
    return k, t


def extras(args, prob, X, dev, b):
    """e2e through the host-buffer entry point; time to the fit target f* - 1e-6 (f*: the FP64 path,
    standard tree, no extrapolation, run to |delta fit| < 1e-12 or 2000 sweeps) and to the 1e-6
    stopping test for plain FP64 CP-ALS-QR, ALS-QR-BRE on both paths (rule, learned proposer) and the
    extrapolation ablation; the QR routes."""
    import torch
    res = {}
    # e2e: pinned host tensor -> device -> init -> sweeps -> factors back, one C call
    S = 30
    Xh = torch.from_numpy(prob.X).pin_memory()
    opts = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16 if args.prec == "split" else b.PREC_FP64,
                          extrap=b.EXTRAP_PAPER)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    calls = []
    for _ in range(2):  # the first call of this shape, then one served by the library's block cache
        torch.cuda.synchronize()
        e0.record()
        _, _, _, ns, _ = b.cp_als_qr_run_host(prob.dims, prob.R, Xh.numpy(), prob.A0, opts, tol=0.0, max_sweeps=S)
        e1.record()
        torch.cuda.synchronize()
        calls.append(e0.elapsed_time(e1))
    e2e_ms = calls[-1]
    fbytes = sum(d * prob.R * 8 for d in prob.dims) + prob.R * 8
    res["e2e"] = {"value": e2e_ms * 1e-3 / ns, "unit": "s/sweep", "h2d_bytes_per_step": prob.X.nbytes / ns,
                  "d2h_bytes_per_step": fbytes / ns + 24, "sweeps_per_call": ns,
                  "first_call_s_per_sweep": calls[0] * 1e-3 / ns,
                  "note": "one cp_als_qr_run_host call (H2D of X from pinned memory, init, sweeps, factors D2H) / "
                          "sweeps; the second call of the shape (the first, untimed warm-up, fills the library's "
                          "device block cache); first_call_s_per_sweep is the first"}
    # f*: the least-squares fit the method converges to, from the FP64 path
    o64 = b.make_options(tree=b.TREE_STANDARD, prec=b.PREC_FP64, extrap=b.EXTRAP_NONE)
    t0 = time.perf_counter()
    with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, o64) as d:
        conv, fstar_red, ns_star = d.fit(1e-12, 2000)
        fstar = d.fit_exact()
    res["fstar"] = {"value": fstar, "reduced_form": fstar_red, "sweeps": ns_star, "converged_1e-12": conv,
                    "seconds": time.perf_counter() - t0,
                    "how": "FP64 path, standard tree, no extrapolation, |delta fit| < 1e-12 or 2000 sweeps; "
                           "explicit residual of its final factors"}
    target = fstar - 1e-6
    from paper_2503_18759_gb300 import learn
    w = learn.load_weights()
    variants = [("fp64_plain_cpalsqr", b.PREC_FP64, b.TREE_NONE, b.EXTRAP_NONE, 0.0, 0.1, None, 600),
                ("fp64_bre_rule", b.PREC_FP64, b.TREE_RESTRUCTURED, b.EXTRAP_PAPER, 0.0, 0.1, None, 600),
                ("split_bre_rule", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_PAPER, 0.0, 0.1, None, 2000),
                ("split_bre_learned", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_LEARNED, 0.0, 0.1, w, 2000),
                ("split_br_none", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_NONE, 0.0, 0.1, None, 2000),
                # extrapolation ablation (eq. 18 is alpha = 1; a fixed beta against the rule)
                ("split_bre_fixed_5e-4", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 5e-4, 0.1, None, 2000),
                ("split_eq18_fixed_5e-4", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_FIXED, 5e-4, 1.0, None, 2000)]
    to_fstar, to_tol, traces = {}, {}, {}
    main = ("fp64_plain_cpalsqr", "fp64_bre_rule", "split_bre_rule", "split_bre_learned", "split_br_none")
    for name, prec, tree, ex, beta, alpha, wt, cap in variants:
        o = b.make_options(tree=tree, prec=prec, extrap=ex, beta_fixed=beta, alpha=alpha, mlp_weights=wt)
        fits, walls, fx, st = _run_to_target(b, prob, X, o, target, cap)
        traces[name] = (fits, walls)
        k, sec = _seconds_to(fits, walls, target)
        wall = sum(t for _, t in walls)
        to_fstar[name] = {"reached": k is not None, "sweeps": k, "seconds": sec, "sweeps_run": len(fits),
                          "s_per_sweep": wall / max(len(fits), 1), "best_fit": float(np.max(fits)),
                          "final_fit_exact": fx, "gap_to_fstar": fstar - float(np.max(fits)),
                          "proposals": int(st.proposals), "accepted": int(st.accepted), "judged": int(st.judged),
                          "lagged_fits": int(st.lagged_fits), "second_cholesky_pass": int(st.qr_second_pass),
                          "householder_qr": int(st.qr_fallbacks)}
        if name in ("fp64_plain_cpalsqr", "fp64_bre_rule", "split_bre_rule", "split_bre_learned", "split_br_none"):
            with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, o) as d:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                conv, f, ns = d.fit(1e-6, cap)
                torch.cuda.synchronize()
                to_tol[name] = {"seconds": time.perf_counter() - t0, "sweeps": ns, "converged": conv, "fit": f,
                                "fit_exact": d.fit_exact()}
    # secondary figure: the lowest best fit any of the main variants reached (each run stops at f* - 1e-6
    # or its sweep cap), and the sweeps and seconds each takes to reach it
    common = min(float(np.max(traces[n][0])) for n in main)
    to_common = {}
    for n in main:
        k, sec = _seconds_to(traces[n][0], traces[n][1], common)
        to_common[n] = {"sweeps": k, "seconds": sec}
    res["time_to_fit"] = {"target": "f*-1e-6", "f*": fstar, "variants": to_fstar,
                          "common_target": {"fit": common, "note": "lowest best fit of the main variants",
                                            "variants": to_common}}
    res["time_to_tol_1e-6"] = to_tol
    # the same split-precision sweeps with every QR on the Householder route (the paper's plain
    # form; cpqr_options.qr_route), against the default guarded Gram route
    routes = {}
    for name, route in (("gram", b.QR_GRAM), ("householder", b.QR_HOUSEHOLDER)):
        o = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER, qr_route=route)
        with b.Decomposition(prob.dims, prob.R, X.data_ptr(), False, prob.A0, o) as d:
            d.sweep(5)
            torch.cuda.synchronize()
            e0.record()
            f = d.sweep(20)
            e1.record()
            torch.cuda.synchronize()
            routes[name] = {"ms_per_sweep": e0.elapsed_time(e1) / 20, "fit_after_25": float(f[-1]) if len(f) else None,
                            "qr_fallbacks": int(d.stats().qr_fallbacks)}
    res["qr_routes"] = routes
    res["other_workloads"] = other_workloads(b, dev)
    res["e1_shapes"] = e1_shapes(b, dev)
    res["high_rank"] = high_rank(b, dev)
    return res


def high_rank(b, dev, sweeps=5):
    """The high-rank regime (Table 7: 500^3 at R = 75 and 150, 600^3 at R = 175) on the split path:
    ms per sweep, and the first-level TTM's device time (per-launch CUDA events) with its
    tensor-core rates.  useful = 2 I^N R flops per full TTM; issued = the four bf16 products the
    MMAs execute, 8 Rp flops per element of the tile-padded tensor.  Fractions are of the measured
    bf16 peak (the MMA pipe's ceiling for these operands)."""
    import torch
    from paper_2503_18759_gb300 import inputs
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
        kind = "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    out = {}
    for dims, R in (([500] * 3, 75), ([500] * 3, 150), ([600] * 3, 175)):
        name = "x".join(str(d) for d in dims) + f"_r{R}"
        prob = inputs.make_problem_device(name, dims, R, seed=9, c=0.5, eta=1e-3, device=str(dev))
        o = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with b.Decomposition(prob.dims, prob.R, prob.X.data_ptr(), False, prob.A0, o) as d:
            d.sweep(2)
            torch.cuda.synchronize()
            e0.record()
            f = d.sweep(sweeps)
            e1.record()
            torch.cuda.synchronize()
            d.set_timing(True)
            d.sweep(sweeps)
            st = d.stats()
            d.set_timing(False)
        n_full = st.n_bucket[0]
        full_ms = st.ms_bucket[0] / max(n_full, 1)
        I = dims[0]
        Rp = (R + 15) // 16 * 16
        useful = 2.0 * I ** 3 * R
        padded = I * I * (-(-I // 64) * 64)  # the contiguous mode padded to whole 64-wide blocks (MN-major)
        issued = 8.0 * Rp * padded
        tf_u = useful / (full_ms * 1e-3) / 1e12 if n_full else None
        tf_i = issued / (full_ms * 1e-3) / 1e12 if n_full else None
        out[name] = {"ms_per_sweep": e0.elapsed_time(e1) / sweeps, "fit_last": float(f[-1]),
                     "ttm_full_ms": full_ms, "ttm_full_launches": int(n_full),
                     "useful_tflops": tf_u, "issued_tflops": tf_i,
                     "useful_frac": tf_u / peak if tf_u else None, "issued_frac": tf_i / peak if tf_i else None,
                     "hbm_gbs": (I ** 3 * 4 + I * I * R * 4) / (full_ms * 1e-3) / 1e9 if n_full else None,
                     "buckets_ms_per_sweep": {nm: st.ms_bucket[i] / sweeps for i, nm in enumerate(b.BUCKETS)},
                     "peak_tflops": peak, "peak_kind": f"{kind} bf16 dense (burst)"}
        del prob
        torch.cuda.empty_cache()
    return out


E1_SHAPES = [[700] * 3, [150] * 4, [50] * 5, [25] * 6]


def e1_shapes(b, dev, ranks=(8, 16, 32), sweeps=10):
    """The paper's per-iteration breakdown over orders 3 to 6 (700^3, 150^4, 50^5, 25^6) and rank:
    split-precision ALS-QR-BRE, ms per sweep (CUDA events, after 3 warm-up sweeps) and the device
    time per bucket (per-launch events, a second run of the same sweeps).  Seeded synthetic tensors:
    N(0,1) rank-R factors, 1e-3 noise."""
    import torch
    from paper_2503_18759_gb300 import inputs
    out = {}
    for dims in E1_SHAPES:
        for R in ranks:
            if R > dims[0]:
                continue
            name = "x".join(str(d) for d in dims) + f"_r{R}"
            prob = inputs.make_problem_device(name, dims, R, seed=5, c=None, eta=1e-3, device=str(dev))
            o = b.make_options(tree=b.TREE_RESTRUCTURED, prec=b.PREC_SPLIT_BF16, extrap=b.EXTRAP_PAPER)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with b.Decomposition(prob.dims, prob.R, prob.X.data_ptr(), False, prob.A0, o) as d:
                d.sweep(3)
                torch.cuda.synchronize()
                e0.record()
                d.sweep(sweeps)
                e1.record()
                torch.cuda.synchronize()
                d.set_timing(True)
                d.sweep(sweeps)
                st = d.stats()
                d.set_timing(False)
            out[name] = {"ms_per_sweep": e0.elapsed_time(e1) / sweeps,
                         "buckets_ms_per_sweep": {nm: st.ms_bucket[i] / sweeps for i, nm in enumerate(b.BUCKETS)},
                         "qr_fallbacks": int(st.qr_fallbacks)}
            del prob
            torch.cuda.empty_cache()
    return out


def other_workloads(b, dev):
    """ms per sweep of the other named workloads (after warm-up sweeps, CUDA events), and the
    restructured / standard TTM flop ratio over the first three sweeps and over 50."""
    import torch
    from paper_2503_18759_gb300 import inputs
    out = {}
    plans = [("cube60_r5_f64", b.PREC_FP64, b.TREE_STANDARD, b.EXTRAP_NONE, 50),
             ("hyper128_r24_c08", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_PAPER, 30),
             ("order5_48_r16", b.PREC_SPLIT_BF16, b.TREE_RESTRUCTURED, b.EXTRAP_PAPER, 30),
             ("order5_48_r16", b.PREC_SPLIT_BF16, b.TREE_STANDARD, b.EXTRAP_PAPER, 30)]
    for name, prec, tree, ex, sweeps in plans:
        cfg = dict(inputs.WORKLOADS[name])
        if cfg.get("dtype") == np.float64:
            prob = inputs.workload(name, seed=0)
            X = torch.from_numpy(prob.X).to(dev)
            x64 = True
        else:
            prob = inputs.make_problem_device(name, cfg.pop("dims"), cfg.pop("R"), seed=0, c=cfg.get("c"),
                                              eta=cfg.get("eta", 0.0), device=str(dev))
            X, x64 = prob.X, False
        o = b.make_options(tree=tree, prec=prec, extrap=ex)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with b.Decomposition(prob.dims, prob.R, X.data_ptr(), x64, prob.A0, o) as d:
            d.sweep(5)
            torch.cuda.synchronize()
            e0.record()
            f = d.sweep(sweeps)
            e1.record()
            torch.cuda.synchronize()
            st = d.stats()
        tname = {b.TREE_STANDARD: "standard", b.TREE_RESTRUCTURED: "restructured"}[tree]
        key = f"{name}_{tname}"
        out[key] = {"ms_per_sweep": e0.elapsed_time(e1) / sweeps, "sweeps_timed": sweeps,
                    "precision": "fp64" if prec == b.PREC_FP64 else "split", "fit_last": float(f[-1]),
                    "ttm_flops_per_sweep_avg": st.ttm_flops / (5 + sweeps)}
        del X
    for name in ("order5_48_r16", "hyper128_r24_c08"):
        dims = inputs.WORKLOADS[name]["dims"]
        R = inputs.WORKLOADS[name]["R"]
        fl = {t: [b.cp_als_qr_schedule(dims, R, t, k)[1] for k in (3, 50)] for t in (b.TREE_STANDARD, b.TREE_RESTRUCTURED)}
        out[f"{name}_ttm_flop_ratio"] = {"first_3_sweeps": fl[b.TREE_RESTRUCTURED][0] / fl[b.TREE_STANDARD][0],
                                         "first_50_sweeps": fl[b.TREE_RESTRUCTURED][1] / fl[b.TREE_STANDARD][1]}
    return out


def run_kernel(args):
    """One library kernel on a seeded case, timed with CUDA events (also the command the ncu
    summaries capture):
      --kernel ttm_tc   --shape P K S R   split-bf16 tensor-core TTM of the middle mode of P x K x S
      --kernel ttm_f32  --shape P K S R   FP32 CUDA-core TTM
      --kernel house_qr --shape M R       FP64 cluster Householder QR
      --kernel krp_qr   --shape m R       QR of the Khatri-Rao product of m triangles"""
    import torch
    from paper_2503_18759_gb300 import binding as b
    from paper_2503_18759_gb300 import build
    build.build()
    b.lib()
    g = np.random.default_rng(0)
    dev = "cuda"
    kind, shp = args.kernel, [int(v) for v in args.shape]
    alg = None
    if kind in ("ttm_tc", "ttm_f32"):
        P, K, S, R = shp
        X = torch.from_numpy(g.standard_normal((P, K, S)).astype(np.float32)).to(dev)
        Qn = np.linalg.qr(g.standard_normal((K, R)))[0]
        Q = torch.from_numpy(Qn if kind == "ttm_tc" else Qn.astype(np.float32)).to(dev)
        out = torch.empty((P, R, S), dtype=torch.float32, device=dev)
        dt = b.TTM_SPLIT_BF16 if kind == "ttm_tc" else b.TTM_F32
        run = lambda: b.cpqr_ttm(X.data_ptr(), [P, K, S], 1, Q.data_ptr(), R, out.data_ptr(), dt)
        alg = {"bytes": 4 * P * K * S + 4 * P * R * S, "note": "the entry point also splits X and Q first"}
    elif kind == "house_qr":
        M, R = shp
        A = torch.from_numpy(g.standard_normal((M, R))).to(dev)
        Q = torch.empty((M, R), dtype=torch.float64, device=dev)
        Rm = torch.empty((R, R), dtype=torch.float64, device=dev)
        run = lambda: b.cpqr_house_qr(A.data_ptr(), M, R, Q.data_ptr(), Rm.data_ptr())
    elif kind == "krp_qr":
        m, R = shp
        tri = [np.linalg.qr(g.standard_normal((R + 8, R)))[1] for _ in range(m)]
        tri = [t * np.sign(np.diag(t))[:, None] for t in tri]
        Rs = torch.from_numpy(np.stack(tri)).to(dev)
        Q0 = torch.empty((R ** m, R), dtype=torch.float64, device=dev)
        R0 = torch.empty((R, R), dtype=torch.float64, device=dev)
        run = lambda: b.cpqr_krp_qr(Rs.data_ptr(), m, R, Q0.data_ptr(), R0.data_ptr())
    else:
        raise SystemExit(run_kernel.__doc__)
    for _ in range(max(args.warmup, 1)):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    return {"kernel": kind, "shape": shp, "ms_per_call": ms, "calls": args.steps, "algorithmic": alg,
            "note": "CUDA events around whole entry-point calls (their own allocations and copies included)"}


_ORACLE_SWEEP = """
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import cpqr_oracle as o
from paper_2503_18759_gb300 import inputs
prob = inputs.workload({w!r}, seed=0)
stamps = [time.perf_counter()]
o.cp_als_qr(prob.X, prob.R, prob.A0, tree=o.TREE_RESTRUCTURED, extrapolate=True, max_sweeps={n},
            on_sweep=lambda k, f: stamps.append(time.perf_counter()))
print(json.dumps(list(np.diff(stamps))))
"""


def _oracle_sweeps_subprocess(threads, sweeps):
    """Oracle sweep times in a fresh process whose BLAS uses `threads` threads."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    code = _ORACLE_SWEEP.format(root=ROOT, w=WORKLOAD, n=sweeps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(prob):
    """The oracle as it stands on the host cores: all cores (BLAS threads) and one core."""
    cores = os.cpu_count()
    from oracle import cpqr_oracle as o
    t_all = oracle_sweep_times(prob, o.TREE_RESTRUCTURED, 4)
    t_one = _oracle_sweeps_subprocess(1, 2)
    one = {"value": float(np.mean(t_one[1:])), "unit": "s/sweep", "cores": 1} if t_one else None
    return {"value": float(np.mean(t_all[1:])), "unit": "s/sweep", "cores": cores, "kind": "oracle",
            "sample": "3 full-size FP64 oracle sweeps (400^3, R=32) after its first sweep, numpy/BLAS on all host "
                      "cores; one_core: 1 sweep after the first with every BLAS limited to one thread",
            "one_core": one}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="split", choices=["split", "fp64"])
    ap.add_argument("--quick", action="store_true", help="skip e2e, time-to-fit and the CPU baseline")
    ap.add_argument("--workload", default=WORKLOAD, help="named workload of inputs.WORKLOADS (default: the bench "
                    "line's); others print timing and buckets only")
    ap.add_argument("--tree", default="restructured", choices=["restructured", "standard", "none"],
                    help="dimension tree of the extra workloads (the bench line is always restructured)")
    ap.add_argument("--kernel", default=None, help="time one library kernel instead (see run_kernel)")
    ap.add_argument("--shape", nargs="*", default=[], help="sizes of the --kernel case")
    ap.add_argument("--metrics-jsonl", default=None,
                    help="append one JSON line per sweep of the bench context (fit, beta) to this file")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed sweeps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.kernel:
        print(json.dumps(run_kernel(args)))
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None and rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
