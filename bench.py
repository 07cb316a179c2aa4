#!/usr/bin/env python
"""Benchmark of deflated MG-MLMC on GB300: MG-MLMC samples/s on the 1024x1024
Wilson-Schwinger workload ("Scale": beta = 5, near-critical m0, a 3-term
multigrid telescoping sum whose solver hierarchy continues three levels below
it, 512 deflated triplets of the level-3 operator, blocks of Z2 vectors sized to
HBM by the library's autotuner), every solve to FP64 relative residual 1e-12.

One step = one block of N samples on every term of the telescoping sum (two
multigrid-preconditioned solves per difference-level sample, one solve plus the
deflation projections for the last term, FP64 sample assembly).  The headline
run solves every block in FP64 by iterative refinement around an FP32 multigrid
cycle with BF16 tensor-core smoothers, coarsest solve and deflation projections.
Beside it: the end-to-end rate through the C ABI with host probes, the time to
tr(D^-1) at relative error 1e-4 (the paper's tolerance) measured for the mixed
path and projected for the all-FP64 batched and the plain FP64 single-rhs paths
from their measured per-sample costs, the fine stencil's HBM bandwidth, a
serving run (trace requests of mixed lattice sizes, p50/p99 time to trace) and
the CPU oracle on the largest workload its direct solves can bound.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  With N > 1 (torchrun) every rank runs an independent
replica on its own GPU (the estimator's samples are independent; no data-path
collective); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

METRIC = "MG-MLMC samples/s"
UNIT = "samples/s"
L2_BYTES = 129e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="schwinger-1024x1024")
    ap.add_argument("--no-tune", action="store_true", help="keep the workload's block width (no autotuner)")
    ap.add_argument("--k", type=int, default=-1,
                    help="deflated triplets (default: the workload's; 0: no deflation, for small profiler cases)")
    ap.add_argument("--fp64-block", type=int, default=32, help="right-hand sides per block of the FP64 comparison")
    ap.add_argument("--fp64-deflation", action="store_true",
                    help="deflate the FP64 comparison too (its eigensolver runs in FP64)")
    ap.add_argument("--cpu-workload", default="schwinger-128x128",
                    help="workload of the oracle CPU baseline (its direct sparse LU must factor the levels)")
    ap.add_argument("--precision", type=int, default=16, choices=[64, 32, 16],
                    help="multigrid precision of the headline run: 32 = FP32 multigrid + BF16 tensor-core "
                         "coarsest solve inside FP64 iterative refinement; 16 = as 32 with the coarse "
                         "smoother's block stencil on the tensor cores in BF16; 64 = all-FP64 (the outer "
                         "solve, its residuals and every sample are FP64 in all three)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the comparison run in the other precision and the single-rhs FP64 run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sequential", action="store_true",
                    help="one context, terms one after another (default: the terms of a step at once, "
                         "one context and CUDA stream per term, via mgmlmc_estimate_concurrent)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--ttt-tol", type=float, default=1e-4,
                    help="relative error of the time-to-trace run (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--block-rhs", type=int, default=0,
                    help="override the workload's right-hand sides per block (smaller ncu captures)")
    ap.add_argument("--restart", type=int, default=0,
                    help="FGMRES restart length without the autotuner (0: the library default)")
    ap.add_argument("--nvtx", action="store_true",
                    help="mark the timed regions with NVTX ranges timed_f64 / timed_mixed / timed_e2e")
    ap.add_argument("--single-rhs-samples", type=int, default=1,
                    help="samples per term of the plain FP64 single-rhs comparison (0 = skip)")
    ap.add_argument("--serving-requests", type=int, default=6,
                    help="requests per phase of the serving run (0 = skip; 1 GPU only)")
    ap.add_argument("--serving-slots", type=int, default=4, help="requests admitted at once by the server")
    ap.add_argument("--serving-load", type=float, default=0.8,
                    help="Poisson arrival rate of the second phase, as a fraction of the saturated rate")
    ap.add_argument("--serving-tol", type=float, default=1e-3, help="relative error asked by each request")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
def dist_setup(args, backend="nccl"):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device="cuda"):
    """The slowest rank's time: every replica's work counts, so the job ends with it."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(w, rank):
    """Noise seed of a replica: each rank draws its own independent Z2 stream."""
    return w.noise_seed + 7919 * rank


def job_throughput(samples_per_rank, ws, seconds):
    """Whole-job samples per second: all ranks' samples over the slowest rank's time."""
    return samples_per_rank * ws / seconds


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
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
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------- peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def source_sha(fn):
    path = os.path.join(ROOT, "paper_2211_15383_gb300", "csrc", fn)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] if os.path.exists(path) else None


def ncu_traffic(kclass, impl_bytes_per_launch=None):
    """DRAM bytes per launch of a kernel class from a committed ncu summary, if the
    kernel's source file has not changed since the counters were taken.  A class whose
    per-launch work varies with the schedule (Gram-Schmidt: the Arnoldi index) stores
    its measured traffic per implementation byte, scaled here to this run's launches."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get("classes", {}).get(kclass)
    if e is None or source_sha(e.get("source", "")) != e.get("source_sha"):
        return None
    if e.get("per_implementation_byte") and impl_bytes_per_launch:
        return e["per_implementation_byte"] * impl_bytes_per_launch
    return e.get("dram_bytes_per_launch")


def roofline(report, peaks, fp64_peak, fp32_peak, cls=None):
    """Roofline of a kernel class (default: the one with the largest device time).

    The bound follows the class's precision and arithmetic intensity: a class is
    compute-bound when its intensity exceeds the ridge point (peak / HBM bandwidth)
    of its unit, else HBM-bound.  BF16 classes run on the tensor cores (peak:
    measured sustained cuBLAS BF16, the kernels run inside a long step); FP64 and
    FP32 classes on the FMA pipes (measured FMA peaks).
    """
    if cls is None:
        cls = max(report.items(), key=lambda kv: kv[1]["ms"])[0]
    st = report[cls]
    per_launch_s = st["ms"] * 1e-3 / st["count"]
    prec = cls.split(".")[-1]
    bytes_l = st["bytes"] / st["count"]
    flops_l = st["flops"] / st["count"]
    hbm = peaks["hbm_gbs"] * 1e9
    if prec == "bf16" and flops_l / max(bytes_l, 1.0) > (peaks.get("bf16_tflops_sustained") or
                                                            peaks["bf16_tflops"]) * 1e12 / hbm:
        peak = peaks.get("bf16_tflops_sustained") or peaks["bf16_tflops"]
        ach = flops_l / per_launch_s / 1e12
        out = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
               "peak_source": f"{peaks['source']} cuBLAS BF16 sustained"}
    elif prec == "bf16":
        ach = bytes_l / per_launch_s / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": ach / peaks["hbm_gbs"], "peak_source": peaks["source"]}
    else:
        alu = fp64_peak if prec == "f64" else fp32_peak
        if flops_l / max(bytes_l, 1.0) > alu / hbm:
            ach = flops_l / per_launch_s / 1e12
            out = {"bound": "alu", "achieved": ach, "peak": alu / 1e12, "unit": "TFLOP/s", "frac": ach * 1e12 / alu,
                   "peak_source": f"measured {prec.upper()} FMA throughput (mgmlmc_fma_peak)"}
        else:
            ach = bytes_l / per_launch_s / 1e9
            out = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": ach / peaks["hbm_gbs"], "peak_source": peaks["source"]}
    impl_l = st.get("impl_bytes", st["bytes"]) / st["count"]
    out.update({"kernel": cls, "launches": st["count"], "avg_launch_us": per_launch_s * 1e6,
                "algorithmic_bytes_per_launch": bytes_l, "algorithmic_flops_per_launch": flops_l,
                "implementation_bytes_per_launch": impl_l,
                "implementation_GB_per_s": impl_l / per_launch_s / 1e9,
                "traffic": ncu_traffic(cls, impl_l), "share_of_profiled_time":
                    st["ms"] / sum(v["ms"] for v in report.values())})
    return out


def class_summary(report, top=8):
    tot = sum(v["ms"] for v in report.values())
    items = sorted(report.items(), key=lambda kv: -kv[1]["ms"])[:top]
    return {k: {"ms": round(v["ms"], 3), "share": round(v["ms"] / tot, 4), "launches": v["count"],
                "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] else None,
                "TFLOP/s": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 3) if v["ms"] else None}
            for k, v in items}


# ----------------------------------------------------------------------------- GPU runs
_GAUGE = {}


def gauge_of(w):
    """The workload's gauge field, generated once per process (host input data)."""
    if w.name not in _GAUGE:
        _GAUGE[w.name] = w.gauge()
    return _GAUGE[w.name]


def make_ctx(pkg, w, prec, nrhs=None, restart=None, k=None, tune=False, test_vectors=None):
    """Context with the workload's hierarchy (and deflation); optionally autotuned.
    test_vectors: another context's test vectors, taken as they are (the same P and D_l
    without running this precision's setup)."""
    t0 = time.time()
    opts = {"mg_precision": prec, "max_block_rhs": nrhs or w.nrhs, "kcycle_iters": w.kcycle}
    if restart:
        opts["fgmres_restart"] = restart
    ctx = pkg.Context(**opts)
    ctx.set_gauge(gauge_of(w))
    ctx.set_mass(w.m0)
    t1 = time.time()
    if test_vectors is None:
        ctx.set_hierarchy(w.agg, w.nvec, w.start_vectors(), setup_iters=w.setup_iters, setup_tol=1e-12)
    else:
        ctx.set_hierarchy(w.agg, w.nvec, test_vectors, setup_iters=0)
    if w.skip:
        ctx.set_terms(list(w.skip))
    t2 = time.time()
    kk = w.k if k is None else k
    defl_converged = True
    if kk:
        try:
            ctx.compute_deflation(kk, w.defl_tol, w.defl_iters)
        except pkg.MgmlmcError as e:          # not converged to defl_tol: the vectors are kept
            if e.code != -3:
                raise
            defl_converged = False
    t3 = time.time()
    setup = {"gauge_upload_s": t1 - t0, "hierarchy_s": t2 - t1, "deflation_s": t3 - t2,
             "deflation": {"k": kk, "tol": w.defl_tol, "max_iters": w.defl_iters, "converged": defl_converged}}
    tuned = None
    if tune:
        t4 = time.time()
        tuned = ctx.autotune(max_trials=8)
        setup["autotune_s"] = time.time() - t4
    return ctx, setup, tuned


def run_steps(ctx, nterms, N, first_step, K, seed):
    """K steps of one block of N samples on every term (one context)."""
    for k in range(K):
        for t in range(nterms):
            ctx.estimate_level(t, (first_step + k) * N, N, seed, samples=False)


def concurrent_ok(w):
    """Terms at once on context copies only where the copies' work space is small."""
    return w.n1 <= (1 << 16)


def timed_region(torch, ws, fn, name=None):
    barrier(ws)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if name:
        torch.cuda.nvtx.range_push(name)
    e0.record(s)
    fn()
    e1.record(s)
    torch.cuda.synchronize()
    if name:
        torch.cuda.nvtx.range_pop()
    barrier(ws)
    return max_over_ranks(e0.elapsed_time(e1) * 1e-3, ws)


def probe_blocks(seed, n_of, N, K, torch):
    """K steps of pinned host int8 +-1 probe blocks [N][n_t] per term (seeded host data)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(K):
        per = []
        for n in n_of:
            arr = torch.empty((N, n), dtype=torch.int8, pin_memory=True)
            a = arr.numpy()
            a[:] = rng.integers(0, 2, size=(N, n), dtype=np.int8)
            a *= 2
            a -= 1
            per.append(a)
        out.append(per)
    return out


def per_term_rate(ctx, nterms, N, first, seed, torch):
    """Seconds per sample of each term on one block of N samples (device time)."""
    out = []
    for t in range(nterms):
        torch.cuda.synchronize()
        _, st = ctx.estimate_level(t, first, N, seed, samples=False)
        out.append(st["seconds"] / N)
    return out


def gpu_arm(args, rank, ws, local):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_15383_gb300 as pkg

    w = inputs.workload(args.workload)
    if args.block_rhs or args.k >= 0:
        import dataclasses
        w = dataclasses.replace(w, nrhs=args.block_rhs or w.nrhs, k=w.k if args.k < 0 else args.k)
    peaks = measured_peaks()
    fp64_peak = pkg.fma_peak(64)
    fp32_peak = pkg.fma_peak(32)
    t_gauge = time.time()
    gauge_of(w)
    gauge_gen_s = time.time() - t_gauge
    ctx, setup, tuned = make_ctx(pkg, w, args.precision, restart=args.restart or None,
                                 tune=not args.block_rhs and not args.no_tune and not args.restart)
    setup["gauge_generation_s"] = gauge_gen_s
    N = tuned["block_rhs"] if tuned else w.nrhs
    nterms, levels = ctx.num_terms()
    K, W = args.steps, args.warmup
    seed = replica_seed(w, rank)
    # small lattices: the terms of a step at once, one context (device copy) and CUDA
    # stream per term; large ones: one context, the terms one after another (each
    # context would hold its own Krylov work space, and the blocks fill the GPU anyway)
    ctxs = [ctx]
    helper_setup_s = 0.0
    if not args.sequential and concurrent_ok(w):
        t0 = time.time()
        for t in range(1, nterms):
            with torch.cuda.stream(torch.cuda.Stream()):
                ctxs.append(pkg.Context(copy_of=ctx))
        helper_setup_s = time.time() - t0

    def steps(first, count, probes=None, outs=None):
        for k in range(first, first + count):
            if len(ctxs) > 1:
                pkg.estimate_concurrent(ctxs, list(range(nterms)), k * N, N, seed,
                                        probes=None if probes is None else probes[k - first],
                                        samples=outs is not None, out=outs)
            elif probes is None:
                run_steps(ctx, nterms, N, k, 1, seed)
            else:
                for t in range(nterms):
                    ctx.estimate_level_probes(t, probes[k - first][t], out=outs[t])

    steps(0, W)                                                             # warm-up
    if len(ctxs) > 1:
        run_steps(ctx, nterms, N, 0, 1, seed)
    ctx.profile(False, reset=True)
    clk = Clocks(local)
    clk.start()
    tag = "timed_f64" if args.precision == 64 else "timed_mixed"
    sec = timed_region(torch, ws, lambda: steps(W, K), tag if args.nvtx else None)
    clocks = clk.stop()
    launches = int(ctx.profile_report().get("__launches__", {}).get("count", 0))
    sec_seq = timed_region(torch, ws, lambda: run_steps(ctx, nterms, N, W + K, K, seed)) if len(ctxs) > 1 else sec
    # K steps on one context with per-kernel-class CUDA events (roofline, class shares)
    # per-class profile and end-to-end pass over min(K, 3) steps: rates, so a few steps do
    Kp = min(K, 3)
    ctx.profile(True, reset=True)
    sec_prof = timed_region(torch, ws, lambda: run_steps(ctx, nterms, N, W + 2 * K, Kp, seed))
    ctx.profile(False)
    report = ctx.profile_report()
    report.pop("__launches__", None)
    samples = K * nterms * N * ws
    value = job_throughput(K * nterms * N, ws, sec)
    dims = w.level_dims()
    n_of = [dims[lv - 1][0] * dims[lv - 1][1] * dims[lv - 1][2] for lv in levels]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": sec / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == 64 else "f64+f32+bf16",
           "precision": ("all FP64" if args.precision == 64 else
                         "FP64 iterative refinement (FP64 residuals, solution updates and sample sums; every "
                         "solve to relative residual 1e-12 in FP64) around an FP32 multigrid-preconditioned "
                         "FGMRES cycle with a BF16 tensor-core coarsest solve" +
                         (", BF16 tensor-core coarse smoother stencils and BF16 tensor-core deflation "
                          "projections (FP32 accumulation; the deflated trace over the same rounded factors "
                          "in FP64)" if args.precision == 16 else "")),
           "data": f"synthetic: seeded Metropolis U(1) gauge field beta={w.beta} {w.Lx}x{w.Lt}, "
                   f"counter-based Z2 noise",
           "config": {"workload": w.name, "lattice": f"{w.Lx}x{w.Lt}", "m0": w.m0, "beta": w.beta,
                      "levels": w.nlevels, "sum_levels": w.nterms,
                      "level_unknowns": n_of + [d[0] * d[1] * d[2] for d in dims[w.nterms:]],
                      "agg": [list(a) for a in w.agg], "nvec": list(w.nvec),
                      "deflated_triplets": w.k, "block_rhs": N, "terms": nterms,
                      "fgmres_restart": tuned["fgmres_restart"] if tuned else ctx.options.fgmres_restart,
                      "nu_post": tuned["nu_post"] if tuned else ctx.options.nu_post,
                      "kcycle_iters": tuned["kcycle_iters"] if tuned else ctx.options.kcycle_iters,
                      "autotune": tuned,
                      "solve_tol": 1e-12, "mg_precision": args.precision,
                      "l2": "inputs exceed L2: one FP64 fine-level block is "
                            f"{w.n1 * N * 16 / 1e6:.0f} MB > 129 MB",
                      "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
           "setup": setup, "clocks": clocks, "ms_per_step_profiled": sec_prof / Kp * 1e3,
           "roofline": roofline(report, peaks, fp64_peak, fp32_peak),
           "roofline_next": [roofline(report, peaks, fp64_peak, fp32_peak, k) for k, _ in
                             sorted(report.items(), key=lambda kv: -kv[1]["ms"])[1:5]],
           "kernel_classes": class_summary(report),
           "profiled_kernel_ms_per_step": sum(v["ms"] for v in report.values()) / Kp,
           "terms_concurrent": len(ctxs) > 1,
           "context_copies_s": helper_setup_s,
           "peaks": {"fp64_fma_tflops": fp64_peak / 1e12, "fp32_fma_tflops": fp32_peak / 1e12,
                     "hbm_gbs": peaks["hbm_gbs"], "hbm_source": peaks["source"]},
           "iters": {t: sum(c.get_stats(t)["iters"] for c in ctxs) for t in range(nterms)}}
    if len(ctxs) > 1:
        out["sequential"] = {"value": job_throughput(K * nterms * N, ws, sec_seq), "unit": UNIT,
                             "ms_per_step": sec_seq / K * 1e3,
                             "what": "same steps, terms one after another on one context and stream"}
    out["gpu_launches"] = launches
    live, peak = ctx.memory()
    out["device_peak_gb"] = peak / 1e9
    # end-to-end through the public C ABI with host probe vectors and host samples
    if not args.no_e2e:
        probes = probe_blocks(9000 + rank, n_of, N, Kp, torch)
        outs = [torch.empty((N, 2), dtype=torch.float64, pin_memory=True).numpy().view(np.complex128)
                .reshape(-1) for _ in range(nterms)]
        sec_e2e = timed_region(torch, ws, lambda: steps(0, Kp, probes, outs), "timed_e2e" if args.nvtx else None)
        out["e2e"] = {"value": Kp * nterms * N * ws / sec_e2e, "unit": UNIT, "steps": Kp,
                      "h2d_bytes_per_step": int(sum(N * n for n in n_of)),
                      "d2h_bytes_per_step": int(nterms * N * 16),
                      "path": ("mgmlmc_estimate_concurrent" if len(ctxs) > 1 else "mgmlmc_estimate_level_probes")
                              + ": pinned host int8 probes in, host samples out, copies inside the timed region"}
    # time to tr(D^-1) at a fixed relative error (the MLMC loop of the library)
    ttt = None
    if args.ttt_tol > 0:
        t0 = time.time()
        res = ctx.estimate_trace(args.ttt_tol, 10 ** 7, seed + 1)
        tt = time.time() - t0
        # the library's setup of this problem: gauge upload, hierarchy, deflation and the
        # autotuner; the host synthesis of the gauge field is input data, not counted
        setup_s = sum(v for k_, v in setup.items() if k_.endswith("_s") and k_ != "gauge_generation_s")
        tune_s = setup.get("autotune_s", 0.0)
        ttt = {"rel_tol": args.ttt_tol, "samples_per_term": [t["nsamples"] for t in res["terms"]]}
        out["time_to_trace"] = {
            "rel_tol": args.ttt_tol,
            "mixed": {"seconds_excl_setup": tt, "seconds_incl_setup": tt + setup_s,
                      "seconds_incl_setup_excl_autotune": tt + setup_s - tune_s,
                      "trace": [res["trace"].real, res["trace"].imag], "rel_err": res["rel_err"],
                      "converged": bool(res["converged"]), "samples_per_term": ttt["samples_per_term"],
                      "variance_per_term": [t["variance"] for t in res["terms"]], "what": "measured"}}
        if len(ctxs) > 1:
            t0 = time.time()
            resc = pkg.estimate_trace_concurrent(ctxs, args.ttt_tol, 10 ** 7, seed + 1)
            out["time_to_trace"]["mixed_concurrent_terms"] = {
                "seconds_excl_setup": time.time() - t0, "rel_err": resc["rel_err"],
                "samples_per_term": [t["nsamples"] for t in resc["terms"]]}
    for c_ in ctxs[1:]:
        c_.close()
    # the FP64 paths on the same workload: the all-FP64 batched solve and the plain FP64
    # single-rhs solve, per-sample device cost of every term; with the identical samples
    # (same noise, same estimator) their time to trace follows from the sample counts of
    # the MLMC run above
    if not args.no_mixed:
        head_samples = [ctx.estimate_level(t, 0, min(N, 32), seed)[0] for t in range(nterms)]
        mixed_cost = per_term_rate(ctx, nterms, N, 10 ** 6, seed, torch)
        tv = [ctx.get_test_vectors(l + 1, w.nvec[l]) for l in range(len(w.agg))]
        ctx.close()
        torch.cuda.empty_cache()
        n64 = min(N, args.fp64_block)
        # the FP64 contexts take the mixed context's test vectors: the same hierarchy (P,
        # D_l), so their samples are the headline's, and no FP64 setup iteration runs
        octx, osetup, _ = make_ctx(pkg, w, 64, nrhs=n64, restart=16, k=w.k if args.fp64_deflation else 0,
                                   test_vectors=tv)
        oth_samples = [octx.estimate_level(t, 0, min(N, 32), seed)[0] for t in range(nterms)]
        errs = []
        for t in range(nterms):
            g, r = head_samples[t], oth_samples[t]
            if w.k and t == nterms - 1 and not args.fp64_deflation:
                continue                       # the FP64 run here is undeflated on the last term
            errs.append(float(np.max(np.abs(g - r) / np.maximum(np.abs(r), np.sqrt(np.mean(np.abs(r) ** 2))))))
        out["max_rel_sample_error_mixed_vs_f64_per_term"] = errs
        octx.reset_stats()
        octx.profile(True, reset=True)
        osec = timed_region(torch, ws, lambda: run_steps(octx, nterms, n64, 2, 1, seed))
        octx.profile(False)
        orep = octx.profile_report()
        orep.pop("__launches__", None)
        f64_cost = [octx.get_stats(t)["seconds"] / octx.get_stats(t)["nsamples"] for t in range(nterms)]
        out["fp64"] = {"value": nterms * n64 * ws / osec, "unit": UNIT, "block_rhs": n64,
                       "ms_per_step": osec * 1e3, "headline_speedup_over_this": value / (nterms * n64 * ws / osec),
                       "setup": osetup, "seconds_per_sample_per_term": f64_cost,
                       "roofline": roofline(orep, peaks, fp64_peak, fp32_peak),
                       "kernel_classes": class_summary(orep)}
        single_cost = None
        if args.single_rhs_samples > 0:
            # the same FP64 context with one right-hand side per solve
            sctx = octx
            sctx.set_options(max_block_rhs=1)
            ns = args.single_rhs_samples
            sctx.estimate_level(0, 10 ** 6, 1, seed, samples=False)
            sctx.reset_stats()
            ssec = timed_region(torch, ws, lambda: [sctx.estimate_level(t, 0, ns, seed, samples=False)
                                                      for t in range(nterms)])
            single_cost = [sctx.get_stats(t)["seconds"] / ns for t in range(nterms)]
            out["plain_fp64_single_rhs"] = {"value": nterms * ns * ws / ssec, "unit": UNIT,
                                            "samples_timed": nterms * ns,
                                            "seconds_per_sample_per_term": single_cost,
                                            "headline_speedup_over_this": value / (nterms * ns * ws / ssec)}
        octx.close()
        torch.cuda.empty_cache()
        if ttt is not None:
            Nt = ttt["samples_per_term"]
            mixed_est = sum(n * c for n, c in zip(Nt, mixed_cost))
            out["time_to_trace"]["mixed_device_seconds_from_costs"] = mixed_est
            out["time_to_trace"]["fp64_batched"] = {
                "seconds_excl_setup": sum(n * c for n, c in zip(Nt, f64_cost)),
                "what": "projected: the mixed run's sample counts (identical samples) x the measured FP64 "
                        "per-sample device cost of each term; the FP64 context reuses the mixed setup's test "
                        "vectors, so no FP64 setup time is measured"}
            if single_cost:
                out["time_to_trace"]["fp64_single_rhs"] = {
                    "seconds_excl_setup": sum(n * c for n, c in zip(Nt, single_cost)),
                    "what": "projected as above from the single-rhs per-sample cost"}
    else:
        ctx.close()
    if args.serving_requests > 0 and ws == 1:
        torch.cuda.empty_cache()
        try:
            out["serving"] = serving_run(pkg, args)
        except Exception as e:       # the headline line stands without it
            out["serving"] = {"error": f"{type(e).__name__}: {e}"}
    fine = {k: v for k, v in report.items() if k.startswith("D1.f32")}
    if fine:
        v = fine["D1.f32"]
        out["stencil_hbm"] = {"kernel": "D1.f32 (fine Wilson stencil, FP32)",
                              "GB/s": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                              "frac_of_measured_hbm": v["bytes"] / (v["ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                              "frac_of_8TBs": v["bytes"] / (v["ms"] * 1e-3) / 8e12,
                              "avg_launch_us": v["ms"] * 1e3 / v["count"], "launches": v["count"],
                              "bytes_per_launch": v["bytes"] / v["count"],
                              # DRAM bytes per launch from the committed ncu capture (null once
                              # the kernel's source has changed)
                              "traffic": ncu_traffic("D1.f32", v["bytes"] / v["count"])}
    return out, w


# ----------------------------------------------------------------------------- serving
def serving_run(pkg, args):
    """Trace requests of mixed lattices (64^2, 128^2, 256^2, 512^2), couplings (beta 3,
    5) and masses through the request server: first all at once (the saturated rate),
    then arriving as a Poisson stream at args.serving_load x that rate.  Each request is
    a whole problem (gauge field, hierarchy, deflation, MLMC loop to args.serving_tol);
    its time to trace runs from submission to result.  64^2 and 128^2 use 3 levels;
    256^2 and 512^2 a 3-term sum with one solver-only level below it (4096 unknowns,
    stored inverse).  Fixed per-term costs (level sizes) make every request's result
    independent of the load."""
    n = args.serving_requests
    rng = np.random.default_rng(20221115)
    sizes = (64, 128, 256, 512)
    shapes = {64: ((4, 4), (2, 2)), 128: ((4, 4), (2, 2)), 256: ((4, 4), (2, 2), (2, 2)),
              512: ((4, 4), (2, 2), (4, 4))}
    t0 = time.time()
    fields, starts = {}, {}
    for L in sizes:
        for beta in (3.0, 5.0):
            fields[(L, beta)] = inputs.metropolis_u1(L, L, beta, 200, 5000 + L + int(10 * beta))
        dims = [(L, L, 2)]
        for a in shapes[L][:-1]:
            dims.append((dims[-1][0] // a[0], dims[-1][1] // a[1], 16))
        starts[L] = [inputs.start_vectors(7000 + L, i + 1, lx * lt * d, 8) for i, (lx, lt, d) in enumerate(dims)]
    gen_s = time.time() - t0
    masses = {3.0: (-0.09, -0.04), 5.0: (-0.03, 0.02)}

    def make(i):
        L = int(rng.choice(sizes))
        beta = float(rng.choice([3.0, 5.0]))
        m0 = float(rng.choice(masses[beta]))
        agg = shapes[L]
        n0, n1, n2 = 2 * L * L, L * L, L * L // 4
        req = pkg.make_request(fields[(L, beta)], m0, agg, (8,) * len(agg), starts[L], args.serving_tol,
                               100 + i, k=32 if L == 64 else 64, setup_iters=4, defl_tol=1e-3, defl_max_iters=60,
                               costs=[(n0 + n1) / n0, (n1 + n2) / n0, n2 / n0], mg_precision=args.precision,
                               sum_levels=3 if len(agg) > 2 else 0)
        return L, req

    deadline = time.time() + 600.0

    def collect(srv, ids):
        res = []
        for i in ids:
            r = srv.wait(i, max(1.0, deadline - time.time()))
            if r is None:
                raise TimeoutError("serving run exceeded 600 s")
            res.append(r)
        return res

    def summary(rs, span):
        ok = [r for r in rs if r["status"] == 0]
        tt = np.array([r["total_s"] for r in ok]) if ok else np.zeros(1)
        qq = np.array([r["queued_s"] for r in ok]) if ok else np.zeros(1)
        smp = sum(sum(t["nsamples"] for t in r["result"]["terms"]) for r in ok)
        return {"span_s": span, "requests_per_s": len(ok) / span, "samples_per_s": smp / span,
                "p50_time_to_trace_s": float(np.percentile(tt, 50)),
                "p99_time_to_trace_s": float(np.percentile(tt, 99)),
                "p50_queue_s": float(np.percentile(qq, 50)), "p99_queue_s": float(np.percentile(qq, 99)),
                "mean_setup_s": float(np.mean([r["setup_s"] for r in ok])) if ok else 0.0,
                "mean_estimate_s": float(np.mean([r["estimate_s"] for r in ok])) if ok else 0.0}

    with pkg.Server(max_active=args.serving_slots) as srv:
        burst = [make(i) for i in range(n)]
        t0 = time.perf_counter()
        res1 = collect(srv, [srv.submit(r) for _, r in burst])
        span1 = time.perf_counter() - t0
        lam = args.serving_load * n / span1
        stream = [make(n + i) for i in range(n)]
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n))
        t0 = time.perf_counter()
        ids = []
        for a, (_, r) in zip(arrivals, stream):
            wait = a - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids.append(srv.submit(r))
        res2 = collect(srv, ids)
        span2 = time.perf_counter() - t0
        st = srv.stats()
    allr = res1 + res2
    lat = [L for L, _ in burst + stream]
    by_L = {}
    for L in sizes:
        rs = [r for r, l in zip(res2, lat[n:]) if l == L and r["status"] == 0]
        peaks = [r["peak_bytes"] for r, l in zip(allr, lat) if l == L and r["status"] == 0]
        by_L[f"{L}x{L}"] = {"requests": sum(1 for l in lat if l == L),
                            "p50_time_to_trace_s_poisson": float(np.median([r["total_s"] for r in rs])) if rs else None,
                            "device_peak_gb": max(peaks) / 1e9 if peaks else None}
    return {"requests_per_phase": n, "slots": args.serving_slots, "rel_tol": args.serving_tol,
            "mix": "lattices 64^2, 128^2, 256^2, 512^2, beta 3 (m0 -0.09, -0.04) and 5 (m0 -0.03, 0.02); "
                   "3-term sums (4x4 then 2x2 aggregates, 8 test vectors; 256^2 and 512^2 with one "
                   "solver-only level below, 2x2 resp. 4x4 aggregates of level 3), k = 32 (64^2) / 64, "
                   "mg_precision %d" % args.precision,
            "saturated": summary(res1, span1),
            "poisson": dict(summary(res2, span2), load=args.serving_load, arrival_rate_per_s=lam),
            "by_lattice": by_L,
            "all_converged": all(r["status"] == 0 and r["result"]["converged"] == 1 for r in allr),
            "failures": [r["error"] for r in allr if r["status"] != 0],
            "deflation_unconverged": sum(1 for r in allr if r["status"] == 0 and not r.get("deflation_converged", 1)),
            "retries": sum(r["retries"] for r in allr),
            "server": {"max_active_seen": st["max_active_seen"], "budget_gb": st["budget"] / 1e9,
                       "max_reserved_gb": st["max_reserved"] / 1e9},
            "inputs_s": gen_s}


# ----------------------------------------------------------------------------- CPU (oracle)
_W = {}


def _cpu_init(H, defl):
    from oracle import estimator as oest
    _W["H"], _W["defl"] = H, defl
    _W["S"] = oest.DirectSolvers(H)
    _W["terms"] = oest.term_list(H.nlevels)
    for lev in range(1, H.nlevels + 1):   # factorise up front
        _W["S"].solve(lev, np.zeros((H.D[lev - 1].shape[0], 1), np.complex128))


def _cpu_job(job):
    from oracle import estimator as oest
    t, first, count, seed = job
    term = _W["terms"][t]
    d = _W["defl"] if term[1] is None else None
    s = oest.noise_samples(_W["H"], term, seed, first, count, _W["S"], d)
    return len(s)


def cpu_oracle_setup(w):
    from oracle import deflation as odefl
    from oracle import hierarchy as ohier
    t0 = time.time()
    H = ohier.build_hierarchy(w.gauge(), w.m0, w.agg, w.nvec, w.start_vectors(), w.setup_iters)
    defl = odefl.coarsest_deflation(H.D[-1], H.g5[-1], w.k)
    return H, defl, time.time() - t0


def cpu_oracle_rate(w, H, defl, seconds, procs, per_term=None):
    """Samples/s of the oracle (direct sparse-LU solves), the same per-step mix of
    terms, samples split over `procs` single-threaded spawned processes."""
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"
    ctxm = mp.get_context("spawn")
    nterms = H.nlevels
    with ctxm.Pool(procs, initializer=_cpu_init, initargs=(H, defl)) as pool:
        pool.map(_cpu_job, [(t, 10 ** 7 + p, 1, w.noise_seed) for p in range(procs) for t in range(nterms)])
        if per_term is None:   # size the sample for ~`seconds` of wall time
            t0 = time.time()
            pool.map(_cpu_job, [(t, 2 * 10 ** 7 + p, 1, w.noise_seed) for p in range(procs) for t in range(nterms)])
            one = time.time() - t0
            per_term = max(1, int(seconds / one))
        jobs = [(t, 3 * 10 ** 7 + 1000 * p, per_term, w.noise_seed) for p in range(procs) for t in range(nterms)]
        t0 = time.time()
        n = sum(pool.map(_cpu_job, jobs))
        dt = time.time() - t0
    return n / dt, n, dt, per_term


ORACLE_LIMIT = ("the oracle's direct sparse LU cannot factor the levels of lattices above 128^2 within a "
                "bounded time (256^2: about 3 minutes of factorisation alone, 1024^2: out of reach), so the CPU "
                "baseline runs the largest workload it can bound")


def cpu_baseline(w, seconds, headline):
    procs = os.cpu_count() or 1
    H, defl, setup_s = cpu_oracle_setup(w)
    rate, n, dt, per = cpu_oracle_rate(w, H, defl, seconds, procs)
    out = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle", "workload": w.name,
           "sample": f"{n} samples ({per} per term per process, {H.nlevels} terms, {procs} spawned "
                     f"single-threaded processes) of {w.name}, direct sparse-LU solves; "
                     f"{dt:.1f} s wall; oracle setup {setup_s:.0f} s not timed"}
    if w.name != headline:
        out["note"] = ORACLE_LIMIT
    return out


def reference_arm(args, rank, ws):
    """The oracle timed on the host cores (rank 0 only), on the largest workload its
    direct solves can bound (args.cpu_workload)."""
    w = inputs.workload(args.cpu_workload)
    if rank != 0:
        return None
    procs = os.cpu_count() or 1
    H, defl, setup_s = cpu_oracle_setup(w)
    budget = max(5.0, 60.0 / max(1, args.steps + args.warmup))
    _, _, _, per = cpu_oracle_rate(w, H, defl, budget, procs)
    rates, times, ns = [], [], []
    for k in range(args.warmup + args.steps):
        r, n, dt, _ = cpu_oracle_rate(w, H, defl, budget, procs, per_term=per)
        if k >= args.warmup:
            rates.append(r)
            times.append(dt)
            ns.append(n)
    value = sum(ns) / sum(times)
    sample = (f"each step {ns[0]} samples ({per} per term per process, {H.nlevels} terms, {procs} spawned "
              f"single-threaded processes) of {w.name} by direct sparse-LU solves; setup {setup_s:.0f} s not timed")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
            "data": f"synthetic: seeded Metropolis U(1) gauge field beta={w.beta} {w.Lx}x{w.Lt}, Z2 noise",
            "config": {"workload": w.name, "lattice": f"{w.Lx}x{w.Lt}", "levels": w.nlevels,
                       "deflated_triplets": w.k, "block_rhs": w.nrhs, "gpu_arm_workload": args.workload,
                       "why_this_workload": ORACLE_LIMIT if w.name != args.workload else None},
            "cpu_baseline": {"kind": "oracle", "cores": procs, "sample": sample, "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, ws, local = dist_setup(args)
    if args.impl == "reference":
        out = reference_arm(args, rank, ws)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out, w = gpu_arm(args, rank, ws, local)
    if rank == 0:
        if not args.no_cpu and ws == 1:
            out["cpu_baseline"] = cpu_baseline(inputs.workload(args.cpu_workload), args.cpu_seconds, w.name)
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
