"""Benchmark: pISTA outer iterations per second on the n = 10,000 grid workload.

One step is one outer iteration of Algorithm 1 through the library (W = Theta^{-1} from the
cached factor, gradient / free set / sign guess / stop test, the sandwich products of eq. b,
and the line search with a Cholesky factorisation per trial), on a 100 x 100 lattice
precision (4-neighbour weights -1, diagonal 4.1), m = 2,000 samples, lambda = 0.1.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|tf32x3|fp64]
                  [--products auto|dense|sparse]
  python bench.py --impl reference ...   the FP64 CPU oracle on a bounded sample

The default line is the BF16x3 split-precision form with the automatic choice of sandwich
products; it also reports the time to relative KKT residual 1e-6 and the plain FP64 form's
iterations/s and time to the same tolerance on the same workload.

For N > 1 (torchrun) every rank solves its own replica (the single solve does not shard):
value = the iterations of all ranks / the slowest rank's time.  Prints one JSON line.
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

METRIC = "pISTA iters/s (n=10k grid, lambda=0.1); time-to-KKT 1e-6"

# DRAM bytes (read + write) per launch of the tensor-core product in the step (the W = X^T X
# and W R launches whose CUDA-event times give the roofline), from one ncu capture of this
# workload (profiles/k_gemm_tc_step_traffic_n10000.md); BF16x3 only, None elsewhere.
TC_TRAFFIC_PER_LAUNCH = {"bf16x3": 2.015e9}
UNIT = "iters/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(x: float) -> float:
    """The maximum of a per-rank scalar over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Whole-job rate: every rank processed units_per_rank; the job took the slowest rank's time."""
    return world * units_per_rank / slowest_seconds


def workload(side: int, m: int):
    from paper_2205_10027_gb300 import inputs
    return inputs.grid_n10000(side=side, m=m, seed=2, lam=0.1)


# ----------------------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------------------
def oracle_rate(sample_side: int, full_n: int, iters: int):
    """Oracle iterations/s on a bounded sample (a smaller lattice of the same family),
    scaled to the full size by the n^3 work of an iteration."""
    from oracle import pista
    p = workload(sample_side, max(2, sample_side * sample_side // 5))
    t0 = time.perf_counter()
    res = pista.pista(p.S, p.lam, tol=0.0, max_iter=iters)
    dt = time.perf_counter() - t0
    ns = sample_side * sample_side
    rate = res["iterations"] / dt * (ns / full_n) ** 3
    return rate, dt, res["iterations"], ns


def oracle_full_iteration(side: int, m: int):
    """One oracle iteration of the workload itself (n = side^2), from its start point:
    (iterations/s, seconds, iterations, line-search trials)."""
    from oracle import pista
    p = workload(side, m)
    t0 = time.perf_counter()
    res = pista.pista(p.S, p.lam, tol=0.0, max_iter=1, trace=True)
    dt = time.perf_counter() - t0
    return res["iterations"] / dt, dt, res["iterations"], res["trace"][0]["trials"]


# Kernel classes of the step (glasso_profile) and what bounds each: FLOP classes on the tensor
# pipe (split-precision products, FLOPs counted once, the narrow type's peak / 3) or on the FP64
# pipe; byte classes on HBM.
CLASS_BOUND = {"factor": "tensor", "inverse": "tensor", "refine": "tensor", "sandwich": "tensor",
               "trailing": "tensor", "panel": "tensor", "spmm": "fp64",
               "gradient": "hbm", "trial": "hbm", "residual": "fp64", "logdet2": "hbm", "aux": "hbm"}
CLASS_UNIT = {"factor": "whole Cholesky-with-inverse factorisations (one CUDA graph each: k_gemm_tc, k_split, "
                        "k_gemm_f32, k_leaf128 in the split-precision forms, k_leaf_chol_inv in FP64)",
              "inverse": "W = X^T X (k_gemm_tc)", "refine": "refinement product W R (k_gemm_tc)",
              "sandwich": "dense sandwich products (k_gemm_tc)", "spmm": "sparse sandwich products (k_spmm)",
              "gradient": "gradient pass (k_gradient)", "trial": "trial-point pass (k_trial)",
              "residual": "FP64 residual I - Theta W (k_spmm residual epilogue; 2 nnz(Theta) n FP64 FLOPs)",
              "logdet2": "second-order log-det difference (CSR of dTheta, k_spmm, k_trace_pairs)",
              "aux": "symmetrising copies (k_mirror_lower, k_add_lower_mirror)"}


def roofline_by_class(prof: dict, step_ms_total: float, args, n: int, fp64_peak_live: float) -> dict:
    """Per kernel class of the timed steps: share of the device time, achieved rate on its
    algorithmic work, the peak that bounds it and the fraction; the roofline object names the
    class with the largest share.  Peaks: MEASURED_PEAKS.json (HBM copy, cuBLAS BF16 sustained x
    the nominal TF32/BF16 ratio / 3 split products); the FP64 pipe from the recipe's unit
    counts: 2 DFMA lanes / clock / SM (measured by glasso_probe_fp64_peak) x 152 SMs x the max
    SM clock x 2 FLOPs."""
    peaks, kind = _peaks()
    fp64_peak = 2.0 * 2.0 * 152 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if args.precision == "fp64":
        tensor_peak, tensor_src = fp64_peak, "FP64 pipe (2 DFMA/clk/SM x 152 SMs x max clock)"
    else:
        ratio = (1100.0 / 2250.0) if args.precision == "tf32x3" else 1.0
        tensor_peak = peaks.get("bf16_tflops_sustained", 1700.0) * ratio / 3.0
        tensor_src = f"{kind}: bf16 sustained x nominal dtype ratio / 3 split products"
    classes = {}
    for c, v in prof.items():
        if not v["ms"] or c not in CLASS_BOUND:
            continue
        bound = CLASS_BOUND[c]
        if bound == "hbm":
            unit, achieved, peak, src = "GB/s", v["work"] / (v["ms"] / 1e3) / 1e9, peaks.get("hbm_gbs", 6800.0), kind
        elif bound == "fp64":
            unit, achieved, peak, src = "TFLOP/s", v["work"] / (v["ms"] / 1e3) / 1e12, fp64_peak, "FP64 pipe"
        else:
            unit, achieved, peak, src = "TFLOP/s", v["work"] / (v["ms"] / 1e3) / 1e12, tensor_peak, tensor_src
            if args.precision == "fp64":
                bound = "alu"
        classes[c] = {"unit_of_work": CLASS_UNIT.get(c, c), "ms": v["ms"], "launches": v["launches"],
                      "share": v["ms"] / step_ms_total if step_ms_total else None, "bound": bound,
                      "achieved": achieved, "unit": unit, "peak": peak, "peak_source": src,
                      "frac": achieved / peak if peak else None}
    dom = max(classes, key=lambda c: classes[c]["ms"])
    d = classes[dom]
    traffic = None
    if dom in ("inverse", "refine") and args.precision in TC_TRAFFIC_PER_LAUNCH and args.side == 100:
        traffic = TC_TRAFFIC_PER_LAUNCH[args.precision]
    return {"bound": d["bound"], "kernel": dom, "unit_of_work": d["unit_of_work"], "achieved": d["achieved"],
            "peak": d["peak"], "unit": d["unit"], "frac": d["frac"], "traffic": traffic,
            "share_of_step": d["share"], "launches": d["launches"], "peak_source": d["peak_source"],
            "fp64_probe_tflops": fp64_peak_live, "classes": classes}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    full_n = args.side * args.side
    cores = os.cpu_count()
    rates = []
    for _ in range(args.warmup):
        oracle_rate(args.sample_side, full_n, 1)
    t_all = time.perf_counter()
    for _ in range(args.steps):
        r, _, _, ns = oracle_rate(args.sample_side, full_n, 1)
        rates.append(r)
    elapsed = time.perf_counter() - t_all
    value = statistics.median(rates)
    sample = (f"one oracle iteration per step on a {args.sample_side}x{args.sample_side} lattice "
              f"(n={args.sample_side ** 2}, m=n/5) from the start point, scaled by (n_sample/n)^3")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"grid{args.side}x{args.side}_n{full_n}_m{args.m}_lam0.1",
                                        "sample_n": args.sample_side ** 2},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2205_10027_gb300 import binding

    p = workload(args.side, args.m)
    n = p.S.shape[0]
    S_dev = torch.from_numpy(np.ascontiguousarray(p.S)).to(dev)
    stream = torch.cuda.current_stream(dev)
    h = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, device=local, stream=stream.cuda_stream,
                       products=args.products, method=args.method)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-resident steps -------------------------------------------------------------
    h.begin(S_dev, p.lam)
    for _ in range(args.warmup):
        h.step(0.0)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    trials = 0
    with ClockSampler(local) as clk:
        h.profile_start()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            st, res = h.step(0.0)
            launches += res["kernel_launches"]
            trials += res["trials"]
        e1.record(stream)
        barrier()
        prof = h.profile_stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    last = res
    h.end()
    value = job_throughput(args.steps, world, ms / 1000.0)

    # ---- end to end through the public API, host buffers ------------------------------------
    S_pin = torch.from_numpy(np.ascontiguousarray(p.S)).pin_memory()
    out_pin = torch.empty((n, n), dtype=torch.float64).pin_memory()
    he = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, device=local, stream=stream.cuda_stream,
                        max_iter=args.steps, products=args.products, method=args.method)
    he.solve(S_pin.numpy(), p.lam, 0.0, out=out_pin.numpy())  # warm the workspace
    barrier()
    t0 = time.perf_counter()
    _, res_e2e = he.solve(S_pin.numpy(), p.lam, 0.0, out=out_pin.numpy())
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    he.close()
    e2e_value = job_throughput(res_e2e["iterations"], world, e2e_s)

    # ---- time to tolerance (device-resident) ---------------------------------------------------
    ttt = None
    if args.time_to_tol:
        ht = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, device=local, stream=stream.cuda_stream, max_iter=2000,
                            products=args.products, method=args.method)
        barrier()
        t0 = time.perf_counter()
        _, rt = ht.solve(S_dev, p.lam, p.tol)
        barrier()
        ttt = {"seconds": time.perf_counter() - t0, "iterations": rt["iterations"], "trials": rt["trials"],
               "rel_kkt_l1": rt["rel_kkt_l1"], "status": binding.STATUS[rt["status"]]}
        ht.close()

    # ---- the same split-precision form with FP32 Cholesky panels (glasso_config.fp32_panels),
    # device-resident steps timed the same way, for the cost of the FP64 panels ---------------
    fp32p = None
    if args.precision != "fp64" and not args.fp32_panels:
        hp = binding.Handle(precision=args.precision, fp32_panels=True, autotune=not args.no_autotune, device=local,
                            stream=stream.cuda_stream, products=args.products, method=args.method)
        hp.begin(S_dev, p.lam)
        for _ in range(args.warmup):
            hp.step(0.0)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            hp.step(0.0)
        p1.record(stream)
        barrier()
        hp.end()
        hp.close()
        pms = max_over_ranks(p0.elapsed_time(p1))
        fp32p = {"iters_per_s": job_throughput(args.steps, world, pms / 1000.0), "ms_per_step": pms / args.steps,
                 "note": "same workload and steps, Cholesky panels factored in FP32 (the option glasso_config.fp32_panels)"}

    # ---- the plain FP64 form on the same workload (what the split-precision form must beat) --
    fp64 = None
    if args.fp64_form and args.precision != "fp64":
        hf = binding.Handle(precision="fp64", device=local, stream=stream.cuda_stream, max_iter=2000,
                            products=args.products)
        hf.begin(S_dev, p.lam)
        hf.step(0.0)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(2):
            hf.step(0.0)
        f1.record(stream)
        barrier()
        hf.end()
        fp64 = {"iters_per_s": job_throughput(2, world, max_over_ranks(f0.elapsed_time(f1)) / 1000.0)}
        if args.time_to_tol:
            barrier()
            t0 = time.perf_counter()
            _, rf = hf.solve(S_dev, p.lam, p.tol)
            barrier()
            fp64.update({"time_to_tol_s": time.perf_counter() - t0, "iterations": rf["iterations"],
                         "rel_kkt_l1": rf["rel_kkt_l1"], "status": binding.STATUS[rf["status"]]})
        hf.close()
    h.close()

    if rank == 0:
        rl = roofline_by_class(prof, ms, args, n, binding.probe_fp64_peak(local))
        hbm = {c: v for c, v in rl["classes"].items() if v["bound"] == "hbm"}
        cpu = None
        if not args.no_cpu_baseline:
            # measured on the workload itself: one full oracle iteration at n (no scaling); the
            # bounded smaller-lattice sample of the reference arm is reported beside it
            rate, dt, its, trials = oracle_full_iteration(args.side, args.m)
            cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"measured at n={n}: {its} full oracle iteration ({trials} line-search trials) "
                             f"from the start point of the {args.side}x{args.side} lattice workload in {dt:.1f}s"}
            srate, sdt, sits, ns = oracle_rate(args.sample_side, n, 1)
            cpu["scaled_sample"] = {
                "value": srate, "unit": UNIT,
                "sample": f"{sits} oracle iteration on a {args.sample_side}x{args.sample_side} lattice (n={ns}, m=n/5) "
                          f"in {sdt:.1f}s, scaled to n={n} by (n_sample/n)^3 (the reference arm's sample)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "tf32x3": "f64+tf32x3", "bf16x3": "f64+bf16x3"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"grid{args.side}x{args.side}_n{n}_m{args.m}_lam0.1",
                       "precision": args.precision, "products": args.products, "method": args.method,
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (each n x n FP64 matrix is %.0f MB)" % (8 * n * n / 1e6)},
            "gpu_launches": launches, "trials_in_timed_steps": trials,
            "last_step": {"rel_kkt_l1": last["rel_kkt_l1"], "iterations": last["iterations"]},
            "roofline": rl, "hbm_passes": hbm, "profile": prof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n * n / max(res_e2e["iterations"], 1),
                    "d2h_bytes_per_step": 8 * n * n / max(res_e2e["iterations"], 1),
                    "note": "one glasso_solve from pinned host S to host Theta, max_iter=steps"},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "time_to_tol": ttt,
            "fp64_form": fp64,
            "fp32_panels_form": fp32p,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_op(args):
    """Micro-benchmark of one kernel class through its single-step entry point (the sandwich
    products Y = Theta X Theta, or the Cholesky factorisation) at n = side^2, for profiling."""
    import torch
    from paper_2205_10027_gb300 import binding
    p = workload(args.side, args.m)
    n = p.S.shape[0]
    rng = np.random.default_rng(0)
    A = np.diag(1.0 / (np.diag(p.S) + p.lam))
    X = rng.standard_normal((n, n))
    X = 0.5 * (X + X.T)
    Ad, Xd = torch.from_numpy(A).cuda(), torch.from_numpy(X).cuda()
    Sd = torch.from_numpy(p.S + np.eye(n)).cuda()
    h = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, products=args.products)
    fn = (lambda: h.op_sandwich(Ad, Xd)) if args.op == "sandwich" else (lambda: h.op_cholesky(Sd))
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    h.profile_start()
    for _ in range(args.steps):
        fn()
    prof = h.profile_stop()
    h.close()
    out = {"op": args.op, "n": n, "precision": args.precision, "steps": args.steps}
    for k, v in prof.items():
        if v["ms"]:
            out[k] = {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                      "tflops" if k not in ("gradient", "trial") else "gbs": v["work"] / (v["ms"] / 1e3) /
                      (1e12 if k not in ("gradient", "trial") else 1e9)}
    print(json.dumps(out))


# Tables 1 and 2 of the paper (pISTA GPU column: seconds, iterations; RTX 2080 Ti, FP32 CuPy)
PAPER_TABLES = {
    1: dict(n=1000, rows=[("chain", 0.6, 0.04, 2.0), ("chain", 0.4, 0.10, 6.6), ("random", 0.6, 0.04, 2.2),
                          ("random", 0.4, 0.10, 6.4), ("planar", 0.6, 0.03, 2.0), ("planar", 0.4, 0.24, 15.4)]),
    2: dict(n=10000, rows=[("chain", 0.4, 5.69, 3.0), ("chain", 0.2, 12.89, 7.0), ("random", 0.4, 1.56, 0.6),
                           ("random", 0.2, 5.67, 3.0), ("planar", 0.4, 3.92, 2.0), ("planar", 0.2, 20.91, 10.2)]),
}


def run_paper_table(args):
    """The paper's own synthetic protocol (Sec. 6.1.1; m = 3% n, stop at 1e-2, samples
    standardised), solved end to end from host S through glasso_solve, beside the printed
    GPU numbers of Table 1 or 2."""
    import torch
    from paper_2205_10027_gb300 import binding, inputs, metrics
    tab = PAPER_TABLES[args.paper_table]
    n = tab["n"]
    seeds = args.paper_seeds
    h = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, max_iter=1000)
    rows = []
    for kind, alpha, paper_s, paper_it in tab["rows"]:
        times, its, nnz, mcc = [], [], [], []
        for rep in range(seeds):
            S, T = inputs.paper_protocol(kind, n, seed=300 + rep, return_theta=True)
            h.solve(S, alpha, 1e-2) if rep == 0 else None   # warm the workspace and graphs
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            theta, res = h.solve(S, alpha, 1e-2)
            times.append(time.perf_counter() - t0)
            its.append(res["iterations"])
            nnz.append(res["nnz"])
            mcc.append(metrics.support_mcc(T, theta))
        rows.append({"kind": kind, "alpha": alpha, "seconds": statistics.mean(times),
                     "iterations": statistics.mean(its), "nnz": statistics.mean(nnz),
                     "mcc": statistics.mean(mcc),
                     "paper_seconds": paper_s, "paper_iterations": paper_it,
                     "speedup_vs_paper": paper_s / statistics.mean(times)})
    h.close()
    print(json.dumps({"paper_table": args.paper_table, "n": n, "precision": args.precision, "seeds": seeds,
                      "protocol": "m = 3% n, standardised samples, eps = 1e-2, start diag(1/(S_ii+alpha))",
                      "timing": "glasso_solve from host S to host Theta, wall clock",
                      "paper_hardware": "GeForce RTX 2080 Ti, FP32 (CuPy)", "rows": rows}))


def run_batch(args):
    """Batched regularisation paths: independent ER problems with n log-uniform in
    [32, 1024], a descending lambda path of 8 values in [0.5, 0.02], warm-started, solved
    concurrently through glasso_solve_batch.  Metric: solves per second."""
    from paper_2205_10027_gb300 import binding, inputs
    probs = inputs.batch_path_problems(count=args.batch_count, seed=3)
    for p in probs:
        p["tol"] = args.batch_tol
    h = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, serve_slots=args.slots, max_iter=args.batch_max_iter)
    warm = inputs.batch_path_problems(count=min(4, len(probs)), seed=97)
    for p in warm:
        p["tol"] = args.batch_tol
    h.solve_batch(warm)
    t0 = time.perf_counter()
    _, res = h.solve_batch(probs)
    dt = time.perf_counter() - t0
    h.close()
    flat = [r for rs in res for r in rs]
    # the plain FP64 form one solve at a time on a seeded sample of the same problems (every
    # lambda of each sampled problem, cold starts in the path order of glasso_solve_batch)
    fp64 = None
    if args.batch_fp64_sample:
        idx = np.linspace(0, len(probs) - 1, args.batch_fp64_sample).astype(int)
        hf = binding.Handle(precision="fp64", serve_slots=1, max_iter=args.batch_max_iter)
        t0 = time.perf_counter()
        _, rf = hf.solve_batch([probs[i] for i in idx])
        dtf = time.perf_counter() - t0
        hf.close()
        nf = sum(len(r) for r in rf)
        fp64 = {"problems": len(idx), "solves": nf, "seconds": dtf, "solves_per_s": nf / dtf,
                "converged": sum(r["status"] == 0 for rs in rf for r in rs),
                "sample": "problems at evenly spaced indices of the same list, one slot (one solve at a time)"}
    print(json.dumps({"mode": "batch", "precision": args.precision, "problems": len(probs),
                      "solves": len(flat), "seconds": dt, "solves_per_s": len(flat) / dt,
                      "slots": args.slots, "tol": args.batch_tol, "max_iter": args.batch_max_iter,
                      "converged": sum(r["status"] == 0 for r in flat),
                      "iterations_total": sum(r["iterations"] for r in flat),
                      "trials_total": sum(r["trials"] for r in flat),
                      "fp64_one_at_a_time": fp64}))


def run_served(args):
    """Served stream: Poisson arrivals, each request (S, lambda) from a pool of seeded chain /
    grid datasets with n log-uniform in [64, n_max], lambda ~ U[0.05, 0.3], warm-started from
    the nearest earlier lambda of the same dataset; requests are admitted by an HBM budget.
    Reports p50 / p99 latency (submit to result) and solves/s, beside the same requests solved
    one at a time in FP64."""
    from paper_2205_10027_gb300 import binding, inputs
    arrivals, ids, lams, pool = inputs.served_stream(count=args.served, rate_hz=args.rate, nmax=args.served_nmax)
    cache = {}

    def S_of(d):
        if d not in cache:
            cache[d] = inputs.served_dataset(pool[d])
        return cache[d]

    for d in sorted(set(ids.tolist())):
        S_of(int(d))
    h = binding.Handle(precision=args.precision, fp32_panels=args.fp32_panels, autotune=not args.no_autotune, serve_slots=args.slots,
                       hbm_budget_bytes=int(args.budget_gb * 1e9), max_iter=args.batch_max_iter)
    t_start = time.perf_counter()
    tickets = []
    for a, d, lam in zip(arrivals, ids, lams):
        now = time.perf_counter() - t_start
        if a > now:
            time.sleep(a - now)
        tickets.append((h.submit(S_of(int(d)), float(lam), args.batch_tol, dataset_id=int(d)),
                        S_of(int(d)).shape[0]))
    lat, done = [], {}
    while len(done) < len(tickets):
        for t, n in tickets:
            if t in done:
                continue
            try:
                st, res, _ = h.poll(t)
            except binding.GlassoError as e:   # a finished request with an error status
                st, res = e.status, {"status": e.status, "t_done": time.perf_counter(), "t_submit": 0.0}
            if st != binding.PENDING:
                done[t] = res
                lat.append(res["t_done"] - res["t_submit"])
        time.sleep(0.001)
    total = time.perf_counter() - t_start
    h.close()
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
    # one at a time in FP64 on a sample of the same requests
    serial = None
    if args.serial_sample:
        hs = binding.Handle(precision="fp64", max_iter=args.batch_max_iter)
        idx = np.linspace(0, len(ids) - 1, args.serial_sample).astype(int)
        t0 = time.perf_counter()
        for i in idx:
            hs.solve(S_of(int(ids[i])), float(lams[i]), args.batch_tol)
        serial = {"requests": len(idx), "seconds": time.perf_counter() - t0,
                  "solves_per_s": len(idx) / (time.perf_counter() - t0)}
        hs.close()
    print(json.dumps({"mode": "served", "precision": args.precision, "requests": len(tickets),
                      "rate_hz": args.rate, "n_max": args.served_nmax, "slots": args.slots,
                      "seconds": total, "solves_per_s": len(tickets) / total,
                      "p50_s": pct(0.50), "p99_s": pct(0.99),
                      "converged": sum(r["status"] == 0 for r in done.values()),
                      "serial_fp64_sample": serial}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "tf32x3", "bf16x3"], default="bf16x3")
    ap.add_argument("--method", choices=["pista", "gista"], default="pista",
                    help="outer method (glasso_method): Algorithm 1, or plain proximal gradient")
    ap.add_argument("--no-autotune", action="store_true",
                    help="split-precision forms: the built-in product kernel rule instead of the autotuner")
    ap.add_argument("--fp32-panels", action="store_true",
                    help="split-precision forms: factor the Cholesky panels in FP32 (default FP64)")
    ap.add_argument("--products", choices=["auto", "dense", "sparse"], default="auto",
                    help="how the sandwich products are formed (glasso_products)")
    ap.add_argument("--side", type=int, default=100)
    ap.add_argument("--m", type=int, default=2000)
    ap.add_argument("--sample-side", type=int, default=50)
    ap.add_argument("--no-time-to-tol", dest="time_to_tol", action="store_false",
                    help="skip the time-to-tolerance solve")
    ap.add_argument("--time-to-tol", dest="time_to_tol", action="store_true")
    ap.add_argument("--no-fp64-form", dest="fp64_form", action="store_false",
                    help="skip the plain FP64 form's iterations/s and time-to-tolerance")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--op", choices=["sandwich", "cholesky"], default=None,
                    help="micro-benchmark one kernel class instead of the step")
    ap.add_argument("--paper-table", type=int, choices=[1, 2], default=None,
                    help="the paper's Table 1 or 2 protocol beside its printed GPU times")
    ap.add_argument("--paper-seeds", type=int, default=3)
    ap.add_argument("--batch", action="store_true", help="batched lambda paths (solves/s)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-tol", type=float, default=1e-6)
    ap.add_argument("--batch-max-iter", type=int, default=500)
    ap.add_argument("--batch-fp64-sample", type=int, default=4,
                    help="problems of the batch also solved one at a time in FP64 (0: none)")
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--served", type=int, default=0, help="served stream of this many requests")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--served-nmax", type=int, default=4096)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--serial-sample", type=int, default=20)
    args = ap.parse_args()
    if args.batch:
        run_batch(args)
        return
    if args.served:
        run_served(args)
        return
    if args.op:
        run_op(args)
        return
    if args.paper_table:
        run_paper_table(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
