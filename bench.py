#!/usr/bin/env python3
"""Benchmark of the Chebyshev typicality hot path on GB300.

One step = one pass of the whole path over the workload: spectral bounds of
every sector (Lanczos), random vectors, K/2 fused Chebyshev steps over all
sectors in one launch each, moment assembly and the thermodynamics (Z, E, C,
chi) on the temperature grid.  Default workload: spin-1/2 Heisenberg ring
N = 20, J = 1, all 21 S^z sectors (dims 1 .. 184756), R = 100 random vectors
per sector, K = 1000 moments, eps = 0.025, 200-point log grid T in [0.02, 10];
headline precision FP32 vectors with FP64 reductions, FP64 reported beside it.

Metric: basis-states x vectors x Chebyshev-steps per second (whole job).
With torchrun (N > 1) every rank runs the same workload on its own random
vectors (r0 = rank * R), the moments are averaged with one all-reduce per
pass, and the value is the work of all ranks over the slowest rank's time.

--impl reference times the CPU oracle (the plain C FP64 recursion) on a
bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import kpm_workloads as W  # noqa: E402

METRIC = "Chebyshev states x vectors x steps / s"
UNIT = "state-vector-steps/s"


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="ring20_sectors", choices=list(W.WORKLOADS))
    p.add_argument("--precision", default=None, choices=["fp32", "fp64"])
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--lanczos-iters", type=int, default=100)
    p.add_argument("--lanczos-tol", type=float, default=1e-8,
                   help="relative residual bound at which the Lanczos bound estimate stops")
    p.add_argument("--no-large", action="store_true",
                   help="skip the blocks of the two largest workloads (ring N=34, 4x6 torus)")
    p.add_argument("--large-steps", type=int, default=20,
                   help="Chebyshev steps per timed block of the large workloads")
    p.add_argument("--large-reps", type=int, default=3)
    p.add_argument("--large-workloads", default="ring34_m0,j1j2sq24_full",
                   help="comma-separated workloads of the large blocks")
    p.add_argument("--only-large", action="store_true",
                   help="time only the large blocks (print one line per workload)")
    p.add_argument("--no-gradient", action="store_true",
                   help="skip the forward + adjoint pass of the gradient workload")
    p.add_argument("--only-gradient", action="store_true",
                   help="time only the forward + adjoint pass of the gradient workload")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip the autotuner runs reported beside the workloads")
    p.add_argument("--tuned", action="store_true",
                   help="autotune the headline workload first and time the tuned schedule")
    return p.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for name in ("kpm_moments.cu", "kpm_block.cu", "kpm_device.cuh", "kpm_internal.h", "kpm_run.h"):
        with open(os.path.join(ROOT, "paper_2104_13218_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(workload, precision):
    """dram bytes per step launch from the committed ncu summary, if it is for this kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{workload}:{precision}")
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="kpm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device_index), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def units_per_step(w):
    dims = [kpm_dim(w.model.n_sites, k) for k in w.n_up]
    return sum(dims) * w.R * w.steps, sum(dims)


def kpm_dim(n, k):
    return (1 << n) if k < 0 else math.comb(n, k)


# --------------------------------------------------------------------------- oracle (CPU) leg

def oracle_sample(w, target_s=12.0):
    """Time the C oracle on the largest sector of the workload, R vectors, a bounded number of steps."""
    from oracle import c_oracle
    bi, bj, J = w.model.arrays()
    k = max(w.n_up, key=lambda kk: kpm_dim(w.model.n_sites, kk))
    D = kpm_dim(w.model.n_sites, k)
    R = w.R
    # probe with 2 steps, then size the sample to about target_s seconds
    t0 = time.perf_counter()
    c_oracle.moments(w.model.n_sites, bi, bj, J, k, 10.0, 0.0, 2 * 2, R, w.seed, 0, 2)
    t_probe = time.perf_counter() - t0
    steps = int(max(2, min(w.steps, 2 * target_s / max(t_probe, 1e-6))))
    t0 = time.perf_counter()
    c_oracle.moments(w.model.n_sites, bi, bj, J, k, 10.0, 0.0, 2 * steps, R, w.seed, 0, steps)
    dt = time.perf_counter() - t0
    value = D * R * steps / dt
    sample = (f"{w.model.name} sector n_up={k} (D={D}), R={R}, {steps} of {w.steps} "
              f"Chebyshev steps, C oracle FP64, {dt:.1f} s")
    return {"value": value, "unit": UNIT, "cores": c_oracle.num_threads(), "kind": "oracle",
            "sample": sample, "seconds": dt}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    w = W.workload(args.workload)
    from oracle import c_oracle
    c_oracle.build()
    vals = []
    for i in range(args.warmup + args.steps):
        s = oracle_sample(w, target_s=4.0)
        if i >= args.warmup:
            vals.append(s)
    value = statistics.median(v["value"] for v in vals)
    sample = vals[-1]["sample"]
    # each step of this arm is one bounded sample of the workload; its time is measured
    sample_ms = statistics.median(v["seconds"] for v in vals) * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sample_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.key, "note": w.note,
                       "step": "one bounded sample of the workload per step (measured): " + sample,
                       "full_pass_ms_extrapolated": units_per_step(w)[0] / value * 1e3},
            "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "sample": sample,
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU leg

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2104_13218_gb300 as kpm
    from paper_2104_13218_gb300 import _lib

    from paper_2104_13218_gb300.replicas import combine_moments, vector_offset

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.workload(args.workload)
    precision = args.precision or ("fp32" if "fp32" in w.precisions else "fp64")
    units, total_rows = units_per_step(w)
    L = kpm.lib()
    r0 = vector_offset(rank, w.R)
    secs_T = w.T
    mirror = w.mirror

    ws_b = torch.empty(kpm.bounds_workspace_size(w.model, w.n_up), dtype=torch.uint8, device=dev)

    def make(prec):
        ws_m = torch.empty(kpm.moments_workspace_size(w.model, w.n_up, w.K, w.R, prec,
                                                      tuned=args.tuned),
                           dtype=torch.uint8, device=dev)
        S = len(w.n_up)
        out = {k: torch.empty((S, w.K), dtype=torch.float64, device=dev) for k in ("mu", "mu_M", "mu_M2")}

        def step():
            bnd = kpm.bounds(w.model, w.n_up, eps=w.eps, max_iter=args.lanczos_iters,
                             tol=args.lanczos_tol, seed=w.seed, workspace=ws_b)
            mom = kpm.moments(w.model, w.n_up, w.K, w.R, w.seed, a=bnd["a"], b=bnd["b"], r0=r0,
                              precision=prec, device=True, out=out, workspace=ws_m,
                              allow_ebounds=True, tuned=args.tuned)
            combine_moments(mom, world)
            secs = kpm.sector_set(w.model.n_sites, w.n_up, bnd["a"], bnd["b"], mirror)
            th = kpm.thermo(mom["mu"], mom["mu_M"], mom["mu_M2"], secs, secs_T, kernel=w.kernel)
            keep["out"] = th
            return th
        keep = {}
        return step, keep

    def timed(step, n_steps, n_warm, profile=False, clocks=False):
        for _ in range(n_warm):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.start()
        launches0 = ctypes_read(L)[2]
        if profile:
            L.kpm_profile_enable(1)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = ctypes_read(L)
        if profile:
            L.kpm_profile_enable(0)
        clk = sampler.stop() if sampler else None
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        return ms, prof, prof[2] - launches0, clk

    hbm_peak, peak_kind = peaks()
    if args.only_gradient:
        res = gradient_block(args, timed)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return 0
    if args.only_large:
        for key in args.large_workloads.split(","):
            res = large_block(args, key, timed, hbm_peak, peak_kind)
            if rank == 0:
                print(json.dumps(res), flush=True)
        return 0
    tune_info = None
    if args.tuned or not args.no_autotune:
        bnd0 = kpm.bounds(w.model, w.n_up, eps=w.eps, max_iter=args.lanczos_iters,
                          tol=args.lanczos_tol, seed=w.seed)
        t = kpm.autotune(w.model, w.n_up, bnd0["a"], bnd0["b"], w.R, precision=precision,
                         trial_steps=16)
        tune_info = {"default_ms_per_step": t["default_ms"], "tuned_ms_per_step": t["best_ms"],
                     "gain": t["default_ms"] / t["best_ms"] if t["best_ms"] > 0 else None,
                     "choice": t["report"].splitlines()[0],
                     "timed_run_uses": "tuned schedule" if args.tuned else "default schedule"}
    step, last = make(precision)
    ms, prof, launches, clk = timed(step, args.steps, args.warmup, profile=True, clocks=True)
    value = units * world * args.steps / (ms / 1e3)
    bytes_per_unit = 12 if precision == "fp32" else 24
    avg_launch_s = (prof[0] / prof[1]) / 1e3 if prof[1] else float("nan")
    alg_bytes = total_rows * w.R * bytes_per_unit
    achieved = alg_bytes / avg_launch_s / 1e9
    traffic = committed_traffic(w.key, precision)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "kernel": step_kernel_name(w, precision), "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                "launches_timed": prof[1]}

    extra = {}
    if not args.no_fp64 and "fp64" in w.precisions and precision != "fp64" and args.fp64_steps > 0:
        step64, last64 = make("fp64")
        ms64, prof64, _, _ = timed(step64, args.fp64_steps, 1, profile=True)
        avg64 = (prof64[0] / prof64[1]) / 1e3 if prof64[1] else float("nan")
        nflip = mean_flips(w)
        flops_unit = 2 * nflip + 7
        peak64 = kpm.fp64_peak()
        extra["fp64"] = {
            "value": units * world * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
            "ms_per_step": ms64 / args.fp64_steps,
            "roofline": {"bound": "alu", "achieved": total_rows * w.R * flops_unit / avg64 / 1e12,
                         "peak": peak64["tflops"], "unit": "TFLOP/s",
                         "frac": total_rows * w.R * flops_unit / avg64 / 1e12 / peak64["tflops"],
                         "peak_source": "measured FP64 FMA rate of this GPU (kpm_fp64_peak)",
                         "hbm_gbs": total_rows * w.R * 24 / avg64 / 1e9,
                         "hbm_frac": total_rows * w.R * 24 / avg64 / 1e9 / hbm_peak,
                         "avg_launch_ms": avg64 * 1e3, "flops_per_unit": flops_unit}}
        # the FP32 form's error on C(T) and chi(T) against the FP64 form of the same pass
        th32, th64 = last["out"], last64["out"]
        err = {}
        for q in ("C", "chi"):
            d = (th32[q] - th64[q]).abs()
            ref = th64[q].abs().max()
            i = int(d.argmax())
            err[q] = {"max_abs": float(d.max()), "max_rel_to_peak": float(d.max() / ref),
                      "T_at_max": float(w.T[i])}
        err["grid"] = f"{len(w.T)}-point log grid T in [{w.T[0]:g}, {w.T[-1]:g}]"
        err["reference"] = "FP64 form of the same pass (itself within 1e-10 of the oracle)"
        extra["fp32_error"] = err

    # end to end through the public API with host buffers (copies inside the timed region)
    def e2e_step():
        bnd = kpm.bounds(w.model, w.n_up, eps=w.eps, max_iter=args.lanczos_iters,
                         tol=args.lanczos_tol, seed=w.seed)
        mom = kpm.moments(w.model, w.n_up, w.K, w.R, w.seed, a=bnd["a"], b=bnd["b"], r0=r0,
                          precision=precision, allow_ebounds=True)
        if world > 1:
            dm = combine_moments({k: torch.from_numpy(mom[k]).to(dev) for k in ("mu", "mu_M", "mu_M2")},
                                 world)
            mom.update({k: v.cpu().numpy() for k, v in dm.items()})
        secs = kpm.sector_set(w.model.n_sites, w.n_up, bnd["a"], bnd["b"], mirror)
        th = kpm.thermo(mom["mu"], mom["mu_M"], mom["mu_M2"], secs, secs_T, kernel=w.kernel)
        return th
    t_e2e, _, _, _ = timed(e2e_step, args.e2e_steps, 1)
    S, K, nT, nb = len(w.n_up), w.K, len(w.T), w.model.n_bonds
    h2d = nb * 16 + S * 4 * 2 + S * 16 * 2 + 3 * S * K * 8 + S * 16 + nT * 8
    d2h = 3 * S * K * 8 + S * 32 + 5 * nT * 8
    e2e = {"value": units * world * args.e2e_steps / (t_e2e / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": w.key, "model": w.model.name, "n_sites": w.model.n_sites,
                       "sectors": len(w.n_up), "basis_states": total_rows, "R": w.R, "K": w.K,
                       "chebyshev_steps_per_pass": w.steps, "eps": w.eps, "n_T": len(w.T),
                       "precision": ("fp32 vectors, fp64 reductions" if precision == "fp32"
                                     else "fp64 vectors and reductions"),
                       "lanczos_iters": args.lanczos_iters, "lanczos_tol": args.lanczos_tol,
                       "l2": f"vectors {2 * total_rows * w.R * bytes_per_unit // 3 / 1e9:.2f} GB "
                             "> 129 MB L2: inputs larger than L2, no flush",
                       "parallelism": f"replica x{world} (disjoint random vectors)"},
            "roofline": roofline, "clocks": clk, "gpu_launches": launches, "e2e": e2e}
    line.update(extra)
    if tune_info is not None:
        line["autotune"] = tune_info
    if not args.no_large:
        line["workloads"] = {key: large_block(args, key, timed, hbm_peak, peak_kind)
                             for key in args.large_workloads.split(",")}
    if not args.no_gradient:
        line["gradient"] = gradient_block(args, timed)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import c_oracle
        c_oracle.build()
        line["cpu_baseline"] = oracle_sample(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------- large workloads

# Fixed rescaling of the two largest workloads (their spectra lie inside): the ring
# N = 34 S^z = 0 sector in [-15.1, 8.5], the 4 x 6 J1-J2 torus in [-20, 18].  The same
# values produce the stored oracle moments the full-size tests compare against.
LARGE = {"ring34_m0": (13.0, -3.5), "j1j2sq24_full": (20.0, 0.0),
         "ring30_m0": (11.5, -3.0), "j1j2sq20_full": (17.0, 0.0)}


def large_block(args, key, timed, hbm_peak, peak_kind):
    """Throughput of the moment loop (random vectors, a block of Chebyshev steps, moment
    assembly) on one of the two largest workloads, FP32 vectors with FP64 reductions;
    the Lanczos bounds and the thermodynamics are left out (fixed a, b)."""
    import torch

    import paper_2104_13218_gb300 as kpm
    from oracle import c_oracle

    w = W.workload(key)
    a, b = LARGE[key]
    steps = args.large_steps
    K = 2 * steps
    dims = [kpm_dim(w.model.n_sites, k) for k in w.n_up]
    D = sum(dims)
    dev = torch.device("cuda", torch.cuda.current_device())
    ws = torch.empty(kpm.moments_workspace_size(w.model, w.n_up, K, w.R, "fp32"), dtype=torch.uint8,
                     device=dev)
    S = len(w.n_up)
    full = any(k < 0 for k in w.n_up)
    out = {"mu": torch.empty((S, K), dtype=torch.float64, device=dev)}
    if full:
        out.update({q: torch.empty((S, K), dtype=torch.float64, device=dev) for q in ("mu_M", "mu_M2")})

    def step():
        return kpm.moments(w.model, w.n_up, K, w.R, w.seed, a=[a] * S, b=[b] * S, precision="fp32",
                           device=True, out=out, workspace=ws, weighted=full, allow_ebounds=True)

    ms, prof, launches, clk = timed(step, args.large_reps, 1, profile=True, clocks=True)
    units = D * w.R * steps * args.large_reps
    avg = (prof[0] / prof[1]) / 1e3 if prof[1] else float("nan")
    alg = D * w.R * 12
    res = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT,
           "ms_per_chebyshev_step": ms / (steps * args.large_reps), "dtype": "f32",
           "config": {"workload": key, "note": w.note, "basis_states": D, "R": w.R,
                      "chebyshev_steps_per_block": steps, "blocks_timed": args.large_reps,
                      "a": a, "b": b,
                      "block": "random vectors + the block's Chebyshev steps + moment assembly "
                               "(bounds and thermodynamics left out: fixed a, b)",
                      "l2": f"vectors {2 * D * w.R * 4 / 1e9:.1f} GB > 129 MB L2: no flush"},
           "roofline": {"bound": "hbm", "achieved": alg / avg / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": alg / avg / 1e9 / hbm_peak, "traffic": committed_traffic(key, "fp32"),
                        "kernel": step_kernel_name(w, "fp32"),
                        "peak_source": f"{peak_kind} hbm_gbs (copy)", "alg_bytes_per_launch": alg,
                        "avg_launch_ms": avg * 1e3, "launches_timed": prof[1]},
           "clocks": clk, "gpu_launches": launches}
    del ws, out
    torch.cuda.empty_cache()
    if not args.no_autotune:
        t = kpm.autotune(w.model, w.n_up, [a] * S, [b] * S, w.R, precision="fp32", trial_steps=4)
        res["autotune"] = {"default_ms_per_step": t["default_ms"], "tuned_ms_per_step": t["best_ms"],
                           "gain": t["default_ms"] / t["best_ms"] if t["best_ms"] > 0 else None,
                           "choice": t["report"].splitlines()[0],
                           "note": "per matrix-vector product of a 5-product trial run, incl. "
                                   "random vectors and assembly"}
    # end to end through the public API with host outputs
    t0 = time.perf_counter()
    kpm.moments(w.model, w.n_up, K, w.R, w.seed, a=[a] * S, b=[b] * S, precision="fp32",
                weighted=full, allow_ebounds=True)
    t_e2e = time.perf_counter() - t0
    res["e2e"] = {"value": D * w.R * steps / t_e2e, "unit": UNIT,
                  "h2d_bytes_per_step": w.model.n_bonds * 16 + S * 20,
                  "d2h_bytes_per_step": (3 if full else 1) * S * K * 8,
                  "note": "one block through kpm_moments with host outputs; includes the "
                          "workspace allocation and the basis tables"}
    if not args.no_cpu_baseline:
        c_oracle.build()
        bi, bj, J = w.model.arrays()
        if full:
            # the two-vector C recursion, R = 1, a few steps
            n = 4
            t0 = time.perf_counter()
            c_oracle.moments_lean(w.model.n_sites, bi, bj, J, w.n_up[0], a, b, 2 * n, w.seed, 0)
            dt = time.perf_counter() - t0
            res["cpu_baseline"] = {"value": D * n / dt, "unit": UNIT, "cores": c_oracle.num_threads(),
                                   "kind": "oracle",
                                   "sample": f"{key}: C oracle two-vector recursion FP64, R = 1, "
                                             f"{n} Chebyshev steps over all {D} states, {dt:.1f} s"}
        else:
            # the state-by-state oracle's first step (v_1 = H' v_0 from the hash), R = 1,
            # on the first ranks of the sector
            n_states = 1 << 26
            t0 = time.perf_counter()
            c_oracle.local_moments(w.model.n_sites, bi, bj, J, w.n_up[0], a, b, 1, w.seed, 0,
                                   n_mom=3, max_states=n_states)
            dt = time.perf_counter() - t0
            res["cpu_baseline"] = {"value": n_states / dt, "unit": UNIT, "cores": c_oracle.num_threads(),
                                   "kind": "oracle",
                                   "sample": f"{key}: state-by-state C oracle, first step "
                                             f"(v_1 = H' v_0), R = 1, first {n_states} of {D} "
                                             f"states, {dt:.1f} s"}
    return res


def gradient_block(args, timed):
    """One forward + adjoint pass of the gradient workload (J1-J2 chain N = 24, sectors
    M = 0..12 with M > 0 mirrored, R = 32, K = 1000, FP64): loss = mean squared error of
    chi(T) on the 50-point grid against the curve at (J1, J2) = (1, 0.3), gradient at
    (1, 0.2) through kpm_thermo_backward and kpm_moments_backward (checkpoints every 32)."""
    import torch

    import paper_2104_13218_gb300 as kpm

    w = W.workload("j1j2chain24_grad")

    def spec_at(model):
        bnd = kpm.bounds(model, w.n_up, eps=w.eps, max_iter=120, tol=1e-8, seed=w.seed)
        # one-state sectors get room for the couplings to move (a is held fixed)
        return dict(model=model, n_up=w.n_up, mirror=w.mirror, a=np.maximum(bnd["a"], 0.5),
                    b=bnd["b"], K=w.K, R=w.R, seed=w.seed, T=w.T, kernel="none",
                    ckpt_interval=32)

    with torch.no_grad():
        target = kpm.chebyshev_thermo(torch.tensor([1.0, 0.3], dtype=torch.float64),
                                      spec_at(w.model.with_couplings([1.0, 0.3])))[3]
    spec = spec_at(w.model)
    keep = {}

    def forward():
        th = torch.tensor([1.0, 0.2], dtype=torch.float64)
        with torch.no_grad():
            keep["loss"] = float(((kpm.chebyshev_thermo(th, spec)[3] - target) ** 2).mean())

    def forward_backward():
        th = torch.tensor([1.0, 0.2], dtype=torch.float64, requires_grad=True)
        loss = ((kpm.chebyshev_thermo(th, spec)[3] - target) ** 2).mean()
        loss.backward()
        keep["grad"] = [float(g) for g in th.grad]

    ms_f, _, _, _ = timed(forward, 1, 0)
    ms_fb, _, launches, clk = timed(forward_backward, 1, 0)
    D = sum(kpm_dim(w.model.n_sites, k) for k in w.n_up)
    units = D * w.R * w.steps
    return {"workload": w.key, "note": w.note, "ms_forward": ms_f, "ms_forward_backward": ms_fb,
            "ms_backward": ms_fb - ms_f, "backward_over_forward": (ms_fb - ms_f) / ms_f,
            "forward_value": units / (ms_f / 1e3), "unit": UNIT, "loss": keep.get("loss"),
            "grad": keep.get("grad"), "clocks": clk, "gpu_launches": launches,
            "dtype": "f64", "ckpt_interval": 32}


def ctypes_read(L):
    import ctypes
    ms = ctypes.c_double(0)
    n = ctypes.c_int64(0)
    kl = ctypes.c_int64(0)
    L.kpm_profile_read(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(kl))
    return ms.value, n.value, kl.value


def step_kernel_name(w, precision):
    """Which step kernel the library picks for this workload: the neighbour-list
    kernel for cooperative row layouts (2+ lanes per state, 1 or 2 chunks per
    lane) with at most 4 distinct couplings, 255 bonds and a diagonal table of
    at most 4096 entries; the hi-block kernel for one-lane rows of sector runs
    with at most 4 distinct couplings and 64 bonds; the matrix-free kernel
    otherwise."""
    vw = 4 if precision == "fp32" else 2
    chunks = -(-w.R // vw)
    cpl = -(-chunks // 32)
    cpl = 8 if cpl > 4 else cpl
    G = -(-chunks // cpl)
    vals = sorted(set(w.model.J))
    table = 1
    for v in vals:
        table *= sum(1 for J in w.model.J if J == v) + 1
    grouped = len(vals) <= 4 and table <= 4096 and w.model.n_bonds > 0
    lists = G >= 2 and cpl <= 2 and grouped and w.model.n_bonds <= 255
    block = G == 1 and grouped and w.model.n_bonds <= 64 and all(k >= 0 for k in w.n_up)
    if block:
        return "cheb_block_kernel"
    return "cheb_step_list_kernel" if lists else "cheb_step_kernel"


def mean_flips(w):
    """Mean number of anti-aligned bonds per basis state over the workload's sectors."""
    n = w.model.n_sites
    tot, cnt = 0.0, 0
    for k in w.n_up:
        D = kpm_dim(n, k)
        if k < 0:
            tot += D * w.model.n_bonds * 0.5
        else:
            # a bond is anti-aligned in 2 C(N-2, k-1) of the C(N, k) states
            tot += w.model.n_bonds * 2 * math.comb(n - 2, k - 1) if 1 <= k <= n - 1 else 0.0
        cnt += D
    return tot / cnt


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
