#!/usr/bin/env python
"""Throughput benchmark of the GB300 spectral D-bar CGO solve.

Workload (default): N = 1024 on [-10pi, 10pi]^2, Q a seeded 4-Gaussian mixture,
128 values of k with |k| log-uniform in [0.1, 8]; FP32 inner GMRES with FP64
refinement to ||b - A S||/||b|| <= 1e-12.  One step = one dbar_solve_cgo call
solving all 128 k (right-hand sides, every Krylov cycle, FP64 residuals).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (launched by torchrun) every
rank solves its own copy of the workload (replicas over k, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

# one BLAS thread per caller: the serving leg generates potentials in a thread pool, and a
# multi-threaded BLAS inside each of its matrix products oversubscribes the host cores
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CGO solves/sec at N=1024^2 (rel err<=1e-10 vs FP64), %HBM roofline, p50/p99 ms"
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------------------- helpers

def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def rank_units(k, rank, world):
    """The k values rank `rank` solves: the workload's list rotated by 2 pi rank/world
    (distinct, statistically equivalent problems per GPU; weak scaling, no data-path
    collective between ranks)."""
    return np.asarray(k) * np.exp(2j * np.pi * rank / world)


def allreduce_max(x, dist, device="cpu"):
    """max over ranks of a host float (barrier-free: one all-reduce on a scalar)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def hbm_roofline(prof, variant=None, traffic_ok=False):
    """Roofline object of the dominant kernel kind of a profile_table() (largest summed
    CUDA-event time): algorithmic bytes / event time against the measured HBM copy rate.
    traffic_ok: the workload's kernels are the captured ones (headline grid), else null."""
    peak, peak_kind = peaks()
    name, (ms, launches, nbytes) = max(prof.items(), key=lambda kv: kv[1][0])
    achieved = nbytes / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    return {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": ncu_traffic(name, nbytes / max(launches, 1), variant=variant) if traffic_ok else None,
            "algorithmic_bytes_per_launch": nbytes / max(launches, 1), "avg_launch_ms": ms / max(launches, 1),
            "kinds": {k: {"ms": round(v[0], 3), "launches": v[1],
                          "GBs": round(v[2] / (v[0] / 1e3) / 1e9, 1) if v[0] > 0 else 0.0}
                      for k, v in prof.items() if v[1]}}


def fp64_column_roofline(kind, N, M):
    """FP64 arithmetic roofline of the FP64 column pass (its bound: FP64 runs at 1/64 of
    FP32 here).  Elements per launch from the profiler's algorithmic bytes (2 F64 per
    slot and step, plus the (M+2) F64 tables per launch); algorithmic flops per element:
    two length-N FFTs at the textbook 5 log2 N each, the Delta_n sum 8(M+1) and the
    product E_k Q conj(h) 12.  FFT additions issue on the FP64 pipe like FMAs but count
    one flop, so 1.0 is out of reach even at a saturated pipe."""
    import math
    ms, launches, nbytes = kind
    f64 = 16.0 * N * N
    elems = max(nbytes - launches * (M + 2) * f64, 0.0) / (2.0 * f64) * N * N
    flop = elems * (10.0 * math.log2(N) + 8.0 * (M + 1) + 12.0)
    peak = N_SM * FP64_FLOP_PER_CLK_SM * 2070e6 / 1e12
    achieved = flop / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": "inner_pass_b_cols (FP64)", "achieved": round(achieved, 4),
            "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz",
            "flop_per_launch": flop / max(launches, 1), "avg_launch_ms": ms / max(launches, 1),
            "flop_model": "per element and step: 2 x 5 log2 N (FFTs) + 8 (M+1) (Delta_n sum) + 12 (product)"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources of the solve's kernels and of their launchers (grid shapes): the captured
# DRAM counters of those kernels stay valid while these files are unchanged.  The plan's
# driver (which kernels run in which order), the convolution route, the allocation-free
# DFT entry point and the serving runtime are not part of it.
DIGEST_SOURCES = ("cx.cuh", "types.cuh", "passes.cuh", "krylov.cuh", "launch.cuh", "kern_pass.cu",
                  "kern_krylov.cu", "dispatch.cu")


def source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1508_02363_gb300", "csrc")
    for f in DIGEST_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kind, algorithmic_bytes_per_launch, variant=None):
    """DRAM bytes per launch of `kind`: the DRAM/algorithmic ratio measured by ncu on a
    smaller capture of the same kernel (profiles/ncu_traffic.json; per tile variant where
    the kind has several) times this launch's algorithmic bytes, if the capture was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        if d.get("source_digest") != source_digest():
            return None
        entry = d.get("kinds", {}).get(kind, {})
        ratio = entry.get("dram_over_algorithmic")
        if variant is not None and "variants" in entry:
            ratio = entry["variants"].get(str(variant))
        return None if ratio is None else round(ratio * algorithmic_bytes_per_launch)
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle

def _oracle_solve(args):
    N, L, M, tol, Q, k = args
    from oracle import dbar_oracle as orc
    r = orc.solve_cgo(Q, k, N, L, M=M, tol=tol, restart=40)
    return r["iters"], r["resid"], r["S"]


def cpu_oracle_step(w, ks, cores):
    """Solve len(ks) k values with the CPU oracle, one per process, in parallel."""
    ctx = mp.get_context("spawn")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("MKL_NUM_THREADS", "1")
    with ctx.Pool(processes=min(cores, len(ks))) as pool:
        t0 = time.perf_counter()
        out = pool.map(_oracle_solve, [(w.N, w.L, w.M, w.tol, w.Q, complex(k)) for k in ks])
        dt = time.perf_counter() - t0
    return dt, out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02363_gb300 import dbar
    import workloads as wl

    w = wl.BY_NAME[args.workload]()
    nk, N = w.k.size, w.N
    if args.nk:
        w.k = w.k[:args.nk]
    w.k = rank_units(w.k, rank, world)
    nk = w.k.size
    plan = dbar.Plan(N, w.L, M=w.M, prec="mixed" if w.mixed else "fp64", tol=w.tol, restart=args.restart,
                     inner_tol=args.inner_tol, max_batch=nk, max_outer=args.max_outer, sstep=args.sstep,
                     autotune=args.autotune, row_shape=args.row_shape, row_shape_plain=args.row_shape_plain)
    colv, tune = dbar.dbar_plan_tuning(plan.handle)
    rowv, rtune = dbar.dbar_plan_row_tuning(plan.handle)
    rowv_ac, rtune_ac = dbar.dbar_plan_row_tuning(plan.handle, "plain")
    stream = torch.cuda.current_stream()
    Qd = torch.from_numpy(w.Q).cuda()
    Sd = torch.empty((nk, N, N), dtype=torch.complex128, device="cuda")

    def step():
        return plan.solve_device(Qd, w.k, Sd, stream=stream)

    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()
    barrier()
    dbar.dbar_profile(plan.handle, True)
    launches0 = dbar.dbar_launch_count(plan.handle)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    results = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        evs[0].record(stream)
        for i in range(args.steps):
            results.append(step())
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = dbar.dbar_launch_count(plan.handle) - launches0
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    prof = dbar.profile_table(plan.handle)
    dbar.dbar_profile(plan.handle, False)
    total_ms = allreduce_max(total_ms, dist, device="cuda")
    ms_per_step = total_ms / args.steps
    value = nk * world * args.steps / (total_ms / 1e3)
    last = results[-1]
    iters = last["iters"]
    resid = last["resid"]
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "workload": w.name, "nk": nk, "ms_per_step": ms_per_step,
                              "solves_per_s": value, "iters_inner_mean": float(np.mean(iters[:, 0])),
                              "resid_max": float(np.max(resid)), "gpu_launches": int(launches),
                              "column_variant": colv, "row_shape": rowv, "row_shape_plain": rowv_ac,
                              "kinds": {k: [round(v[0], 3), v[1], round(v[2] / (v[0] / 1e3) / 1e9, 1)
                                            if v[0] > 0 else 0] for k, v in prof.items()}}))
        return

    # error of the mixed results against the plain FP64 GPU solve, per sampled k,
    # and the plain single-k FP64 solve rate on the same GPU
    sample = np.unique(np.linspace(0, nk - 1, min(nk, args.check_k)).astype(int))
    p64 = dbar.Plan(N, w.L, M=w.M, prec="fp64", tol=min(w.tol, 1e-13), restart=args.restart, max_batch=len(sample))
    S64 = torch.empty((len(sample), N, N), dtype=torch.complex128, device="cuda")
    p64.solve_device(Qd, w.k[sample], S64, stream=stream)
    torch.cuda.synchronize()
    errs = []
    for j, i in enumerate(sample):
        d = (Sd[i] - S64[j]).abs().max().item() / S64[j].abs().max().item()
        errs.append(d)
    p1 = dbar.Plan(N, w.L, M=w.M, prec="fp64", tol=w.tol, restart=args.restart, max_batch=1)
    S1 = torch.empty((1, N, N), dtype=torch.complex128, device="cuda")
    p1.solve_device(Qd, w.k[:1], S1, stream=stream)  # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    nrep = 3
    for _ in range(nrep):
        p1.solve_device(Qd, w.k[:1], S1, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_single_rate = nrep / (e0.elapsed_time(e1) / 1e3)

    # the same workload with the refinement's residual and right-hand side in native FP64
    # (resid_mode = fp64) instead of double-float: its rate, and its solutions for the
    # oracle comparison below
    S64r = None
    if w.mixed and not args.no_fp64_resid:
        pr = dbar.Plan(N, w.L, M=w.M, prec="mixed", tol=w.tol, restart=args.restart, inner_tol=args.inner_tol,
                       max_batch=nk, max_outer=args.max_outer, sstep=args.sstep, autotune=args.autotune,
                       resid_mode="fp64")
        S64r = torch.empty_like(Sd)
        pr.solve_device(Qd, w.k, S64r, stream=stream)   # warm
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        nrep_r = 2
        for _ in range(nrep_r):
            r64r = pr.solve_device(Qd, w.k, S64r, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_resid = {"solves_per_s": round(nrep_r * nk / (e0.elapsed_time(e1) / 1e3), 3),
                      "resid_max": float(np.max(r64r["resid"])),
                      "iters_inner_mean": float(np.mean(r64r["iters"][:, 0]))}
        pr.close()
        del pr

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Qh = torch.from_numpy(w.Q).pin_memory()
    Sh = torch.empty((nk, N, N), dtype=torch.complex128).pin_memory()
    kh = np.ascontiguousarray(w.k)
    e2e_steps = max(1, args.steps)
    plan.solve(Qh.numpy(), kh, want_m=False)  # warm the host path
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dbar.dbar_solve_cgo(plan.handle, Qh.numpy(), kh, Sh.numpy(), None, None, None, io_on_device=False,
                            stream=stream)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": nk / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(Qh.numel() * 16 + kh.size * 16),
           "d2h_bytes_per_step": int(Sh.numel() * 16)}

    # roofline of the dominant kernel kind
    peak, peak_kind = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_launches, dom_bytes) = dom
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    traffic = ncu_traffic(dom_name, dom_bytes / max(dom_launches, 1), variant=colv)
    all_bytes = sum(v[2] for v in prof.values())
    all_ms = sum(v[0] for v in prof.values())
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic,
                "algorithmic_bytes_per_launch": dom_bytes / max(dom_launches, 1),
                "avg_launch_ms": dom_ms / max(dom_launches, 1),
                "whole_step": {"bytes_per_step": all_bytes / args.steps,
                               "gbs_over_kernel_time": round(all_bytes / (all_ms / 1e3) / 1e9, 1) if all_ms else 0,
                               "gbs_over_step_time": round(all_bytes / args.steps / (ms_per_step / 1e3) / 1e9, 1),
                               "frac_of_peak_over_step_time": round(
                                   all_bytes / args.steps / (ms_per_step / 1e3) / 1e9 / peak, 4)},
                "kinds": {k: {"ms": round(v[0], 3), "launches": v[1], "GBs": round(v[2] / (v[0] / 1e3) / 1e9, 1)
                              if v[0] > 0 else 0.0} for k, v in prof.items()}}

    out = {"metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           # mixed: FP32 inner GMRES; right-hand side, true residual, x and b in double-float
           # (float pairs, ~48-bit significand); read-out to FP64
           "dtype": "f32+df32x2" if w.mixed else "f64",
           "data": "synthetic (seeded Gaussian-mixture potential and k list)",
           "config": {"workload": w.name, "N": N, "L": w.L, "nk": nk, "M": w.M, "tol": w.tol,
                      "prec": "mixed" if w.mixed else "fp64", "restart": args.restart, "sstep": args.sstep,
                      "inner_tol": args.inner_tol,
                      "column_variant": colv, "column_tune_ms": [round(x, 4) for x in tune],
                      "row_shape": rowv, "row_tune_ms": [round(x, 4) for x in rtune],
                      "row_shape_plain": rowv_ac, "row_tune_ms_plain": [round(x, 4) for x in rtune_ac],
                      "parallelism": f"replicas over k x{world}",
                      "l2": "inputs larger than L2 (device working set %.1f GB)" % (plan.device_bytes / 1e9)},
           "step_p50_ms": round(statistics.median(step_ms), 3),
           "step_p99_ms": round(float(np.percentile(step_ms, 99)), 3),
           "iters_inner_mean": float(np.mean(iters[:, 0])), "cycles_max": int(np.max(iters[:, 1])),
           "resid_max": float(np.max(resid)), "err_vs_fp64_max": float(max(errs)),
           "err_vs_fp64_sampled_k": [int(i) for i in sample],
           "fp64_plain_single_k_solves_per_s": round(fp64_single_rate, 3),
           "fp64_plain_single_k_latency_ms": round(1e3 / fp64_single_rate, 3),
           "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "clocks": clk.summary()}
    if not w.mixed and prof.get("inner_pass_b_cols", (0, 0, 0))[0] > 0:
        out["roofline_fp64_alu"] = fp64_column_roofline(prof["inner_pass_b_cols"], N, w.M)

    if w.mixed and S64r is not None:
        out["fp64_resid"] = fp64_resid
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        ncpu = min(cores, args.cpu_sample)
        idx = np.linspace(0, nk - 1, ncpu).astype(int)
        ks = w.k[idx]
        dt, res = cpu_oracle_step(w, ks, cores)
        out["cpu_baseline"] = {"value": round(len(ks) / dt, 4), "unit": "solves/s", "cores": min(cores, len(ks)),
                               "kind": "oracle",
                               "sample": f"{len(ks)} of the {nk} k values solved once each by the FP64 CPU "
                                         f"oracle, one process per core, wall {dt:.1f} s"}
        # the headline's accuracy: the timed solutions against the oracle's, element by element
        def err_vs(Sx):
            return float(max(np.max(np.abs(Sx[i].cpu().numpy() - So)) / np.max(np.abs(So))
                             for i, (_, _, So) in zip(idx, res)))
        out["err_vs_oracle_max"] = err_vs(Sd)
        out["err_vs_oracle_sampled_k"] = [int(i) for i in idx]
        if S64r is not None:
            out["fp64_resid"]["err_vs_oracle_max"] = err_vs(S64r)
    if rank == 0 and world == 1 and not args.no_serving and args.workload == "mixed_1024":
        # request-level latency under continuous batching (the metric's p50/p99), with the
        # plain single-k FP64 solve's latency beside it
        plan.close()
        p64.close()
        p1.close()
        del Sd, S64, S1, Sh, Qh, S64r
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        sv = serving_leg(args, dbar, torch, local)
        out["serving"] = sv
        out["p50_ms"], out["p99_ms"] = sv["p50_ms"], sv["p99_ms"]
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- uneven batch

def run_uneven(args):
    """1000 mixed-size solves grouped by (N, potential), one plan per N.  One timed call
    of dbar_solve_batches per pass: the groups of different grid sizes run at the same
    time (one host thread and CUDA stream per plan), the groups of one plan in order.
    Throughput = solves / device-synchronised wall time of the call; the same groups
    solved one call after another are timed beside it."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02363_gb300 import dbar
    import workloads as wl

    L = 4.0
    reqs = wl.uneven_batch(n=args.nreq, L=L)
    groups = {}
    for idx, (N, pot, k) in enumerate(reqs):
        groups.setdefault((N, pot), []).append((idx, k))
    stream = torch.cuda.current_stream()
    plans, pots = {}, {}
    for (N, pot) in groups:
        if N not in plans:
            nmax = max(len(v) for (n2, _), v in groups.items() if n2 == N)
            plans[N] = dbar.Plan(N, L, prec="mixed", restart=args.restart, sstep=args.sstep, tol=1e-12,
                                 inner_tol=args.inner_tol,
                                 max_batch=min(nmax, 256 if N <= 1024 else 64), autotune=int(args.autotune))
            pots[N] = [torch.from_numpy(q).cuda() for q in wl.uneven_potentials(N, L)]
    outS = {key: torch.empty((len(v), key[0], key[0]), dtype=torch.complex128, device="cuda")
            for key, v in groups.items()}
    # largest grids first: their long launches start while the small grids fill in around them
    order = sorted(groups, key=lambda g: -g[0] * g[0] * len(groups[g]))
    batch = [{"plan": plans[N].handle, "Q": pots[N][pot], "k": np.array([kk for _, kk in groups[(N, pot)]]),
              "S_out": outS[(N, pot)]} for (N, pot) in order]

    def one_call():
        return dbar.dbar_solve_batches(batch, stream=stream)

    def one_serial():
        for (N, pot), bt in zip(order, batch):
            plans[N].solve_device(bt["Q"], bt["k"], bt["S_out"], stream=stream)

    for _ in range(args.warmup):
        one_call()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st, sts, iters, resid = one_call()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / args.steps * 1e3
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_serial()
    torch.cuda.synchronize()
    ms_serial = (time.perf_counter() - t0) / args.steps * 1e3
    resid_max = max(float(np.max(r)) for r in resid)
    # error vs the plain FP64 GPU solve on a sample of one request per group
    errs = []
    for (N, pot), bt in zip(order, batch):
        p64 = dbar.Plan(N, L, prec="fp64", restart=args.restart, tol=1e-13, max_batch=1)
        ref = p64.solve(pots[N][pot].cpu().numpy(), bt["k"][:1], want_m=False)["S"][0]
        got = outS[(N, pot)][0].cpu().numpy()
        errs.append(float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
        p64.close()
    out = {"metric": "uneven batch: CGO solves/sec over mixed grid sizes", "workload": "uneven",
           "solves": len(reqs), "ms_per_pass": round(ms, 2), "solves_per_s": round(len(reqs) / (ms / 1e3), 2),
           "one_call_per_pass": "dbar_solve_batches (groups of different N concurrently)",
           "ms_per_pass_serial": round(ms_serial, 2),
           "solves_per_s_serial": round(len(reqs) / (ms_serial / 1e3), 2),
           "status_ok": bool(st == dbar.DBAR_OK and all(x == dbar.DBAR_OK for x in sts)),
           "resid_max": resid_max, "err_vs_fp64_max": max(errs), "err_sample": len(errs),
           "groups": {f"{N}/{'ab'[pot]}": len(v) for (N, pot), v in sorted(groups.items())},
           "autotune": bool(args.autotune),
           "tiles": {str(N): dict(zip(("column_variant", "ms_per_variant", "row_shape", "ms_per_row_shape",
                                       "row_shape_plain", "ms_per_row_shape_plain"),
                                      dbar.dbar_plan_tuning(p.handle) + dbar.dbar_plan_row_tuning(p.handle)
                                      + dbar.dbar_plan_row_tuning(p.handle, "plain")))
                     for N, p in sorted(plans.items())},
           "config": {"L": L, "kmax": 12.0, "restart": args.restart, "inner_tol": args.inner_tol},
           "clocks": clk.summary()}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- reflection workload

def run_reflection(args):
    """DS II reflection coefficient r(k) over the resolved k-grid of Sec. 6's example
    (q = exp(-(x^2+y^2)), N = 128, L = 3.2, M = 11): 2401 values of k, two CGO solves
    each, all slots of one sign in one batch.  Throughput = r values / device time."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02363_gb300 import dbar
    import workloads as wl

    N, L = 128, 3.2
    Q, k, M = wl.reflection_grid(N, L, full=args.iterated)
    Qd = torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream()
    if args.iterated:   # Sec. 5.3 route: one solve per k, every k of the xi-grid
        plan = dbar.Plan(N, L, M=M, prec="mixed", tol=1e-12, restart=16, iterated=1, inner_tol=args.inner_tol,
                         max_batch=min(k.size, 4096), sstep=args.sstep, inner_M=args.inner_m)
    else:               # Sec. 4 route: two solves per k, the k the grid resolves
        plan = dbar.Plan(N, L, M=M, prec="mixed", tol=1e-12, restart=args.restart, sstep=args.sstep,
                         inner_tol=args.inner_tol, max_batch=k.size, inner_M=args.inner_m)
    for _ in range(args.warmup):
        dbar.dbar_reflection(plan.handle, Qd, k, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dbar.dbar_profile(plan.handle, True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            r, iters, resid, status = dbar.dbar_reflection(plan.handle, Qd, k, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    roofline = hbm_roofline(dbar.profile_table(plan.handle))
    dbar.dbar_profile(plan.handle, False)
    ms = e0.elapsed_time(e1) / args.steps
    # sampled parity against the FP64 GPU path (same entry point, FP64 plan) and the Born-free
    # CPU oracle on a few k (host cores, spawned pool)
    sample = np.linspace(0, k.size - 1, 6).astype(int)
    p64 = dbar.Plan(N, L, M=M, prec="fp64", tol=1e-13, max_batch=len(sample), iterated=int(args.iterated))
    r64 = dbar.dbar_reflection(p64.handle, Q, k[sample])[0]
    scale = float(np.max(np.abs(r)))
    err64 = float(np.max(np.abs(r[sample] - r64)) / scale)
    per_r = 1 if args.iterated else 2
    out = {"metric": "DS II reflection coefficient: r(k) values/s over the k-grid",
           "workload": "reflection", "route": "iterated equation (Sec. 5.3), one solve per k, whole xi-grid"
           if args.iterated else "Sec. 4 equation, two solves per k, the k the grid resolves",
           "N": N, "L": L, "M": M, "inner_M": args.inner_m or M, "nk": int(k.size),
           "ms_per_grid": round(ms, 2), "r_per_s": round(k.size / (ms / 1e3), 1),
           "solves_per_s": round(per_r * k.size / (ms / 1e3), 1),
           "iters_inner_mean_per_r": float(np.mean(iters[:, 0])), "resid_max": float(np.max(resid)),
           "status_ok": bool(status == dbar.DBAR_OK), "err_vs_fp64_gpu_max": err64,
           "err_sample_k": [complex(x).__repr__() for x in k[sample]],
           "max_abs_r": scale, "roofline": roofline, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        from oracle import dbar_oracle as orc
        t0 = time.perf_counter()
        fn = orc.reflection_iterated if args.iterated else orc.reflection
        ro = [fn(Q, kk, N, L, M=M, tol=1e-13)["r"] for kk in k[sample[:2]]]
        dt = time.perf_counter() - t0
        out["err_vs_oracle_max"] = float(np.max(np.abs(r[sample[:2]] - np.array(ro))) / scale)
        out["cpu_baseline"] = {"value": round(2 / dt, 4), "unit": "r/s", "cores": 1, "kind": "oracle",
                               "sample": f"r at 2 of the {k.size} k by the FP64 CPU oracle on one core, {dt:.1f} s"}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- DS II round trip workload

def run_ds2(args):
    """Sec. 6.2: q(x,y,0) = exp(-x^2-y^2) -> r(k) on the whole k-grid (one iterated solve per k)
    -> q on the whole x-grid (one iterated solve per point), at the paper's (N, L) = (128, 3.2)
    and (256, 4.2), M = 11; the reconstruction error against q and the paper's printed error,
    and q at t = 0.1 (eq. rt) with its L2 norm (conserved by DS II)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02363_gb300 import dbar
    import workloads as wl

    table = json.load(open(os.path.join(ROOT, "tests", "golden", "ds2_reconstruction.json")))
    M = table["M"]
    stream = torch.cuda.current_stream()
    rows = []
    for N, L, err_paper in table["rows"][4:]:
        X, Y = wl.mesh(N, L)
        q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
        Lp = N / (2.0 * np.pi * L)
        j = np.arange(N)
        kg = Lp * (-np.pi + 2.0 * np.pi * j / N)
        K1, K2 = np.meshgrid(kg, kg, indexing="xy")
        k = (K1 + 1j * K2).ravel()
        z = (X + 1j * Y).ravel()
        mb = min(N * N, 4096)
        kw = dict(M=M, prec=args.ds2_prec, iterated=1, restart=16, tol=args.ds2_tol, max_batch=mb,
                  inner_M=args.inner_m if args.ds2_prec == "mixed" else 0)
        fwd, inv = dbar.Plan(N, L, **kw), dbar.Plan(N, Lp, **kw)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        dbar.dbar_profile(fwd.handle, True)
        e[0].record(stream)
        r, it_r, res_r, st_r = dbar.dbar_reflection(fwd.handle, q, k, stream=stream)
        e[1].record(stream)
        torch.cuda.synchronize()
        roofline = hbm_roofline(dbar.profile_table(fwd.handle))
        dbar.dbar_profile(fwd.handle, False)
        qr, it_q, res_q, st_q = dbar.dbar_ds2_potential(inv.handle, r.reshape(N, N), z, stream=stream)
        e[2].record(stream)
        qt = dbar.dbar_ds2_potential(inv.handle, r.reshape(N, N), z, t=0.1, stream=stream)[0]
        e[3].record(stream)
        torch.cuda.synchronize()
        routes = None
        if args.ds2_routes:
            # remark of Sec. 6 (time dependence): q(., t) from the same r through the Sec. 4 route
            # (two solves per point) against the iterated route, L-infinity difference
            direct = dbar.Plan(N, Lp, M=M, prec=args.ds2_prec, restart=32, tol=args.ds2_tol, max_batch=mb,
                               inner_M=kw["inner_M"])
            routes = {}
            for tt in (0.1, 0.8):
                qi = dbar.dbar_ds2_potential(inv.handle, r.reshape(N, N), z, t=tt, stream=stream)[0]
                qd = dbar.dbar_ds2_potential(direct.handle, r.reshape(N, N), z, t=tt, stream=stream)[0]
                routes[f"t{tt}"] = float(np.max(np.abs(qi - qd)))
            direct.close()
        err = float(np.max(np.abs(qr.reshape(N, N) - q)))
        rows.append({"N": N, "L": L, "solves": 3 * N * N, "ms_r": round(e[0].elapsed_time(e[1]), 1),
                     "ms_q": round(e[1].elapsed_time(e[2]), 1), "ms_q_t": round(e[2].elapsed_time(e[3]), 1),
                     "err_reconstruction": err, "err_paper": err_paper,
                     "iters_mean": float(np.mean(np.concatenate([it_r[:, 0], it_q[:, 0]]))),
                     "resid_max": float(max(np.max(res_r), np.max(res_q))),
                     "status_ok": bool(st_r == dbar.DBAR_OK and st_q == dbar.DBAR_OK),
                     "l2_ratio_t0.1": float(np.linalg.norm(qt) / np.linalg.norm(qr)),
                     "route_difference": routes, "roofline_r_direction": roofline})
        if N == table["rows"][4][0] and not args.no_cpu_baseline:
            # the FP64 CPU oracle on two points of q (one iterated solve each), from the GPU's r
            from oracle import dbar_oracle as orc
            t0 = time.perf_counter()
            pts = [(N // 2, N // 2), (N // 3, 2 * N // 3)]
            qo = [orc.ds2_potential(r.reshape(N, N), X[a, b] + 1j * Y[a, b], N, L, M=M, tol=1e-13) for a, b in pts]
            dt = time.perf_counter() - t0
            rows[-1]["cpu_baseline"] = {"value": round(len(pts) / dt, 4), "unit": "q values/s", "cores": 1,
                                        "kind": "oracle",
                                        "sample": f"q at 2 of the {N * N} points by the FP64 CPU oracle on one core, "
                                                  f"{dt:.1f} s"}
            rows[-1]["err_vs_oracle_max"] = float(max(abs(qr.reshape(N, N)[a, b] - v) for (a, b), v in zip(pts, qo)))
        fwd.close()
        inv.close()
    out = {"metric": "DS II round trip q -> r -> q over whole grids (Sec. 6.2), error vs the paper's table",
           "workload": "ds2", "M": M, "inner_M": args.inner_m if args.ds2_prec == "mixed" else M,
           "prec": args.ds2_prec, "tol": args.ds2_tol, "rows": rows}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- convolution regularisation

FP64_FLOP_PER_CLK_SM = 4.0   # 2 FP64 FMAs per clock per SM (the 1.25 TFLOP/s nominal at 152 SMs, 2.07 GHz)
N_SM = 152


def _conv_oracle(args):
    Q, k, N, L = args
    from oracle import dbar_oracle as orc
    t0 = time.perf_counter()
    r = orc.solve_cgo_conv(Q, k, N, L, tol=1e-13, restart=40)
    return time.perf_counter() - t0, r["S"]


def run_conv(args):
    """The convolution regularisation G = S e^{-|xi|^2} (Sec. 4.2, remark after eq. fourreg5a):
    a batch of FP64 CGO solves whose F^{-1}(G/xi) is the direct N^4 grid sum, the paper's
    independent test of the Taylor-Gaussian code.  N = 128, L = 5 (the box the smooth
    remainder needs), q = exp(-(x^2+y^2)), 64 k on the disc |k| <= 2.  Reports solves/s, the
    direct sum's FP64 roofline, and the agreement with the Taylor route (M = 11) on the same k."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02363_gb300 import dbar
    import workloads as wl

    N, L, nk = 128, 5.0, 64
    X, Y = wl.mesh(N, L)
    Q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
    k = wl.random_k_disc(np.random.default_rng(args.seed), nk, 2.0)
    Qd = torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream()
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", tol=1e-13, restart=16, max_batch=nk)
    Sd = torch.empty((nk, N, N), dtype=torch.complex128, device="cuda")
    for _ in range(args.warmup):
        r = plan.solve_device(Qd, k, Sd, stream=stream)
    torch.cuda.synchronize()
    dbar.dbar_profile(plan.handle, True)
    launches0 = dbar.dbar_launch_count(plan.handle)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        evs[0].record(stream)
        for i in range(args.steps):
            r = plan.solve_device(Qd, k, Sd, stream=stream)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    launches = dbar.dbar_launch_count(plan.handle) - launches0
    prof = dbar.profile_table(plan.handle)
    dbar.dbar_profile(plan.handle, False)
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    ms = sum(step_ms) / args.steps
    cms, claunch, cflop = prof["conv_direct_sum"]
    csum = clk.summary()
    peak_max = N_SM * FP64_FLOP_PER_CLK_SM * 2070e6 / 1e12
    achieved = cflop / (cms / 1e3) / 1e12 if cms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": "conv_direct_sum (k_conv_sum<1>, FP64 FMA pipe)",
                "achieved": round(achieved, 4), "peak": round(peak_max, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak_max, 4),
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz",
                "frac_at_median_clock": round(achieved / (N_SM * FP64_FLOP_PER_CLK_SM * csum["sm_mhz"] / 1e6), 4)
                if csum.get("sm_mhz") else None,
                "traffic": None, "flop_per_launch": cflop / max(claunch, 1), "avg_launch_ms": cms / max(claunch, 1),
                "share_of_step": round(cms / args.steps / ms, 4),
                "kinds": {kk: {"ms": round(v[0], 3), "launches": v[1]} for kk, v in prof.items() if v[1]}}
    S_conv = Sd.cpu().numpy()
    # the same k through the Taylor-Gaussian route (M = 11): FP64 and the mixed default
    cross = {}
    for prec in ("fp64", "mixed"):
        tp = dbar.Plan(N, L, M=11, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12, max_batch=nk)
        St = torch.empty_like(Sd)
        tp.solve_device(Qd, k, St, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tp.solve_device(Qd, k, St, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        St = St.cpu().numpy()
        d = max(float(np.max(np.abs(S_conv[i] - St[i])) / np.max(np.abs(St[i]))) for i in range(nk))
        cross[prec] = {"solves_per_s": round(nk / (e0.elapsed_time(e1) / 1e3), 1), "max_rel_diff_S": d}
        tp.close()
    out = {"metric": "convolution regularisation (Sec. 4.2 remark): FP64 CGO solves/sec, direct N^4 sum",
           "workload": "conv", "value": round(nk / (ms / 1e3), 3), "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
           "dtype": "f64", "data": "synthetic (q = exp(-(x^2+y^2)), seeded k on |k| <= 2)",
           "config": {"workload": "conv", "N": N, "L": L, "nk": nk, "tol": 1e-13, "restart": 16,
                      "l2": "working set %.2f GB (fits in L2: the direct sum is FP64-bound)"
                            % (plan.device_bytes / 1e9)},
           "iters_inner_mean": float(np.mean(r["iters"][:, 0])), "resid_max": float(np.max(r["resid"])),
           "taylor_route_same_k": cross, "gpu_launches": int(launches), "roofline": roofline, "clocks": csum}
    if not args.no_cpu_baseline:
        import multiprocessing as mp
        ks = k[:2]
        with mp.get_context("spawn").Pool(2) as pool:
            t0 = time.perf_counter()
            res = pool.map(_conv_oracle, [(Q, kk, N, L) for kk in ks])
            wall = time.perf_counter() - t0
        err = max(float(np.max(np.abs(S_conv[i] - res[i][1])) / np.max(np.abs(res[i][1]))) for i in range(2))
        out["cpu_baseline"] = {"value": round(len(ks) / wall, 4), "unit": "solves/s", "cores": 2, "kind": "oracle",
                               "sample": f"2 of the {nk} k solved by the CPU oracle (direct sum by numpy einsum), "
                                         f"one process each, wall {wall:.1f} s"}
        out["err_vs_oracle_max"] = err
    print(json.dumps(out))


# ----------------------------------------------------------------------------- serving workload

def _oracle_serving(args):
    N, L, mixture, k = args
    import workloads as wl
    from oracle import dbar_oracle as orc
    r = orc.solve_cgo(wl.gaussian_mixture(N, L, *mixture), k, N, L, M=2, tol=1e-13, restart=40)
    return r["S"]


def serving_leg(args, dbar, torch, clock_gpu=0):
    """Poisson arrivals of CGO requests into the continuous-batching server.

    Request i is drawn from default_rng(seed + i) (workloads.serving_request): N uniform
    over {256, 512, 1024, 2048}, raised to the smallest size that resolves its k
    (N/(2L) >= 2 max(|k1|,|k2|) + 20, L = 6); its own Gaussian mixture of 1-6 terms;
    |k| log-uniform in [0.1, 20].  Each potential is generated on the host just ahead of
    its arrival by a thread pool (one matrix product of separable factors), submitted at
    its arrival time (the server copies it), and its result released as soon as it is
    done.  Device memory is admitted by the server's budget.  2 % of the requests (every
    50th) are checked against the plain FP64 GPU solve, and those of them with N <= 512
    (at most `serve_oracle`) against the FP64 CPU oracle (solved in a spawned process
    pool; larger grids take the oracle minutes per solve)."""
    import concurrent.futures as cf
    import workloads as wl

    L, XI_Q, KMAX = 6.0, 20.0, 20.0
    arrivals = wl.poisson_arrivals(args.rate, args.duration, seed=args.seed)
    reqs = [wl.serving_request(i, base_seed=args.seed, L=L, kmax=KMAX, xi_q=XI_Q) for i in range(arrivals.size)]
    sampled = set(range(0, len(reqs), 50))
    free = torch.cuda.mem_get_info()[0]
    srv = dbar.Server(int(free * 0.7), prec="mixed", restart=args.restart, tol=1e-12, inner_tol=args.inner_tol,
                      max_batch=args.serve_batch)
    gen = cf.ThreadPoolExecutor(max_workers=6)
    LOOK = 64
    kept_Q, kept_S = {}, {}

    queue, cycles = [], []  # per request of the last stream, in submission order

    def stream(arr, rq, keep):
        """Submits rq[i] at arr[i] (generated just ahead by the pool), collects and releases each
        result as it completes; keeps Q and S of the requests in `keep`.  Returns the latencies,
        statuses and residuals in submission order, the wall time from the first submission to
        the last completion, and the number of submissions more than 5 ms late."""
        futs, lat, status, resid, tickets = {}, [], [], [], []
        del queue[:], cycles[:]
        ready = threading.Condition()
        late = [0]

        def generate(i):
            N, k, mix = rq[i]
            return wl.gaussian_mixture(N, L, *mix)

        def collect():
            # results in completion order (a polling client): each one's page-locked
            # buffers go back to the server's pool as soon as it is done, not after the
            # slower requests submitted before it
            j, pending, got, last = 0, {}, {}, False
            while not last or pending:
                with ready:
                    while j >= len(tickets) and not pending:
                        ready.wait()
                    while j < len(tickets):
                        if tickets[j] is None:
                            last = True
                        else:
                            pending[tickets[j][0]] = tickets[j][1]
                        j += 1
                done = []
                for i, t in pending.items():
                    r = srv.poll(t, copy=i in keep)
                    if r is None:
                        continue
                    srv.release(t)
                    got[i] = (r["latency_ms"], r["status"], r["resid"], r["queue_ms"], r["cycles"])
                    if i in keep:
                        kept_S[i] = r["S"]
                    done.append(i)
                for i in done:
                    del pending[i]
                if not done:
                    time.sleep(0.001)
            for i in sorted(got):  # submission order
                lat.append(got[i][0])
                status.append(got[i][1])
                resid.append(got[i][2])
                queue.append(got[i][3])
                cycles.append(got[i][4])

        collector = threading.Thread(target=collect, daemon=True)
        collector.start()
        for i in range(min(LOOK, len(rq))):
            futs[i] = gen.submit(generate, i)
        t0 = time.perf_counter()
        for i, ta in enumerate(arr):
            if i + LOOK < len(rq):
                futs[i + LOOK] = gen.submit(generate, i + LOOK)
            Q = futs.pop(i).result()
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            elif dt < -0.005:
                late[0] += 1
            N, k, _ = rq[i]
            t = srv.submit(N, L, Q, k)
            if i in keep:
                kept_Q[i] = Q
            with ready:
                tickets.append((i, t))
                ready.notify()
        with ready:
            tickets.append(None)
            ready.notify()
        collector.join()
        return lat, status, resid, time.perf_counter() - t0, late[0]

    # warm-up: a few seconds of the same kind of traffic (other requests), not counted, so
    # that the measured stream sees the server in its steady state (lanes and plans built,
    # page-locked host buffers allocated)
    if args.serve_warmup > 0:
        warr = wl.poisson_arrivals(args.rate, args.serve_warmup, seed=args.seed + 1)
        wreq = [wl.serving_request(10_000_000 + i, base_seed=args.seed, L=L, kmax=KMAX, xi_q=XI_Q)
                for i in range(warr.size)]
        stream(warr, wreq, set())
    with ClockSampler(clock_gpu) as clk:
        lat, status, resid, wall, late = stream(arrivals, reqs, sampled)
    gen.shutdown()
    srv.close()
    torch.cuda.empty_cache()
    # checks: the oracle on the sampled requests with N <= 512 (spawned pool, CPU), while the
    # GPU solves every sampled request with a plain FP64 plan per grid
    orc_idx = [i for i in sorted(sampled) if reqs[i][0] <= 512][:args.serve_oracle]
    cores = cpu_cores()
    ctx = mp.get_context("spawn")
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    pool = ctx.Pool(processes=max(1, min(cores, len(orc_idx)))) if orc_idx else None
    pending = pool.map_async(_oracle_serving, [(reqs[i][0], L, reqs[i][2], reqs[i][1]) for i in orc_idx]) \
        if pool else None
    plans64, err64 = {}, []
    for i in sorted(sampled):
        N, k, _ = reqs[i]
        if N not in plans64:
            plans64[N] = dbar.Plan(N, L, prec="fp64", restart=args.restart, tol=1e-13, max_batch=1)
        ref = plans64[N].solve(kept_Q[i], [k], want_m=False)["S"][0]
        err64.append(float(np.max(np.abs(kept_S[i] - ref)) / np.max(np.abs(ref))))
    for p in plans64.values():
        p.close()
    err_orc = []
    if pool:
        for i, So in zip(orc_idx, pending.get()):
            err_orc.append(float(np.max(np.abs(kept_S[i] - So)) / np.max(np.abs(So))))
        pool.close()
        pool.join()
    lat = np.array(lat)
    nmix = {str(N): int(sum(1 for r in reqs if r[0] == N)) for N in wl.SERVING_SIZES}
    lat_by_n, q_by_n, cyc_by_n = {}, {}, {}
    for i, t in enumerate(lat):  # latencies in submission order
        lat_by_n.setdefault(reqs[i][0], []).append(t)
        q_by_n.setdefault(reqs[i][0], []).append(queue[i])
        cyc_by_n.setdefault(reqs[i][0], []).append(cycles[i])
    return {"rate_req_s": args.rate, "duration_s": args.duration, "requests": len(reqs),
            "solves_per_s": round(len(lat) / wall, 2), "wall_s": round(wall, 2),
            "warmup_s": args.serve_warmup,
            "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "status_ok": int(sum(s_ == dbar.DBAR_OK for s_ in status)), "resid_max": float(max(resid)),
            "err_vs_fp64_gpu_max": float(max(err64)), "err_vs_fp64_gpu_sample": len(err64),
            "err_vs_oracle_max": float(max(err_orc)) if err_orc else None,
            "err_vs_oracle_sample": f"{len(err_orc)} requests with N <= 512 of the 2% sample "
                                    f"(N of the sample: {sorted(set(reqs[i][0] for i in orc_idx))})",
            "late_submits": late, "n_mix": nmix,
            "p50_p99_ms_by_N": {str(n): [round(float(np.percentile(lat_n, 50)), 2), round(float(np.percentile(lat_n, 99)), 2)]
                                for n, lat_n in sorted(lat_by_n.items())},
            "queue_p50_p99_ms_by_N": {str(n): [round(float(np.percentile(q, 50)), 2), round(float(np.percentile(q, 99)), 2)]
                                      for n, q in sorted(q_by_n.items())},
            "cycles_max_by_N": {str(n): int(max(c)) for n, c in sorted(cyc_by_n.items())},
            "config": {"L": L, "kmax": KMAX, "xi_q": XI_Q, "per_request_seed": f"{args.seed} + request index",
                       "terms": "1-6 per request", "restart": args.restart, "inner_tol": args.inner_tol,
                       "serve_batch": args.serve_batch, "budget_bytes": int(free * 0.7)},
            "clocks": clk.summary()}


def run_serving(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1508_02363_gb300 import dbar
    out = {"metric": "serving: CGO solves/sec and latency under Poisson arrivals", "workload": "serving"}
    out.update(serving_leg(args, dbar, torch, int(os.environ.get("LOCAL_RANK", "0"))))
    print(json.dumps(out))


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import workloads as wl
    w = wl.BY_NAME[args.workload]()
    cores = cpu_cores()
    nper = min(cores, args.cpu_sample)
    small = wl.plain_fp64()
    for _ in range(args.warmup):  # warm-up: start the pool and touch the code paths on a small case
        cpu_oracle_step(small, small.k[:1], 1)
    times, done = [], 0
    for s in range(args.steps):
        idx = (np.arange(nper) * max(1, w.k.size // nper) + s) % w.k.size
        dt, _ = cpu_oracle_step(w, w.k[idx], cores)
        times.append(dt)
        done += nper
    total = sum(times)
    value = done / total
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Gaussian-mixture potential and k list)",
           "config": {"workload": w.name, "N": w.N, "L": w.L, "nk": int(w.k.size), "M": w.M, "tol": w.tol,
                      "parallelism": "CPU processes"},
           "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "cores": min(cores, nper),
                            "kind": "oracle",
                            "sample": f"each step solves {nper} of the {w.k.size} k values with the FP64 CPU "
                                      f"oracle, one process per core"},
           "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed_1024")
    ap.add_argument("--restart", type=int, default=32)
    ap.add_argument("--ds2-prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ds2-tol", type=float, default=1e-13)
    ap.add_argument("--ds2-routes", action="store_true",
                    help="ds2: also q(., t) through the Sec. 4 route, difference to the iterated one")
    ap.add_argument("--iterated", action="store_true",
                    help="reflection workload: the iterated equation of Sec. 5 over the whole k-grid")
    ap.add_argument("--sstep", type=int, default=0,
                    help="Krylov vectors per basis sweep: 1, 2, 4, or 0 = the library's automatic choice")
    ap.add_argument("--inner-tol", dest="inner_tol", type=float, default=1e-6)
    ap.add_argument("--inner-m", dest="inner_m", type=int, default=0,
                    help="reflection / ds2 (M = 11, mixed): Taylor order of the FP32 inner operator (0: M)")
    ap.add_argument("--check-k", dest="check_k", type=int, default=4)
    ap.add_argument("--cpu-sample", dest="cpu_sample", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nk", type=int, default=0, help="solve only the first nk k values (profiling cases)")
    ap.add_argument("--max-outer", dest="max_outer", type=int, default=40)
    ap.add_argument("--rate", type=float, default=200.0, help="serving: requests per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--serve-batch", dest="serve_batch", type=int, default=128, help="serving: slots per lane")
    ap.add_argument("--serve-oracle", dest="serve_oracle", type=int, default=32,
                    help="serving: at most this many sampled requests (N <= 512) checked against the CPU oracle")
    ap.add_argument("--no-serving", action="store_true", help="default workload: skip the serving leg")
    ap.add_argument("--serve-warmup", dest="serve_warmup", type=float, default=3.0,
                    help="serving: seconds of uncounted traffic before the measured stream")
    ap.add_argument("--no-fp64-resid", dest="no_fp64_resid", action="store_true",
                    help="default workload: skip the leg with the refinement in native FP64")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--nreq", type=int, default=1000, help="uneven: number of solves")
    ap.add_argument("--autotune", type=int, default=1,
                    help="column-pass tiles: 1 timed at plan creation (default); 0, 2 or 3 pin variant 0, 1 or 2")
    ap.add_argument("--row-shape", dest="row_shape", type=int, default=0,
                    help="row-pass shape of the FP32 passes: 0 chosen by the autotuner; 1..5 pin one")
    ap.add_argument("--row-shape-plain", dest="row_shape_plain", type=int, default=0,
                    help="row-pass shape of the plain FP32 row passes A and C alone (1..5; 0: as --row-shape)")
    ap.add_argument("--quick", action="store_true",
                    help="time the solve only (no FP64 comparison, end-to-end leg or CPU baseline)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "reflection":
        run_reflection(args)
    elif args.workload == "ds2":
        run_ds2(args)
    elif args.workload == "conv":
        run_conv(args)
    elif args.workload == "uneven":
        run_uneven(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
