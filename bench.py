#!/usr/bin/env python
"""Benchmark: implicit grey M1 step throughput (cell-steps/s at 1e-8 relative
residual) on the 2D radiation-only beam in a lognormal opacity field,
1024 x 1024 cells, periodic in y / outflow in x, dt = 10 explicit CFL steps
(the configuration's smallest implicit step; at 50 dt_CFL the Newton iterates
leave the realizable set and do not converge, at 100 backtracking converges in
46 Newton steps).

One step = one backward-Euler M1 step from the same seeded initial state
(time-n face data, Newton with full steps tested on the FP64 residual, FP32
GMRES(30) with the multigrid preconditioner under FP64 refinement), inputs
resident in HBM. The plain FP64 path (point-block Jacobi GMRES(30), Armijo
backtracking) is measured beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0. Under torchrun (N > 1) every rank solves its
own replica of the workload (no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "implicit M1 cell-steps/s at 1e-8 rel. residual: mixed+learned vs plain FP64"
UNIT = "cell-steps/s"
L2_FLUSH_BYTES = 256 << 20
MG_CYCLE_DRAM_BYTES_1024 = 439.6e6


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--dt-factor", type=float, default=10.0)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--precond", default="mg", choices=["mg", "bj"],
                    help="preconditioner of the headline path (the plain FP64 path uses point-block Jacobi)")
    ap.add_argument("--newton", default="full", choices=["full", "backtrack"],
                    help="full Newton steps, or Armijo backtracking (halving theta up to 6 times)")
    ap.add_argument("--pc-rebuild", type=int, default=1,
                    help="rebuild the multigrid hierarchy on every k-th Newton step (1: every step)")
    ap.add_argument("--plain-steps", type=int, default=1, help="timed plain-FP64 steps beside the headline")
    ap.add_argument("--profile-steps", type=int, default=1,
                    help="steps run after the timed region with per-kernel-class event timers")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=48)
    return ap.parse_args()


def workload(n, dtf):
    import seeded_inputs as si
    return si.beam_lognormal_2d(n, dt_factor=dtf)


def workload_name(n, dtf):
    return (f"beam_lognormal_2d {n}x{n}: radiation-only grey M1, periodic y / outflow x, lognormal sigma "
            f"(ell=32 cells, sigma*dx in [1e-3,1e3], seed 2), beam |F|=0.99cE at x=0, dt={dtf:g} dt_CFL")


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(x: float) -> float:
    """Max of a per-rank float over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, steps: int, world: int, local_ms: float) -> float:
    """Whole-job cell-steps/s: every rank solves its own replica; the job time is
    the slowest rank's."""
    return world * cells_per_rank * steps / (max_over_ranks(local_ms) / 1e3)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


# ----------------------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(n, dtf, steps=1, line_search=False):
    """The oracle as it stands on a bounded sample: full implicit steps of the
    same recipe on an n x n grid (numpy, one host core for the stencil work)."""
    from oracle import Scheme, newton_solve
    p = workload(n, dtf)
    t0 = time.perf_counter()
    conv = True
    for _ in range(steps):
        r = newton_solve(Scheme(p), rtol=1e-8, line_search=line_search)
        conv = conv and r.converged
    dt = time.perf_counter() - t0
    return {"value": p.ncell * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} implicit step(s) of the same recipe at {n}x{n} (numpy FP64 oracle, "
                      f"block-Jacobi GMRES(30)+MGS, {'Armijo backtracking' if line_search else 'full Newton steps'}, "
                      f"1e-8), converged={conv}, {dt:.1f}s"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = a.cpu_sample_n
    ls = a.newton == "backtrack"
    for _ in range(a.warmup):
        cpu_oracle_sample(n, a.dt_factor, line_search=ls)
    t0 = time.perf_counter()
    res = cpu_oracle_sample(n, a.dt_factor, steps=a.steps, line_search=ls)
    el = time.perf_counter() - t0
    v = res["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(n, a.dt_factor), "sample_of": workload_name(a.n, a.dt_factor)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU path
def main():
    a = args_()
    if a.impl == "reference":
        return run_reference(a)
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2011_13926_gb300 import PREC_FP64, PREC_MIXED, context_from_problem, default_opts
    from paper_2011_13926_gb300.m1 import PRECOND_BJ, PRECOND_MG

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p = workload(a.n, a.dt_factor)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = context_from_problem(p, stream=stream, device=True)
    N = p.ncell
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    prec = PREC_MIXED if a.precision == "mixed" else PREC_FP64
    use_mg = a.precond == "mg" and prec == PREC_MIXED
    ls = int(a.newton == "backtrack")
    opts = default_opts(advance=0, precision=prec, precond=PRECOND_MG if use_mg else PRECOND_BJ, line_search=ls,
                        pc_rebuild=a.pc_rebuild)
    # the plain FP64 arm keeps the library defaults (point-block Jacobi, Armijo backtracking): with
    # full Newton steps its less exact point-block Jacobi solves do not converge in 30 Newton steps
    opts_plain = default_opts(advance=0, precision=PREC_FP64)

    def timed_steps(o, k, label):
        infos, ms = [], []
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st, info = ctx.implicit_step(p.dt, o, raise_on_fail=False)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        return ms, infos

    # warm-up (headline path)
    timed_steps(opts, a.warmup, "warmup")
    # timed region, headline path (no per-kernel timers inside it)
    s0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ms, infos = timed_steps(opts, a.steps, "timed")
    barrier()
    clk = clocks.stop()
    s1 = ctx.stats()
    value = job_throughput(N, a.steps, world, sum(ms))
    total_ms = max_over_ranks(sum(ms))
    converged = all(i.converged for i in infos)

    # the same step again with per-kernel-class CUDA-event timers, for the
    # breakdown and the roofline of the dominant class (not part of the headline)
    ctx.profile(True)
    p0 = ctx.stats()
    ms_prof, _ = timed_steps(opts, a.profile_steps, "profiled")
    p1 = ctx.stats()
    ctx.profile(False)
    # plain FP64 beside it (not part of the headline number)
    ms_plain, infos_plain = timed_steps(opts_plain, a.plain_steps, "plain")
    plain = {"value": N * len(ms_plain) / (sum(ms_plain) / 1e3) if ms_plain else None,
             "ms_per_step": statistics.mean(ms_plain) if ms_plain else None,
             "converged": all(i.converged for i in infos_plain),
             "newton_iters": [i.newton_iters for i in infos_plain],
             "gmres_iters": [i.gmres_iters for i in infos_plain],
             "config": "FP64 GMRES(30), point-block Jacobi, Armijo backtracking"}

    # roofline of the dominant kernel class over the profiled step(s)
    peak, peak_src = measured_peaks()
    kms = {k: p1["kernel_ms"][k] - p0["kernel_ms"][k] for k in p1["kernel_ms"]}
    kcount = {k: p1["kernel_count"][k] - p0["kernel_count"][k] for k in p1["kernel_count"]}
    dom = max(kms, key=kms.get)
    prof_ms = sum(ms_prof)
    roof = {"bound": "hbm", "kernel_class": dom, "share_of_step": kms[dom] / prof_ms if prof_ms else None,
            "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None,
            "peak_source": peak_src, "profiled_steps": a.profile_steps,
            "profiled_ms_per_step": prof_ms / max(1, a.profile_steps), "kernel_ms": kms, "kernel_count": kcount}
    bytes_map = {"jv32": p1["bytes_per_jv32"], "jv64": p1["bytes_per_jv"], "residual": p1["bytes_per_residual"],
                 "pc_apply": p1.get("bytes_per_mg_cycle", 0.0) if use_mg else 0.0}
    if dom == "ortho":
        ob = p1.get("ortho_bytes", 0.0) - p0.get("ortho_bytes", 0.0)
        if ob and kms[dom] > 0:
            roof["achieved"] = ob / (kms[dom] / 1e3) / 1e9
    elif bytes_map.get(dom) and kcount[dom] > 0:
        roof["achieved"] = bytes_map[dom] / (kms[dom] / kcount[dom] / 1e3) / 1e9
    if roof["achieved"] is not None:
        roof["frac"] = roof["achieved"] / peak
    # DRAM bytes (read + write) of one multigrid cycle on the 1024^2 beam, summed over its 13 launches
    # from one ncu capture (profiles/multigrid_beam_lognormal_1024_dt10.md); only for that workload
    if dom == "pc_apply" and use_mg and a.n == 1024 and a.dt_factor == 10.0:
        roof["traffic"] = MG_CYCLE_DRAM_BYTES_1024
        roof["traffic_unit"] = "bytes per cycle (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
        roof["algorithmic_bytes"] = bytes_map["pc_apply"]

    # end to end through the C ABI with host buffers (H2D inputs, D2H result)
    e2e = None
    if not a.no_e2e:
        E_h = torch.from_numpy(np.ascontiguousarray(p.E.ravel())).pin_memory()
        F_h = torch.from_numpy(np.ascontiguousarray(p.F.reshape(-1))).pin_memory()
        out_h = torch.empty(ctx.nu * N, dtype=torch.float64).pin_memory()
        ew = []
        for it in range(max(1, a.steps)):
            barrier()
            t0 = time.perf_counter()
            ctx.set_state(E_h, F_h)
            ctx.implicit_step(p.dt, opts, raise_on_fail=False)
            ctx.get_solution(out_h)
            torch.cuda.synchronize()
            ew.append(time.perf_counter() - t0)
        h2d = (E_h.numel() + F_h.numel()) * 8
        e2e = {"value": world * N * len(ew) / sum(ew), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": out_h.numel() * 8}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_oracle_sample(a.cpu_sample_n, a.dt_factor, line_search=a.newton == "backtrack")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == PREC_MIXED else "f64", "data": "synthetic",
                "config": {"workload": workload_name(a.n, a.dt_factor), "cells": N,
                           "path": "FP32 inner GMRES(30) + FP64 refinement" if prec == PREC_MIXED
                           else "FP64 GMRES(30)",
                           "preconditioner": ("aggregation multigrid V(1,1) (Galerkin, damped point-block Jacobi "
                                              "smoothing)" if use_mg else "point-block Jacobi"),
                           "newton_rtol": 1e-8, "newton": ("full steps" if a.newton == "full"
                                                            else "Armijo backtracking"),
                           "gmres_forcing": 1e-4, "wave_speeds": "frozen at time n",
                           "l2": "256 MiB buffer written between timed steps; basis traffic exceeds L2",
                           "parallelism": f"replicas x{world}"},
                "converged": converged,
                "newton_iters": [i.newton_iters for i in infos], "gmres_iters": [i.gmres_iters for i in infos],
                "plain_fp64": plain,
                "speedup_vs_plain_fp64": (value / world) / plain["value"] if plain["value"] else None,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": s1["kernel_launches"] - s0["kernel_launches"], "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
