#!/usr/bin/env python
"""Benchmark: implicit grey M1 step throughput (cell-steps/s at 1e-8 relative
residual) on the 2D radiation-only beam in a lognormal opacity field,
1024 x 1024 cells, periodic in y / outflow in x, dt = 50 explicit CFL steps
(the headline; 10 and 100 dt_CFL are timed beside it).

One step = one backward-Euler M1 step from the same seeded initial state
(time-n face data, Newton with full steps tested on the FP64 residual, FP32
GMRES(30) with the multigrid preconditioner under FP64 refinement, each linear
solve to 5e-3 relative, and the admissibility fallback that keeps every cell's
E > 0 and |F| <= cE), inputs resident in HBM. The plain FP64 path (point-block
Jacobi GMRES(30) to 1e-4, with full Newton steps and with Armijo backtracking,
the same fallback) is measured beside it.

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
PROFILES = os.path.join(ROOT, "profiles")


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="beam", choices=["beam", "learned", "gas3d", "batch"],
                    help="beam: the 1024^2 beam (headline); learned: the learned preconditioner on 512^2 "
                         "lognormal Gaussian-pulse systems at 50 dt_CFL (training, then held-out solves); "
                         "gas3d: the 256^3 gas-coupled point source (advection, implicit step, velocity sources); "
                         "batch: 256 independent 2D problems of 64^2-256^2 cells in one batched step")
    ap.add_argument("--train-rounds", type=int, default=8)
    ap.add_argument("--train-pairs", type=int, default=512, help="pairs per training round (learned workload)")
    ap.add_argument("--train-krylov-steps", type=int, default=0,
                    help="learned workload: random training directions are smooth fields (0) or the error they "
                         "leave after this many point-block Jacobi GMRES steps")
    ap.add_argument("--train-first-stage", type=int, default=0, choices=[0, 1],
                    help="learned workload: 1 turns each random training direction e into the error one "
                         "point-block Jacobi stage leaves of it (the input of the two-stage forms)")
    ap.add_argument("--learned-forms", default="0,1",
                    help="forms of the learned preconditioner timed (m1_set_learned_form: 0 additive, 1 two-stage "
                         "on odd Arnoldi steps, 2 two-stage on every step); the first is the line's value")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--dt-factor", type=float, default=50.0)
    ap.add_argument("--other-dts", default="10,100",
                    help="dt factors timed beside the headline on the same path (comma list, '' for none)")
    ap.add_argument("--other-steps", type=int, default=2, help="timed steps per other dt")
    ap.add_argument("--forcing", default="fixed", choices=["fixed", "ew"],
                    help="linear-solve tolerance: fixed (--gmres-rtol), or Eisenstat-Walker (m1_solver_opts.forcing)")
    ap.add_argument("--gmres-rtol", type=float, default=None,
                    help="fixed relative tolerance of every linear solve of the mixed path "
                         "(m1_solver_opts.gmres_rtol; default 5e-3 for the beam and the batch, 1e-4 otherwise); the Newton "
                         "test stays ||R|| <= 1e-8 ||R(U^n)|| in FP64")
    ap.add_argument("--plain-gmres-rtol", type=float, default=1e-4,
                    help="the same for the plain FP64 arm (1e-4: its fastest measured forcing; at 1e-3 its full "
                         "steps take longer and its backtracking does not converge within 80 Newton steps)")
    ap.add_argument("--realizability", type=int, default=1, choices=[0, 1],
                    help="1: the admissibility fallback of the implicit step (m1_solver_opts.realizability)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--precond", default="mg", choices=["mg", "bj"],
                    help="preconditioner of the headline path (the plain FP64 path uses point-block Jacobi)")
    ap.add_argument("--newton", default="full", choices=["full", "backtrack"],
                    help="full Newton steps, or Armijo backtracking (halving theta up to 6 times)")
    ap.add_argument("--pc-rebuild", type=int, default=1,
                    help="rebuild the multigrid hierarchy on every k-th Newton step (1: every step)")
    ap.add_argument("--plain-steps", type=int, default=1, help="timed plain-FP64 steps per globalisation")
    ap.add_argument("--profile-steps", type=int, default=1,
                    help="steps run after the timed region with per-kernel-class event timers")
    ap.add_argument("--fp64-arith", default="auto", choices=["auto", "native", "double_word"],
                    help="FP64 arithmetic of the headline path's residual and J v (m1_set_fp64_arithmetic); "
                         "the plain FP64 arm always uses FP64 operations")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket each timed headline step by cudaProfilerStart/Stop, for an ncu capture of the "
                         "whole step as one range (--replay-mode app-range)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=80,
                    help="grid side of the oracle's one-step sample in the line's cpu_baseline (about 10 s)")
    ap.add_argument("--ref-sample-n", type=int, default=48,
                    help="grid side of each oracle step of --impl reference (about 2 s per step)")
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


# ----------------------------------------------------------------------------- algorithmic bytes
# Minimum DRAM traffic per launch in the per-cell units of the scope table (2D,
# radiation only: n_u = 3 unknowns, d = 2 faces of alpha per cell, one opacity,
# FP32 words on the inner path): what a kernel must read and write at least.
# Stored extras (time-n wave speeds, the pressure Jacobian dP/dU) are not
# counted, so a kernel that reads them shows DRAM traffic above these figures.
NU, DIM, W32, W64 = 3, 2, 4, 8


def bytes_jv32(N):
    """J v, FP32: read v, U, sigma, alpha (d faces); write J v."""
    return N * W32 * (NU + NU + 1 + DIM + NU)


def bytes_residual64(N):
    """R(U), FP64: read U, U^n, sigma, alpha, B; write R."""
    return N * W64 * (NU + NU + 1 + DIM + 1 + NU)


def bytes_jv64(N):
    return N * W64 * (NU + NU + 1 + DIM + NU)


def mg_level_sizes(nx, ny, nlev):
    out = [(nx, ny)]
    for _ in range(1, nlev):
        nx, ny = (nx + 1) // 2, (ny + 1) // 2
        out.append((nx, ny))
    return out


def bytes_mg_cycle(nx, ny, nlev):
    """One V(1,1) cycle (FP32). Level 0, down pass: the point-block Jacobi apply
    (read r, M^-1; write z), J z (read U, sigma, alpha; z comes from shared
    memory), restriction (write n_u words per coarse cell); up pass: read r, z,
    the coarse correction, U, sigma, alpha, M^-1; write the smoothed z.
    Assembled levels: each pass reads the 5-point block stencil A (5 n_u^2
    words), M^-1 (n_u^2) and r, writes z (down: plus the restricted residual;
    up: reads z and the coarse correction). The coarsest level reads A, M^-1,
    r and writes z once (its sweeps stay on chip)."""
    lv = mg_level_sizes(nx, ny, nlev)
    cells = [a * b for a, b in lv]
    jv_in = NU + 1 + DIM
    w = 0.0
    if nlev == 1:
        return W32 * cells[0] * (5 * NU * NU + NU * NU + 2 * NU)
    w += cells[0] * ((NU + NU * NU + NU + jv_in) + (NU + NU + jv_in + NU * NU + NU)) + 2 * NU * cells[1]
    for l in range(1, nlev - 1):
        w += cells[l] * ((5 * NU * NU + NU * NU + NU + NU) + (5 * NU * NU + NU * NU + NU + NU + NU)) \
            + 2 * NU * cells[l + 1]
    w += cells[nlev - 1] * (5 * NU * NU + NU * NU + 2 * NU)
    return W32 * w


def profile_traffic(name):
    """(bytes per launch, record) from a committed ncu summary under profiles/: its
    'traffic_bytes_per_launch:' and 'sources:' / 'source_sha:' lines. None when the
    file is missing or the kernel sources changed since the capture."""
    path = os.path.join(PROFILES, name)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None, {"file": f"profiles/{name}", "status": "missing"}
    kv = {}
    for ln in lines:
        ln = ln.strip().lstrip("-* ")
        for key in ("traffic_bytes_per_launch:", "sources:", "source_sha:"):
            if ln.startswith(key):
                kv[key[:-1]] = ln[len(key):].strip().strip("`")
    if not all(k in kv for k in ("traffic_bytes_per_launch", "sources", "source_sha")):
        return None, {"file": f"profiles/{name}", "status": "no traffic record"}
    from paper_2011_13926_gb300.ncu_summary import source_hash
    files = [f.strip() for f in kv["sources"].split(",") if f.strip()]
    now = source_hash(files)
    rec = {"file": f"profiles/{name}", "source_sha_at_capture": kv["source_sha"], "source_sha_now": now,
           "bytes_per_launch_at_capture": float(kv["traffic_bytes_per_launch"])}
    if now != kv["source_sha"]:
        rec["status"] = "stale: the kernel sources changed since the capture"
        return None, rec
    rec["status"] = "current"
    return float(kv["traffic_bytes_per_launch"]), rec


# ----------------------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(n, dtf, steps=1, line_search=False, realizability=True, gmres_rtol=1e-3):
    """The oracle as it stands on a bounded sample: full implicit steps of the
    same recipe on an n x n grid (numpy, one host core for the stencil work)."""
    from oracle import Scheme, newton_solve
    p = workload(n, dtf)
    t0 = time.perf_counter()
    conv = True
    for _ in range(steps):
        r = newton_solve(Scheme(p), rtol=1e-8, line_search=line_search, realizability=realizability,
                         newton_max=60, gmres_rtol=gmres_rtol)
        conv = conv and r.converged
    dt = time.perf_counter() - t0
    return {"value": p.ncell * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} implicit step(s) of the same recipe at {n}x{n} (numpy FP64 oracle, "
                      f"block-Jacobi GMRES(30)+MGS to {gmres_rtol:g}, "
                      f"{'Armijo backtracking' if line_search else 'full Newton steps'}, "
                      f"{'admissibility fallback, ' if realizability else ''}1e-8), converged={conv}, {dt:.1f}s"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = a.ref_sample_n
    ls = a.newton == "backtrack"
    for _ in range(a.warmup):
        cpu_oracle_sample(n, a.dt_factor, line_search=ls, realizability=bool(a.realizability),
                          gmres_rtol=a.gmres_rtol)
    t0 = time.perf_counter()
    res = cpu_oracle_sample(n, a.dt_factor, steps=a.steps, line_search=ls, realizability=bool(a.realizability),
                            gmres_rtol=a.gmres_rtol)
    el = time.perf_counter() - t0
    v = res["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(n, a.dt_factor), "sample_of": workload_name(a.n, a.dt_factor)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- learned workload
def run_learned(a):
    """Train the network on 512^2 problems (seeds 1000+), then time one implicit step of
    held-out problems (seeds 1100, 1101) with mixed precision + the learned preconditioner
    (FGMRES(30)) beside mixed point-block Jacobi, mixed multigrid and plain FP64
    point-block Jacobi; errors are the oracle's residual of each GPU state."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    import seeded_inputs as si
    from oracle import Scheme, unet
    from paper_2011_13926_gb300 import learned, m1
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream().cuda_stream
    n = 512

    def prob(seed):
        return si.gaussian_lognormal_2d(n, seed, dt_factor=a.dt_factor if a.dt_factor else 50.0)

    res = learned.train(prob, range(1000, 1100), n=n, rounds=a.train_rounds, pairs_per_round=a.train_pairs,
                        epochs=4, lr=1e-3, lr_final=1e-4, krylov_steps=a.train_krylov_steps,
                        init=unet.init_params(0), first_stage=bool(a.train_first_stage))
    form_names = {0: "additive", 1: "two_stage", 2: "two_stage_all"}
    forms = [int(f) for f in a.learned_forms.split(",") if f.strip()]
    paths = {"mixed_learned": dict(precision=m1.PREC_MIXED, precond=learned.PRECOND_LEARNED, form=forms[0])}
    for f in forms[1:]:
        paths[f"mixed_learned_{form_names[f]}"] = dict(precision=m1.PREC_MIXED, precond=learned.PRECOND_LEARNED,
                                                       form=f)
    paths.update({
             "mixed_bj": dict(precision=m1.PREC_MIXED, precond=m1.PRECOND_BJ),
             "mixed_mg": dict(precision=m1.PREC_MIXED, precond=3),
             "plain_fp64_bj": dict(precision=m1.PREC_FP64, precond=m1.PRECOND_BJ)})
    out = {k: {"ms": [], "newton_iters": [], "gmres_iters": [], "converged": [], "oracle_residual_ratio": []}
           for k in paths}
    infer = m1.Net(n, n, 1, s)
    infer.set_params(res["params"])
    launches0 = 0
    for seed in (1100, 1101):
        p = prob(seed)
        sch = Scheme(p)
        r0 = np.linalg.norm(sch.residual(p.state_vector()))
        for name, kw in paths.items():
            ctx = m1.context_from_problem(p, stream=s, device=True)
            kw = dict(kw)
            form = kw.pop("form", None)
            if form is not None:
                ctx.set_preconditioner(infer)
                ctx.set_learned_form(form)
            opts = m1.default_opts(advance=0, **kw)
            for _ in range(max(1, a.warmup)):
                ctx.implicit_step(p.dt, opts, raise_on_fail=False)
            st0 = ctx.stats()
            for _ in range(a.steps):
                st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
                out[name]["ms"].append(info.time_ms)
                out[name]["newton_iters"].append(info.newton_iters)
                out[name]["gmres_iters"].append(info.gmres_iters)
                out[name]["converged"].append(bool(info.converged))
            if name == "mixed_learned":
                launches0 += ctx.stats()["kernel_launches"] - st0["kernel_launches"]
            u = ctx.get_solution()
            out[name]["oracle_residual_ratio"].append(float(np.linalg.norm(sch.residual(u)) / r0))
            ctx.close()
    for v in out.values():
        v["value"] = n * n * len(v["ms"]) / (sum(v["ms"]) / 1e3) if v["ms"] else None
    # the network on the tensor cores: one forward pass at 512^2 (BF16), CUDA events
    x = torch.randn(n * n * 7, device="cuda", dtype=torch.float32)
    for _ in range(3):
        infer.forward(x, bf16=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    reps = 20
    for _ in range(reps):
        infer.forward(x, bf16=True)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    flops = learned.forward_flops(n, n)
    peak = None
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        peak = 1900.0
    v = out["mixed_learned"]["value"]
    plain = out["plain_fp64_bj"]["value"]
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": statistics.mean(out["mixed_learned"]["ms"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32+f64", "data": "synthetic",
            "config": {"workload": f"gaussian_lognormal_2d {n}x{n}: radiation-only grey M1, periodic, lognormal "
                                   f"sigma (ell=n/32, sigma*dx in [1e-2,1e3]), Gaussian pulse, dt=50 dt_CFL; "
                                   f"held-out seeds 1100-1101, training seeds 1000+",
                       "path": "FP32 inner FGMRES(30) + FP64 refinement, learned correction in the "
                               f"{form_names[forms[0]]} form (m1_set_learned_form {forms[0]})"},
            "training": {"pairs": res["pairs"], "seconds": res["seconds"], "first_loss": res["first_loss"],
                         "final_loss": res["final_loss"], "rounds": a.train_rounds,
                         "directions": ("smooth random fields" if a.train_krylov_steps == 0 else
                                        f"errors left by {a.train_krylov_steps} point-block Jacobi GMRES steps")
                                       + (", then the error one point-block Jacobi stage leaves"
                                          if a.train_first_stage else "")},
            "paths": out, "speedup_vs_plain_fp64": v / plain if v and plain else None,
            "roofline": {"bound": "tensor", "kernel_class": "network forward (tensor-core convolutions)",
                         "achieved": flops / (fwd_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (fwd_ms / 1e3) / 1e12 / peak, "traffic": None,
                         "flops_per_forward": flops, "forward_ms": fwd_ms,
                         "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops)"},
            "gpu_launches": launches0}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- 3D gas workload
def bytes_jv32_3d_gas(N):
    """J v, FP32, 3D with gas (n_u = 5): read v, U, sigma, alpha (3 faces); write J v (76 B per cell)."""
    return N * W32 * (5 + 5 + 1 + 3 + 5)


def run_gas3d(a):
    """One step of the 256^3 gas workload from the same seeded state per step: the
    explicit advection of the gas energy, the implicit M1 step (mixed precision,
    point-block Jacobi GMRES(30)) and the explicit velocity-dependent sources."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    import seeded_inputs as si
    from paper_2011_13926_gb300 import m1
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream().cuda_stream
    n = a.n if a.n != 1024 else 256
    dtf = a.dt_factor
    p = si.gas_point_source_3d(n, dt_factor=dtf)
    ctx = m1.context_from_problem(p, stream=s, device=True)
    arith = {"auto": m1.FP64_AUTO, "native": m1.FP64_NATIVE, "double_word": m1.FP64_DOUBLE_WORD}
    ctx.set_fp64_arithmetic(arith[a.fp64_arith])
    fp64_in_use = "double_word" if ctx.fp64_arithmetic()[0] == m1.FP64_DOUBLE_WORD else "native"
    ux, uy, uz = si.divergence_free_velocity_3d(n, 7)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()  # noqa: E731
    ctx.set_velocity(dev(ux), dev(uy), dev(uz))
    E0, F0, T0, rc = dev(p.E), dev(p.F), dev(p.T), dev(p.rho_cv)
    N = p.ncell
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(opts):
        ctx.set_state(E0, F0, T0, rc)
        ctx.advect(p.dt)
        st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
        ctx.velocity_sources(p.dt)
        return info

    def timed(opts, k, profile_range=False):
        ms, infos = [], []
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if profile_range:  # the step alone between cudaProfilerStart and cudaProfilerStop
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
            e0.record()
            info = step(opts)
            e1.record()
            torch.cuda.synchronize()
            if profile_range:
                torch.cuda.profiler.stop()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        return ms, infos

    rtol = 1e-4 if a.gmres_rtol is None else a.gmres_rtol
    opts = m1.default_opts(precision=m1.PREC_MIXED, gmres_max=3000, gmres_rtol=rtol)
    timed(opts, a.warmup)
    s0 = ctx.stats()
    clocks = ClockSampler(0)
    clocks.start()
    ms, infos = timed(opts, a.steps, profile_range=a.profile_range)
    clk = clocks.stop()
    s1 = ctx.stats()
    ctx.profile(True)
    p0 = ctx.stats()
    msp, _ = timed(opts, 1)
    p1 = ctx.stats()
    ctx.profile(False)
    ctx.set_fp64_arithmetic(m1.FP64_NATIVE)  # the plain arm: FP64 operations
    mplain, iplain = timed(m1.default_opts(precision=m1.PREC_FP64, gmres_max=3000, gmres_rtol=a.plain_gmres_rtol),
                           a.plain_steps)
    peak, peak_src = measured_peaks()
    kms = {k: p1["kernel_ms"][k] - p0["kernel_ms"][k] for k in p1["kernel_ms"]}
    kcount = {k: p1["kernel_count"][k] - p0["kernel_count"][k] for k in p1["kernel_count"]}
    dom = max(kms, key=kms.get)
    roof = {"bound": "hbm", "kernel_class": dom, "share_of_step": kms[dom] / sum(msp), "achieved": None,
            "peak": peak, "unit": "GB/s", "frac": None, "traffic": None, "peak_source": peak_src,
            "kernel_ms": kms, "kernel_count": kcount}
    if dom == "ortho":
        ob = p1.get("ortho_bytes", 0.0) - p0.get("ortho_bytes", 0.0)
        roof["achieved"] = ob / (kms[dom] / 1e3) / 1e9
    elif dom == "jv32" and kcount[dom]:
        roof["achieved"] = bytes_jv32_3d_gas(N) / (kms[dom] / kcount[dom] / 1e3) / 1e9
        roof["algorithmic_bytes"] = bytes_jv32_3d_gas(N)
    if roof["achieved"]:
        roof["frac"] = roof["achieved"] / peak
    # whole-step bytes per cell-update from the committed range capture of this workload's step
    bps, rec = profile_traffic(f"step_traffic_gas_point_source_{n}.md")
    roof["step_dram_bytes_per_cell_update"] = bps / N if bps else None
    roof["step_traffic_record"] = rec
    cpu = None
    if not a.no_cpu_baseline:
        from oracle import Scheme, newton_solve
        q = si.gas_point_source_3d(24, dt_factor=dtf)
        t0 = time.perf_counter()
        r = newton_solve(Scheme(q), rtol=1e-8)
        el = time.perf_counter() - t0
        cpu = {"value": q.ncell / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"1 implicit step at 24^3 (numpy FP64 oracle, block-Jacobi GMRES(30)+MGS, Armijo "
                         f"backtracking, 1e-8), converged={r.converged}, {el:.1f}s"}
    line = {"metric": METRIC, "value": N * len(ms) / (sum(ms) / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"gas_point_source_3d {n}^3: grey M1 + gas energy, lognormal density "
                                   f"(ell=16), sigma = kappa rho (kappa dx = 1), point source, outflow, dt={dtf:g} "
                                   f"dt_CFL, divergence-free flow (max |u| = 1e-3 c); advection + implicit step + "
                                   f"velocity sources", "cells": N,
                       "path": "FP32 inner GMRES(30) + FP64 refinement, point-block Jacobi, Armijo backtracking",
                       "fp64_arithmetic": ("double-word (FP32 pairs) residual and J v, FP64 arrays"
                                           if fp64_in_use == "double_word" else "FP64 operations"),
                       "l2": "256 MiB buffer written between timed steps; the state alone is 670 MB"},
            "converged": all(i.converged for i in infos), "newton_iters": [i.newton_iters for i in infos],
            "gmres_iters": [i.gmres_iters for i in infos],
            "realizability_violations": [i.realizability_violations for i in infos],
            "plain_fp64": {"ms_per_step": statistics.mean(mplain) if mplain else None,
                           "value": N * len(mplain) / (sum(mplain) / 1e3) if mplain else None,
                           "converged": all(i.converged for i in iplain),
                           "newton_iters": [i.newton_iters for i in iplain],
                           "gmres_iters": [i.gmres_iters for i in iplain]},
            "roofline": roof, "cpu_baseline": cpu,
            "gpu_launches": s1["kernel_launches"] - s0["kernel_launches"], "clocks": clk}
    if line["plain_fp64"]["value"]:
        line["speedup_vs_plain_fp64"] = line["value"] / line["plain_fp64"]["value"]
    print(json.dumps(line), flush=True)
    ctx.close()


# ----------------------------------------------------------------------------- batched workload
def run_batch(a):
    """One batched implicit step of 256 independent problems (sizes uniform from 64^2,
    96^2, 128^2, 192^2, 256^2, own opacity and pulse, dt log-uniform in [10, 100]
    dt_CFL): persistent CTA-per-problem classes from one CUDA graph, large classes
    through single-grid contexts beside it, the split chosen by m1_batch_tune during
    the warm-up. Plain FP64 point-block Jacobi solves of every problem, one after
    another, are timed beside it."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    import seeded_inputs as si
    from oracle import Scheme
    from paper_2011_13926_gb300 import m1
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream().cuda_stream
    probs = si.batch_problems(256)
    cells = sum(p.ncell for p in probs)
    dts = [p.dt for p in probs]
    B = m1.Batch(probs, s)
    opts = m1.default_opts(gmres_rtol=1e-4 if a.gmres_rtol is None else a.gmres_rtol)
    chosen = B.tune(dts, opts)
    for _ in range(max(1, a.warmup - 1)):
        B.implicit_step(dts, opts)
    clocks = ClockSampler(0)
    clocks.start()
    ms, infos = [], []
    for _ in range(a.steps):
        info, t = B.implicit_step(dts, opts)
        ms.append(t)
        infos.append(info)
    clk = clocks.stop()
    last = infos[-1]
    # parity sample: the first problem of every size class, oracle residual of the GPU state
    sample, seen = {}, set()
    for k, p in enumerate(probs):
        if p.n[0] in seen:
            continue
        seen.add(p.n[0])
        sch = Scheme(p)
        r0 = np.linalg.norm(sch.residual(p.state_vector()))
        sample[f"{p.n[0]}^2 (problem {k})"] = float(np.linalg.norm(sch.residual(B.get_solution(k))) / r0)
    B.close()
    # plain FP64, problem by problem through single-grid contexts
    plain_ms, plain_conv = 0.0, True
    po = m1.default_opts(advance=0, precision=m1.PREC_FP64, gmres_rtol=a.plain_gmres_rtol)
    for p in probs:
        ctx = m1.context_from_problem(p, stream=s, device=True)
        st, inf = ctx.implicit_step(p.dt, po, raise_on_fail=False)
        plain_ms += inf.time_ms
        plain_conv = plain_conv and bool(inf.converged)
        ctx.close()
    cpu = None
    if not a.no_cpu_baseline:
        from oracle import newton_solve
        q = si.gaussian_lognormal_2d(64, 5000, dt_factor=30.0)
        t0 = time.perf_counter()
        r = newton_solve(Scheme(q), rtol=1e-8)
        el = time.perf_counter() - t0
        cpu = {"value": q.ncell / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"1 implicit step of one 64^2 problem of the batch recipe (numpy FP64 oracle, block-Jacobi "
                         f"GMRES(30)+MGS, 1e-8), converged={r.converged}, {el:.1f}s"}
    sizes = sorted({p.n[0] for p in probs})
    line = {"metric": METRIC, "value": cells * len(ms) / (sum(ms) / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "256 independent gaussian_lognormal_2d problems (seeds 5000+k), sizes uniform "
                                   "from 64^2, 96^2, 128^2, 192^2, 256^2, dt log-uniform in [10, 100] dt_CFL",
                       "cells": cells, "problems": len(probs),
                       "path": "persistent CTA-per-problem classes (one CUDA graph) + single-grid contexts for the "
                               "classes m1_batch_tune sends there; FP32 inner GMRES(30) + FP64 refinement, "
                               "point-block Jacobi",
                       "gmres_forcing": opts.gmres_rtol},
            "per_class": {f"{n}^2": {"problems": sum(1 for p in probs if p.n[0] == n),
                                     "path": ("single-grid" if int(chosen[i]) == 0
                                              else f"persistent, {int(chosen[i])} threads"),
                                     "newton_iters_mean": float(np.mean([last[k]["newton_iters"] for k, p in
                                                                         enumerate(probs) if p.n[0] == n])),
                                     "gmres_iters_mean": float(np.mean([last[k]["gmres_iters"] for k, p in
                                                                        enumerate(probs) if p.n[0] == n]))}
                          for i, n in enumerate(sizes)},
            "converged": all(i["converged"] == 1 for i in last),
            "oracle_residual_ratio_sample": sample,
            "plain_fp64": {"ms": plain_ms, "value": cells / (plain_ms / 1e3), "converged": plain_conv,
                           "config": "FP64 GMRES(30), point-block Jacobi, Armijo backtracking, one problem after "
                                     "another"},
            "speedup_vs_plain_fp64": (cells * len(ms) / (sum(ms) / 1e3)) / (cells / (plain_ms / 1e3)),
            "roofline": None, "roofline_note": "one persistent launch per size class runs whole solves; no "
                                               "single kernel class dominates",
            "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU path
def main():
    a = args_()
    if a.gmres_rtol is None and a.workload in ("beam", "batch"):
        a.gmres_rtol = 5e-3
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "learned":
        return run_learned(a)
    if a.workload == "gas3d":
        return run_gas3d(a)
    if a.workload == "batch":
        return run_batch(a)
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
    from paper_2011_13926_gb300 import m1 as m1mod
    arith = {"auto": m1mod.FP64_AUTO, "native": m1mod.FP64_NATIVE, "double_word": m1mod.FP64_DOUBLE_WORD}
    ctx.set_fp64_arithmetic(arith[a.fp64_arith])
    fp64_in_use = "double_word" if ctx.fp64_arithmetic()[0] == m1mod.FP64_DOUBLE_WORD else "native"
    N = p.ncell
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    prec = PREC_MIXED if a.precision == "mixed" else PREC_FP64
    use_mg = a.precond == "mg" and prec == PREC_MIXED
    ls = int(a.newton == "backtrack")
    rz = a.realizability
    opts = default_opts(advance=0, precision=prec, precond=PRECOND_MG if use_mg else PRECOND_BJ, line_search=ls,
                        pc_rebuild=a.pc_rebuild, realizability=rz, newton_max=60, gmres_rtol=a.gmres_rtol,
                        forcing=1 if a.forcing == "ew" else 0)
    dt_cfl = p.dt / a.dt_factor

    def timed_steps(o, k, dt=None, profile_range=False):
        infos, ms = [], []
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if profile_range:  # the step alone between cudaProfilerStart and cudaProfilerStop
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
            e0.record()
            st, info = ctx.implicit_step(p.dt if dt is None else dt, o, raise_on_fail=False)
            e1.record()
            torch.cuda.synchronize()
            if profile_range:
                torch.cuda.profiler.stop()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        return ms, infos

    def step_record(ms, infos):
        return {"ms_per_step": statistics.mean(ms) if ms else None,
                "value": N * len(ms) / (sum(ms) / 1e3) if ms else None,
                "converged": all(i.converged for i in infos),
                "newton_iters": [i.newton_iters for i in infos], "gmres_iters": [i.gmres_iters for i in infos],
                "realizability_violations": [i.realizability_violations for i in infos],
                "fallback_cells": [i.fallback_cells for i in infos]}

    # warm-up (headline path)
    timed_steps(opts, a.warmup)
    # timed region, headline path (no per-kernel timers inside it)
    s0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ms, infos = timed_steps(opts, a.steps, profile_range=a.profile_range)
    barrier()
    clk = clocks.stop()
    s1 = ctx.stats()
    value = job_throughput(N, a.steps, world, sum(ms))
    total_ms = max_over_ranks(sum(ms))
    converged = all(i.converged for i in infos)

    # the same path at the other step sizes of the workload (not part of the headline number)
    per_dt = {f"{a.dt_factor:g}": step_record(ms, infos)}
    for f in [float(x) for x in a.other_dts.split(",") if x.strip()]:
        timed_steps(opts, 1, f * dt_cfl)
        m2, i2 = timed_steps(opts, a.other_steps, f * dt_cfl)
        per_dt[f"{f:g}"] = step_record(m2, i2)

    # the same step again with per-kernel-class CUDA-event timers, for the
    # breakdown and the roofline of the dominant class (not part of the headline)
    ctx.profile(True)
    p0 = ctx.stats()
    ms_prof, infos_prof = timed_steps(opts, a.profile_steps)
    p1 = ctx.stats()
    ctx.profile(False)
    # plain FP64 beside it (not part of the headline number): point-block Jacobi GMRES(30), the same
    # admissibility fallback, with full Newton steps and with Armijo backtracking
    plain = {}
    ctx.set_fp64_arithmetic(m1mod.FP64_NATIVE)
    for name, lsv in (("full_steps", 0), ("backtracking", 1)):
        o = default_opts(advance=0, precision=PREC_FP64, precond=PRECOND_BJ, line_search=lsv, realizability=rz,
                         newton_max=80, gmres_rtol=a.plain_gmres_rtol)
        m3, i3 = timed_steps(o, a.plain_steps)
        rec = step_record(m3, i3)
        rec["config"] = (f"FP64 GMRES(30) to {a.plain_gmres_rtol:g}, point-block Jacobi, FP64 operations, "
                         + ("full Newton steps" if lsv == 0 else "Armijo backtracking"))
        plain[name] = rec
    best_plain = max((r for r in plain.values() if r["converged"] and r["value"]), key=lambda r: r["value"],
                     default=None)

    # roofline of the dominant kernel class over the profiled step(s): algorithmic bytes per launch
    # (the scope table's per-cell units, computed here from the grid and the level sizes) over the
    # class's mean event-timed launch; traffic from the committed ncu summary of that launch
    peak, peak_src = measured_peaks()
    kms = {k: p1["kernel_ms"][k] - p0["kernel_ms"][k] for k in p1["kernel_ms"]}
    kcount = {k: p1["kernel_count"][k] - p0["kernel_count"][k] for k in p1["kernel_count"]}
    dom = max(kms, key=kms.get)
    prof_ms = sum(ms_prof)
    roof = {"bound": "hbm", "kernel_class": dom, "share_of_step": kms[dom] / prof_ms if prof_ms else None,
            "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None,
            "peak_source": peak_src, "profiled_steps": a.profile_steps,
            "profiled_ms_per_step": prof_ms / max(1, a.profile_steps), "kernel_ms": kms, "kernel_count": kcount}
    nlev = ctx.mg_levels() if use_mg else 0
    alg, launch_name, prof_file = None, None, None
    if dom == "pc_apply" and use_mg:
        alg = bytes_mg_cycle(p.n[0], p.n[1], nlev)
        launch_name = f"one multigrid V(1,1) cycle ({2 * nlev - 1} launches, {nlev} levels)"
        prof_file = f"multigrid_cycle_beam_lognormal_{a.n}_dt{a.dt_factor:g}.md"
    elif dom == "jv32":
        alg = bytes_jv32(N)
        launch_name = "FP32 J v"
    elif dom == "jv64":
        alg = bytes_jv64(N)
        launch_name = "FP64 J v"
    elif dom == "residual":
        alg = bytes_residual64(N)
        launch_name = "FP64 residual"
    if dom == "ortho":
        ob = p1.get("ortho_bytes", 0.0) - p0.get("ortho_bytes", 0.0)
        if ob and kms[dom] > 0:
            roof["achieved"] = ob / (kms[dom] / 1e3) / 1e9
            roof["algorithmic_bytes_note"] = "Gram-Schmidt: (j+2) words read per element for the dots, (j+3) " \
                                             "for the update, j the Arnoldi step (FP32 basis)"
    elif alg and kcount[dom] > 0:
        roof["achieved"] = alg / (kms[dom] / kcount[dom] / 1e3) / 1e9
        roof["algorithmic_bytes"] = alg
        roof["launch"] = launch_name
    if roof["achieved"] is not None:
        roof["frac"] = roof["achieved"] / peak
    if prof_file:
        tr, rec = profile_traffic(prof_file)
        roof["traffic"] = tr
        roof["traffic_record"] = rec
    # whole-step bytes per cell-update from the committed launch list of the headline step
    bpc, rec = profile_traffic(f"step_traffic_beam_lognormal_{a.n}_dt{a.dt_factor:g}.md")
    roof["step_dram_bytes_per_cell_update"] = bpc / N if bpc else None
    roof["step_traffic_record"] = rec

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
        cpu = cpu_oracle_sample(a.cpu_sample_n, a.dt_factor, line_search=a.newton == "backtrack",
                                realizability=bool(rz), gmres_rtol=a.gmres_rtol)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == PREC_MIXED else "f64", "data": "synthetic",
                "config": {"workload": workload_name(a.n, a.dt_factor), "cells": N,
                           "path": "FP32 inner GMRES(30) + FP64 refinement" if prec == PREC_MIXED
                           else "FP64 GMRES(30)",
                           "fp64_arithmetic": ("double-word (FP32 pairs) residual and J v, FP64 arrays"
                                               if fp64_in_use == "double_word" else "FP64 operations"),
                           "preconditioner": ("aggregation multigrid V(1,1) (Galerkin, damped point-block Jacobi "
                                              "smoothing)" if use_mg else "point-block Jacobi"),
                           "newton_rtol": 1e-8, "newton": ("full steps" if a.newton == "full"
                                                            else "Armijo backtracking"),
                           "admissibility": ("a posteriori fallback: centred source, alpha = 1, speeds +-c in "
                                             "flagged cells" if rz else "none (violations counted)"),
                           "gmres_forcing": ("Eisenstat-Walker" if a.forcing == "ew" else a.gmres_rtol),
                           "learned_arm": ("bench.py --workload learned: the learned preconditioner on 512^2 "
                                           "systems, where it does not beat point-block Jacobi; this line's "
                                           "preconditioner is the multigrid cycle"),
                           "wave_speeds": "frozen at time n",
                           "l2": "256 MiB buffer written between timed steps; basis traffic exceeds L2",
                           "parallelism": f"replicas x{world}"},
                "converged": converged,
                "newton_iters": [i.newton_iters for i in infos], "gmres_iters": [i.gmres_iters for i in infos],
                "realizability_violations": [i.realizability_violations for i in infos],
                "fallback_cells": [i.fallback_cells for i in infos],
                "per_dt_factor": per_dt,
                "plain_fp64": plain,
                "speedup_vs_plain_fp64": (value / world) / best_plain["value"] if best_plain else None,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": s1["kernel_launches"] - s0["kernel_launches"], "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
