"""Training recipe of the learned preconditioner (the library's own addition: the
paper has no learned component; its preconditioners are those of Sect. 3.3.2).

The network (m1_nn, include/m1.h) maps a Krylov vector, the log opacity and the
state at which the Jacobian is taken to the part of J^-1 v that point-block
Jacobi misses. Training pairs come from the plain solver's own Jacobians, on the
GPU (m1_nn_make_pair): for each seeded problem the Newton iterates U_0 = U^n,
U_1, ... of its mixed-precision point-block Jacobi solve, and at each iterate the
directions e = U_{k+1} - U_k (the Newton updates) and smooth random fields of
several correlation lengths (the Krylov vectors FGMRES feeds the network are
neither), and a zero direction (whose target is zero). Training is online: each round draws fresh problems, fills the pair
buffer on the device and runs Adam over it (m1_nn_train), so the number of
distinct pairs seen grows with the rounds while the buffer stays bounded.

Everything runs through the C ABI; torch provides device memory, the random
fields (its CUDA generator and FFT) and the stream.
"""
from __future__ import annotations

import math
import time
from typing import Callable, Dict, Iterable, List, Optional

import numpy as np

from .m1 import PREC_MIXED, PRECOND_BJ, Net, context_from_problem, default_opts

PRECOND_LEARNED = 2


def smooth_fields(ny: int, nx: int, ell: float, gen, count: int = 3):
    """`count` periodic Gaussian random fields (ny x nx, torch float64 on the GPU):
    white noise from `gen` filtered by exp(-2 pi^2 ell^2 |k|^2), each normalised to
    unit standard deviation. Returns a flat vector of count * ny * nx values."""
    import torch
    z = torch.randn((count, ny, nx), generator=gen, device="cuda", dtype=torch.float64)
    ky = torch.fft.fftfreq(ny, device="cuda", dtype=torch.float64).reshape(ny, 1)
    kx = torch.fft.fftfreq(nx, device="cuda", dtype=torch.float64).reshape(1, nx)
    mult = torch.exp(-2.0 * math.pi ** 2 * ell ** 2 * (ky * ky + kx * kx))
    g = torch.fft.ifft2(torch.fft.fft2(z) * mult).real
    g = g - g.mean(dim=(1, 2), keepdim=True)
    g = g / g.std(dim=(1, 2), keepdim=True).clamp_min(1e-300)
    return g.reshape(-1).contiguous()


def newton_iterates(ctx, dt: float, newton_max: int = 8) -> List:
    """U^n and the Newton iterates of the plain mixed-precision point-block Jacobi
    solve (torch float64 device vectors), up to convergence or newton_max."""
    import torch
    out = []
    U0 = torch.empty(ctx.nu * ctx.N, dtype=torch.float64, device="cuda")
    ctx.get_state_vector(U0)
    out.append(U0)
    for k in range(1, newton_max + 1):
        opts = default_opts(advance=0, precision=PREC_MIXED, precond=PRECOND_BJ, newton_max=k)
        st, info = ctx.implicit_step(dt, opts, raise_on_fail=False)
        U = torch.empty_like(U0)
        ctx.get_solution(U)
        out.append(U)
        if info.converged:
            break
    return out


def slow_modes(ctx, dt: float, U, e_true, krylov_steps: int):
    """The error e_true - x_k left after krylov_steps steps of point-block Jacobi
    GMRES (FP32 inner, from x = 0) on J(U) x = J(U) e_true: the components this
    preconditioner resolves slowly."""
    import torch
    b = torch.empty_like(e_true)
    ctx.jv(dt, U, e_true, out=b)
    x = torch.empty_like(e_true)
    opts = default_opts(precision=PREC_MIXED, precond=PRECOND_BJ, gmres_max=krylov_steps, gmres_rtol=1e-12,
                        refine_max=1)
    ctx.gmres_solve(dt, b, U=U, out=x, opts=opts, raise_on_fail=False)
    return e_true - x


def first_stage_pair(ctx, dt: float, U, e, x_out, t_out):
    """The pair of the error a point-block Jacobi stage leaves of e, e1 = e - J_bj^-1 J e
    (up to scale): the network's input is then r1 = J e1, the residual the two-stage
    forms hand it (m1_set_learned_form). The first m1_nn_make_pair gives e1 / s as its
    target; the second makes the pair of e1."""
    N = ctx.N
    ctx.make_pair(dt, e, U=U, out=(x_out, t_out))
    e1 = t_out.reshape(N, 3).t().contiguous().reshape(-1).double()
    ctx.make_pair(dt, e1, U=U, out=(x_out, t_out))


def collect_pairs(ctx, dt: float, X, T, start: int, gen, n_random: int = 6,
                  ells=(1.0, 2.0, 4.0, 8.0), newton_max: int = 8, krylov_steps: int = 0,
                  first_stage: bool = False) -> int:
    """Fill rows start, start + 1, ... of the device buffers X (pairs x N x 7) and
    T (pairs x N x 3) from this context; returns the next free row (stops at the
    buffer's end). krylov_steps > 0: the random directions are replaced by the
    error they leave after that many point-block Jacobi GMRES steps (slow_modes);
    first_stage: by the error one point-block Jacobi stage leaves (first_stage_pair)."""
    import torch
    cap = X.shape[0]
    i = start
    its = newton_iterates(ctx, dt, newton_max)
    ny, nx = ctx.shape2d
    for k, U in enumerate(its):
        dirs = [torch.zeros_like(U)]  # a zero residual: the correction must vanish
        if k + 1 < len(its):
            dirs.append(its[k + 1] - U)
        first = len(dirs)
        for q in range(n_random):
            e = smooth_fields(ny, nx, ells[q % len(ells)], gen)
            dirs.append(slow_modes(ctx, dt, U, e, krylov_steps) if krylov_steps > 0 else e)
        for j, e in enumerate(dirs):
            if i >= cap:
                return i
            if first_stage and j >= first:
                first_stage_pair(ctx, dt, U, e, X[i].reshape(-1), T[i].reshape(-1))
            else:
                ctx.make_pair(dt, e, U=U, out=(X[i].reshape(-1), T[i].reshape(-1)))
            i += 1
    return i


def train(problem: Callable[[int], object], seeds: Iterable[int], *, n: int, rounds: int, pairs_per_round: int,
          epochs: int = 2, lr: float = 1e-3, lr_final: float = 1e-4, batch: int = 4, n_random: int = 6,
          krylov_steps: int = 10, init: Optional[np.ndarray] = None, seed: int = 1,
          log: Optional[Callable[[str], None]] = None, first_stage: bool = False) -> Dict:
    """Online training on problems problem(seed) of n x n cells (2D, radiation only);
    the random directions are the slow modes of krylov_steps point-block Jacobi GMRES
    steps (0: the smooth fields themselves).

    Returns {"net": the training Net (batch `batch`), "params": FP32 parameters,
    "pairs": distinct pairs seen, "first_loss", "final_loss", "seconds"} with the
    learning rate decayed geometrically from lr to lr_final over the rounds."""
    import torch
    seeds = list(seeds)
    net = Net(n, n, batch, torch.cuda.current_stream().cuda_stream)
    if init is not None:
        net.set_params(np.asarray(init, dtype=np.float32))
    X = torch.empty((pairs_per_round, n * n, 7), dtype=torch.float32, device="cuda")
    T = torch.empty((pairs_per_round, n * n, 3), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    t0 = time.perf_counter()
    si = 0
    seen = 0
    first = None
    last = None
    for r in range(rounds):
        filled = 0
        while filled < pairs_per_round:
            p = problem(seeds[si % len(seeds)])
            si += 1
            ctx = context_from_problem(p, stream=torch.cuda.current_stream().cuda_stream, device=True)
            filled = collect_pairs(ctx, p.dt, X, T, filled, gen, n_random=n_random, krylov_steps=krylov_steps,
                                   first_stage=first_stage)
            ctx.close()
        seen += filled
        frac = r / max(rounds - 1, 1)
        lr_r = lr * (lr_final / lr) ** frac
        info = net.train(X, T, filled, epochs=epochs, lr=lr_r, seed=seed + r)
        if first is None:
            first = info["first_loss"]
        last = info["final_loss"]
        if log:
            log(f"round {r}: pairs {filled} (total {seen}), lr {lr_r:.2e}, loss {info['first_loss']:.4f} -> "
                f"{info['final_loss']:.4f}, {time.perf_counter() - t0:.1f}s")
    torch.cuda.synchronize()
    return {"net": net, "params": net.get_params(), "pairs": seen, "first_loss": first, "final_loss": last,
            "seconds": time.perf_counter() - t0}


def forward_flops(H: int, W: int) -> float:
    """Multiply-add FLOPs (2 per product) of one forward pass of the network on an H x W image."""
    per_level = {0: [(7, 16), (16, 16), (32, 16), (16, 3)], 1: [(16, 32), (32, 32), (64, 32), (32, 16)],
                 2: [(32, 32), (32, 32)]}
    f = 0.0
    for lvl, layers in per_level.items():
        pix = (H >> lvl) * (W >> lvl)
        f += sum(2.0 * 9 * ci * co * pix for ci, co in layers)
    return f


def compare(p, params: np.ndarray, repeats: int = 2, form: int = 0, **opt_kw) -> Dict:
    """One implicit step of problem p with FGMRES(30) + the learned preconditioner in
    the given form (m1_set_learned_form) against GMRES(30) + point-block Jacobi (both
    FP32 inner under FP64 refinement): Newton and Krylov steps, device time (best of
    `repeats`), and the solutions."""
    import torch
    s = torch.cuda.current_stream().cuda_stream
    out = {}
    for kind in ("bj", "learned"):
        ctx = context_from_problem(p, stream=s, device=True)
        infer = None
        opts = default_opts(advance=0, precision=PREC_MIXED, precond=PRECOND_BJ, **opt_kw)
        if kind == "learned":
            infer = Net(p.n[1], p.n[0], 1, s)
            infer.set_params(params)
            ctx.set_preconditioner(infer)
            ctx.set_learned_form(form)
            opts.precond = PRECOND_LEARNED
        best, info = None, None
        for _ in range(repeats):
            st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
            best = info.time_ms if best is None else min(best, info.time_ms)
        U = ctx.get_solution()
        out[kind] = {"converged": bool(info.converged), "newton_iters": info.newton_iters,
                     "gmres_iters": info.gmres_iters, "ms": best, "U": U}
        ctx.close()
        if infer is not None:
            infer.close()
    return out
