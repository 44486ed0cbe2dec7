"""Parity at the full sizes of the workloads, in the launch configuration bench.py times.

* beam_lognormal_2d 1024^2, dt = 10 dt_CFL (the bench workload): the FP64 residual and
  the FP64 and FP32 J v of the whole grid against the oracle, element by element
  (1e-12, 1e-12, 1e-4); the bench's implicit step (FP32 inner GMRES(30) with the
  multigrid preconditioner under FP64 refinement, full Newton steps, 1e-8) leaves an
  oracle residual within 1e-8 of ||R(U^n)|| (a property that holds at any size; an
  oracle Newton solve of 3 M unknowns is out of reach).
* two_slab_1d, 512 cells: 200 implicit steps at 10 dt_CFL (FP64 GMRES(30) with the
  block-tridiagonal line preconditioner, and with point-block Jacobi), each checked by
  the oracle's residual of the GPU's new state for that step (within 1e-8 of
  ||R(U^n)||), and 2000 explicit steps at dt_CFL against the oracle's march (1e-10 per
  field). At 50 dt_CFL the backward-Euler solution of the second step is not realizable
  (E < 0, |F| > cE, in the oracle's exact Newton as well) and Newton stalls by the fourth.
* gas_point_source_3d 256^3: the oracle evaluates windows of the grid. All sides of
  this workload are outflow, and a window cut out with outflow sides sees the true
  neighbours at every cell two or more cells inside a cut face, where the GPU's
  full-grid values are compared: the FP64 residual of a perturbed state (1e-12), and
  the oracle residual at the GPU's mixed-precision implicit step (within 1e-8 of the
  global ||R(U^n)||). Windows: the corner cell block, the point source, a seeded one.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme
from tests.m1_cases import perturbed_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m1mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2011_13926_gb300 import m1
    return m1


def _ctx(m1mod, p):
    import torch
    return m1mod.context_from_problem(p, stream=torch.cuda.current_stream().cuda_stream, device=True)


def _max_rel(got, want, nu, N):
    out = []
    for k in range(nu):
        a, b = got[k * N:(k + 1) * N], want[k * N:(k + 1) * N]
        out.append(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    return max(out)


# ----------------------------------------------------------------- 1024^2 beam
@pytest.fixture(scope="module")
def beam():
    p = si.beam_lognormal_2d(1024, dt_factor=10.0)
    return p, Scheme(p)


def test_beam_residual_and_jv_full_grid(m1mod, beam):
    p, s = beam
    ctx = _ctx(m1mod, p)
    u = perturbed_state(p, 31)
    assert _max_rel(ctx.residual(p.dt, u), s.residual(u), s.nu, s.N) < 1e-12
    v = np.random.default_rng(32).standard_normal(u.size)
    ref = s.jv(u, v)
    assert _max_rel(ctx.jv(p.dt, u, v, precision=m1mod.PREC_FP64), ref, s.nu, s.N) < 1e-12
    assert _max_rel(ctx.jv(p.dt, u, v, precision=m1mod.PREC_MIXED), ref, s.nu, s.N) < 1e-4
    ctx.close()


def test_beam_bench_step_solves_the_oracle_system(m1mod, beam):
    p, s = beam
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(advance=0, precision=m1mod.PREC_MIXED, precond=m1mod.PRECOND_MG, line_search=0)
    st, info = ctx.implicit_step(p.dt, opts)
    assert st == m1mod.M1_OK and info.converged
    u = ctx.get_solution()
    r0 = np.linalg.norm(s.residual(p.state_vector()))
    assert abs(info.res0 - r0) <= 1e-12 * r0
    assert np.linalg.norm(s.residual(u)) <= 1.05e-8 * r0
    ctx.close()


# ----------------------------------------------------------------- 1D two slabs, 512 cells
@pytest.mark.parametrize("pc", ["line", "bj"])
def test_slab_200_implicit_steps_each_solves_the_oracle_system(m1mod, pc):
    p = si.two_slab_1d(512, dt_factor=10.0)
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(precision=m1mod.PREC_FP64,
                              precond=m1mod.PRECOND_LINE if pc == "line" else m1mod.PRECOND_BJ)
    N = p.ncell
    q = p.copy()
    for k in range(200):
        st, info = ctx.implicit_step(p.dt, opts)
        assert st == m1mod.M1_OK and info.converged, k
        E, F, _ = ctx.get_state()
        s = Scheme(q)  # U^n: the GPU's previous state
        r0 = np.linalg.norm(s.residual(q.state_vector()))
        assert np.linalg.norm(s.residual(np.concatenate([E, F]))) <= 1.05e-8 * r0, k
        q.E, q.F = E.copy(), F.reshape(1, N).copy()
    ctx.close()


def test_slab_2000_explicit_steps(m1mod):
    p = si.two_slab_1d(512, dt_factor=1.0)
    ctx = _ctx(m1mod, p)
    q = p.copy()
    for _ in range(2000):
        ctx.explicit_step(p.dt)
        out = Scheme(q).explicit_step()
        q.E, q.F = out[0], np.stack(out[1:])
    E, F, _ = ctx.get_state()
    scale = np.abs(q.E).max()
    assert np.abs(E - q.E).max() <= 1e-10 * scale
    assert np.abs(F - q.F[0]).max() <= 1e-10 * p.c * scale
    ctx.close()


# ----------------------------------------------------------------- 256^3 gas point source
N3 = 256
W = 20


def _window(p, o):
    """The window of W^3 cells at corner o (x, y, z) as a problem with outflow sides,
    and the mask of its cells that see only true neighbours."""
    sl = tuple(slice(o[a], o[a] + W) for a in reversed(range(3)))
    q = si.make_problem(3, (W, W, W), lo=[0.0] * 3, hi=[W * p.dx[a] for a in range(3)], gas=True, dt=p.dt)
    for f in ("c", "a_r", "well_balanced", "ap_correction", "fixed_eigs", "lambda_floor", "wb_boundary",
              "implicit_eigs"):
        setattr(q, f, getattr(p, f))
    q.E, q.T, q.rho_cv = p.E[sl].copy(), p.T[sl].copy(), p.rho_cv[sl].copy()
    q.F = p.F[(slice(None),) + sl].copy()
    q.sigma_a, q.sigma_f = p.sigma_a[sl].copy(), p.sigma_f[sl].copy()
    q.S = p.S[sl].copy()
    q.B = None
    keep = np.ones((W, W, W), bool)
    for a in range(3):
        ax = 2 - a
        idx = [slice(None)] * 3
        if o[a] > 0:  # a cut face on the low side
            idx[ax] = slice(0, 2)
            keep[tuple(idx)] = False
        if o[a] + W < N3:  # a cut face on the high side
            idx[ax] = slice(W - 2, W)
            keep[tuple(idx)] = False
    return q, sl, keep


def _restrict(vec, sl, nu):
    """Window components of a full-grid vector [comp * N + cell]."""
    full = vec.reshape((nu, N3, N3, N3))
    return np.concatenate([full[k][sl].ravel() for k in range(nu)])


@pytest.fixture(scope="module")
def gas3d():
    p = si.gas_point_source_3d(N3)
    rng = np.random.default_rng(41)
    o = tuple(int(x) for x in rng.integers(W, N3 - 2 * W, size=3))
    h = N3 // 2 - W // 2
    return p, [(0, 0, 0), (h, h, h), o]


def test_gas3d_residual_windows(m1mod, gas3d):
    p, windows = gas3d
    ctx = _ctx(m1mod, p)
    u = perturbed_state(p, 42)
    R = ctx.residual(p.dt, u)
    ctx.close()
    nu = p.n_u
    for o in windows:
        q, sl, keep = _window(p, o)
        ref = Scheme(q).residual(_restrict(u, sl, nu)).reshape(nu, -1)
        got = _restrict(R, sl, nu).reshape(nu, -1)
        m = keep.ravel()
        for k in range(nu):
            scale = max(np.abs(ref[k][m]).max(), 1e-300)
            assert np.abs(got[k][m] - ref[k][m]).max() <= 1e-12 * scale, (o, k)


def test_gas3d_mixed_step_windows(m1mod, gas3d):
    p, windows = gas3d
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(advance=0, precision=m1mod.PREC_MIXED, gmres_max=3000)
    st, info = ctx.implicit_step(p.dt, opts)
    assert st == m1mod.M1_OK and info.converged
    u = ctx.get_solution()
    ctx.close()
    nu = p.n_u
    for o in windows:
        q, sl, keep = _window(p, o)
        R = Scheme(q).residual(_restrict(u, sl, nu)).reshape(nu, -1)[:, keep.ravel()]
        assert np.linalg.norm(R) <= 1.05e-8 * info.res0, o
