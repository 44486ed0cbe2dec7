"""GPU parity of the multigrid preconditioner (M1_PRECOND_MG) against oracle/mg.py.

Tolerances: stencil blocks are FP32 (assembled, or read off FP32 J v probes), so each block row is
compared to 2e-5 of its largest entry; one V-cycle runs in FP32 through
~30 damped sweeps of the level operators, compared to 2e-4 in the 2-norm.
The implicit step with the multigrid preconditioner meets the FP64 implicit
parity bar (1e-8 residual, 1e-7 state) with fewer Krylov steps than
point-block Jacobi.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, newton_solve
from oracle import mg as omg
from tests.m1_cases import gas_2d, gas_3d, perturbed_state

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


def _periodic(p):
    return p.bc[0][0] == "periodic", p.bc[1][0] == "periodic"


def _row_rel(got, ref):
    """max over (row, cell) of |got - ref| / max |ref| over that row's five blocks."""
    scale = np.abs(ref).max(axis=(0, 2))  # (nu, N)
    err = np.abs(got - ref).max(axis=(0, 2))
    return float((err / np.maximum(scale, 1e-300)).max())


@pytest.mark.parametrize("shape", [(24, 20), (80, 72), (67, 45)])
def test_stencil_levels_match_oracle(m1mod, shape):
    nx, ny = shape
    p = si.beam_lognormal_2d(nx, ny, dt_factor=10.0)
    s = Scheme(p)
    u = perturbed_state(p, 21)
    px, py = _periodic(p)
    ctx = _ctx(m1mod, p)
    r = np.random.default_rng(22).standard_normal(u.size)
    ctx.mg_apply(p.dt, r, U=u)
    H = omg.Hierarchy(lambda v: s.jv(u, v), s.nu, nx, ny, px, py)
    assert ctx.mg_levels() == len(H.ops)
    for lvl, (A, (lx, ly)) in enumerate(zip(H.ops, H.sizes)):
        got = ctx.mg_blocks(lvl, lx, ly)
        assert _row_rel(got, A) < 2e-5, (lvl, _row_rel(got, A))


# 2 to 6 levels; (280, 264) runs four tiled coarse levels (140 x 132 down to 18 x 17)
@pytest.mark.parametrize("shape", [(24, 20), (80, 72), (67, 45), (280, 264)])
def test_cycle_matches_oracle(m1mod, shape):
    nx, ny = shape
    p = si.beam_lognormal_2d(nx, ny, dt_factor=10.0)
    s = Scheme(p)
    u = perturbed_state(p, 23)
    px, py = _periodic(p)
    ctx = _ctx(m1mod, p)
    H = omg.Hierarchy(lambda v: s.jv(u, v), s.nu, nx, ny, px, py)
    rng = np.random.default_rng(24)
    for _ in range(2):
        r = rng.standard_normal(u.size)
        got = ctx.mg_apply(p.dt, r, U=u)
        ref = H.cycle(r)
        assert np.linalg.norm(got - ref) <= 2e-4 * np.linalg.norm(ref)


def test_cycle_with_gas_coupling_matches_oracle(m1mod):
    # n_u = 4: the level-0 stencil is probed through J v
    p = gas_2d()
    s = Scheme(p)
    u = perturbed_state(p, 27)
    px, py = _periodic(p)
    ctx = _ctx(m1mod, p)
    H = omg.Hierarchy(lambda v: s.jv(u, v), s.nu, p.n[0], p.n[1], px, py)
    r = np.random.default_rng(28).standard_normal(u.size)
    got = ctx.mg_apply(p.dt, r, U=u)
    for lvl, (A, (lx, ly)) in enumerate(zip(H.ops, H.sizes)):
        assert _row_rel(ctx.mg_blocks(lvl, lx, ly), A) < 2e-5, lvl
    assert np.linalg.norm(got - H.cycle(r)) <= 2e-4 * np.linalg.norm(H.cycle(r))


def test_cycle_is_linear_on_gpu(m1mod):
    p = si.beam_lognormal_2d(80, 72, dt_factor=10.0)
    u = perturbed_state(p, 25)
    ctx = _ctx(m1mod, p)
    rng = np.random.default_rng(26)
    r1, r2 = rng.standard_normal(u.size), rng.standard_normal(u.size)
    z1 = ctx.mg_apply(p.dt, r1, U=u)
    z2 = ctx.mg_apply(p.dt, r2, U=u)
    z = ctx.mg_apply(p.dt, 2.0 * r1 - 3.0 * r2, U=u)
    assert np.linalg.norm(z - (2.0 * z1 - 3.0 * z2)) <= 1e-5 * np.linalg.norm(z)


def test_implicit_step_with_multigrid(m1mod):
    p = si.beam_lognormal_2d(64, 48, dt_factor=10.0)
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    assert ref.converged
    iters = {}
    for name, pc in (("bj", m1mod.PRECOND_BJ), ("mg", m1mod.PRECOND_MG)):
        ctx = _ctx(m1mod, p)
        opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0,
                                  precision=m1mod.PREC_MIXED, precond=pc)
        st, info = ctx.implicit_step(p.dt, opts)
        assert info.converged
        u = ctx.get_solution()
        assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
        N = s.N
        for k in range(1 + p.dim):
            a, b = u[k * N:(k + 1) * N], ref.u[k * N:(k + 1) * N]
            assert np.abs(a - b).max() <= 1e-7 * max(np.abs(b).max(), 1e-300)
        iters[name] = info.gmres_iters
    print("Krylov steps per step:", iters)
    assert iters["mg"] < iters["bj"], iters


def test_multigrid_rejects_unsupported(m1mod):
    p3 = gas_3d()  # 3D
    ctx = _ctx(m1mod, p3)
    o = m1mod.default_opts(precision=m1mod.PREC_MIXED, precond=m1mod.PRECOND_MG, advance=0)
    st, info = ctx.implicit_step(p3.dt, o, raise_on_fail=False)
    assert st == m1mod.M1_ERR_ARG
    p2 = si.beam_lognormal_2d(24, 20, dt_factor=10.0)
    ctx2 = _ctx(m1mod, p2)
    o = m1mod.default_opts(precision=m1mod.PREC_FP64, precond=m1mod.PRECOND_MG, advance=0)
    st, info = ctx2.implicit_step(p2.dt, o, raise_on_fail=False)
    assert st == m1mod.M1_ERR_ARG


def test_implicit_step_with_lagged_multigrid(m1mod):
    # the hierarchy rebuilt on every third Newton step only: the cycle applies the
    # current J on level 0 with older smoothers and coarse operators; the step
    # still meets the FP64 bar
    p = si.beam_lognormal_2d(64, 48, dt_factor=10.0)
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0, precision=m1mod.PREC_MIXED,
                              precond=m1mod.PRECOND_MG, pc_rebuild=3)
    st, info = ctx.implicit_step(p.dt, opts)
    assert info.converged
    u = ctx.get_solution()
    assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
    N = s.N
    for k in range(1 + p.dim):
        a, b = u[k * N:(k + 1) * N], ref.u[k * N:(k + 1) * N]
        assert np.abs(a - b).max() <= 1e-7 * max(np.abs(b).max(), 1e-300)
