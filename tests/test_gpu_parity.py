"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs (element by element).

Tolerances (north-star): FP64 explicit step 1e-12 relative per field; FP64
residual, J v and point blocks 1e-12 relative per component (same formulas,
different rounding order); implicit solves within 1e-8 relative residual and
1e-7 relative in E and F; FP32 J v within 1e-4 relative (FP32 rounding of
U, v and every intermediate; the derivation is in the design notes).
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, dense_solve, newton_solve
from tests.m1_cases import cases, gas_3d, perturbed_state

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


def ctx_for(m1mod, p):
    import torch
    return m1mod.context_from_problem(p, stream=torch.cuda.current_stream().cuda_stream, device=True)


def rel_by_component(a, b, nu, N):
    out = []
    for k in range(nu):
        x, y = a[k * N:(k + 1) * N], b[k * N:(k + 1) * N]
        out.append(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))
    return out


CASES = cases()


@pytest.mark.parametrize("name", list(CASES))
def test_residual(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    u = perturbed_state(p, 1)
    ctx = ctx_for(m1mod, p)
    r_gpu = ctx.residual(p.dt, u)
    r_ref = s.residual(u)
    assert max(rel_by_component(r_gpu, r_ref, s.nu, s.N)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_jv_fp64(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    u = perturbed_state(p, 2)
    v = np.random.default_rng(3).standard_normal(u.size)
    ctx = ctx_for(m1mod, p)
    assert max(rel_by_component(ctx.jv(p.dt, u, v), s.jv(u, v), s.nu, s.N)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_jv_fp32(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    u = perturbed_state(p, 4)
    v = np.random.default_rng(5).standard_normal(u.size)
    ctx = ctx_for(m1mod, p)
    got = ctx.jv(p.dt, u, v, precision=m1mod.PREC_MIXED)
    ref = s.jv(u, v)
    # the FP32 kernel rounds U, v and sigma to FP32: compare in the norm of the result
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err


@pytest.mark.parametrize("name", list(CASES))
def test_diag_blocks(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    u = perturbed_state(p, 6)
    ctx = ctx_for(m1mod, p)
    got = ctx.diag_blocks(p.dt, u).reshape(s.nu, s.nu, s.N)  # [row, col, cell]
    ref = s.diag_blocks(u)  # [cell, row, col]
    ref = np.transpose(ref, (1, 2, 0))
    # relative to each cell's block: entries that cancel exactly in one rounding
    # order leave a few ulps of the block's scale in the other
    scale = np.abs(ref).max(axis=(0, 1), keepdims=True)
    assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(scale, 1e-300))


@pytest.mark.parametrize("name", ["slab1d", "beam2d", "gas3d"])
@pytest.mark.parametrize("wb", [True, False])
def test_explicit_step(m1mod, name, wb):
    p = CASES[name]()
    p.well_balanced = wb
    p.dt = p.dt_cfl  # CFL step
    ref = Scheme(p).explicit_step()
    ctx = ctx_for(m1mod, p)
    ctx.explicit_step(p.dt)
    E, F, T = ctx.get_state()
    fields = [(E, ref[0])] + [(F[b * p.ncell:(b + 1) * p.ncell], ref[1 + b]) for b in range(p.dim)]
    if p.gas:
        fields.append((T, ref[1 + p.dim]))
    # flux components are compared in units of c max|E| (a component that stays
    # zero in one rounding order keeps a few ulps of the transverse terms in the other)
    scaleE = np.abs(ref[0]).max()
    for k, (got, want) in enumerate(fields):
        want = np.asarray(want).ravel()
        scale = np.abs(want).max()
        if 1 <= k <= p.dim:
            scale = max(scale, p.c * scaleE)
        assert np.abs(got - want).max() <= 1e-12 * scale


def test_explicit_step_periodic_and_degenerate(m1mod):
    # periodic lines of length 1, 2 and 7; Sherman-Morrison and the small cases
    for n in ((7, 1), (7, 2), (7, 5)):
        p = si.make_problem(2, n, bc=[("periodic", "periodic")] * 2, dt_factor=1.0)
        rng = np.random.default_rng(sum(n))
        p.E = rng.uniform(0.5, 1.5, p.shape)
        p.F = 0.3 * rng.uniform(-1, 1, (2,) + p.shape) * p.E
        p.sigma_a = 10.0 ** rng.uniform(-1, 2, p.shape)
        p.sigma_f = p.sigma_a.copy()
        ref = Scheme(p).explicit_step()
        ctx = ctx_for(m1mod, p)
        ctx.explicit_step(p.dt)
        E, F, _ = ctx.get_state()
        scaleE = np.abs(ref[0]).max()
        assert np.abs(E - ref[0].ravel()).max() <= 1e-12 * scaleE
        for b in range(2):
            want = ref[1 + b].ravel()
            scale = max(np.abs(want).max(), p.c * scaleE)
            assert np.abs(F[b * p.ncell:(b + 1) * p.ncell] - want).max() <= 1e-12 * scale


@pytest.mark.parametrize("krylov", [0, 1], ids=["gmres", "bicgstab"])
@pytest.mark.parametrize("shape", [(8,), (4, 4), (3, 3, 3)])
def test_gmres_matches_dense_lu(m1mod, shape, krylov):
    dim = len(shape)
    if dim == 3:
        p = gas_3d(shape, seed=7)
    else:
        p = si.make_problem(dim, shape, dt_factor=20)
        rng = np.random.default_rng(8 + dim)
        p.E = rng.uniform(0.5, 2.0, p.shape)
        p.F = 0.4 * rng.uniform(-1, 1, (dim,) + p.shape) * p.E
        p.sigma_a = 10.0 ** rng.uniform(-1, 2, p.shape)
        p.sigma_f = p.sigma_a.copy()
    s = Scheme(p)
    u = perturbed_state(p, 9)
    b = np.random.default_rng(10).standard_normal(u.size)
    x_lu = dense_solve(s, u, b)
    ctx = ctx_for(m1mod, p)
    opts = m1mod.default_opts(gmres_rtol=1e-13, gmres_max=5000, krylov=krylov)
    x, info = ctx.gmres_solve(p.dt, b, U=u, opts=opts)
    assert info.converged
    assert np.linalg.norm(x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)


@pytest.mark.parametrize("name", list(CASES))
def test_implicit_step_fp64(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    assert ref.converged
    ctx = ctx_for(m1mod, p)
    opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0)
    st, info = ctx.implicit_step(p.dt, opts)
    assert info.converged
    # the device norm of R(U^n) (block partial sums, fixed-order finish) is the oracle's
    assert info.res0 == pytest.approx(ref.res0, rel=1e-12)
    u = ctx.get_solution()
    # the GPU result solves the oracle's system: relative residual <= 1e-8
    assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
    errs = rel_by_component(u, ref.u, s.nu, s.N)
    assert max(errs[:1 + p.dim]) < 1e-7, errs
    # realizability count: the same integer decision in FP64 on the same state
    assert info.realizability_violations == s.realizability_violations(u)


@pytest.mark.parametrize("name", list(CASES))
def test_implicit_step_mixed(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    ctx = ctx_for(m1mod, p)
    opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0, precision=m1mod.PREC_MIXED)
    st, info = ctx.implicit_step(p.dt, opts)
    assert info.converged
    u = ctx.get_solution()
    assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
    errs = rel_by_component(u, ref.u, s.nu, s.N)
    assert max(errs[:1 + p.dim]) < 1e-7, errs


def test_advance_and_state_roundtrip(m1mod):
    p = CASES["slab1d"]()
    ctx = ctx_for(m1mod, p)
    st, info = ctx.implicit_step(p.dt, m1mod.default_opts())
    assert info.converged
    E, F, _ = ctx.get_state()
    u = ctx.get_solution()
    assert np.array_equal(E, u[:p.ncell]) and np.array_equal(F, u[p.ncell:])


def test_not_converged_leaves_state(m1mod):
    p = CASES["beam2d"]()
    ctx = ctx_for(m1mod, p)
    E0, F0, _ = ctx.get_state()
    st, info = ctx.implicit_step(p.dt, m1mod.default_opts(newton_max=1, gmres_max=1), raise_on_fail=False)
    assert st == m1mod.M1_ERR_NOT_CONVERGED and not info.converged
    E1, F1, _ = ctx.get_state()
    assert np.array_equal(E0, E1) and np.array_equal(F0, F1)


def test_nonfinite_input_reported(m1mod):
    p = CASES["slab1d"]()
    p.E = p.E.copy()
    p.E[17] = np.nan
    ctx = ctx_for(m1mod, p)
    st, info = ctx.implicit_step(p.dt, m1mod.default_opts(), raise_on_fail=False)
    assert st == m1mod.M1_ERR_NONFINITE


@pytest.mark.parametrize("name", ["gas3d", "gas2d_frozen"])
def test_advection(m1mod, name):
    p = CASES[name]()
    rng = np.random.default_rng(12)
    u = []
    for a in range(p.dim):
        shp = list(p.shape)
        shp[p.dim - 1 - a] += 1
        u.append(rng.uniform(-0.5, 0.5, shp))
    ref = Scheme(p).advect_internal_energy(u)
    ctx = ctx_for(m1mod, p)
    ctx.set_velocity(*[np.ascontiguousarray(x).ravel() for x in u])
    ctx.advect(p.dt)
    _, _, T = ctx.get_state()
    assert np.abs(T - ref.ravel()).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["slab1d", "beam2d", "gas2d_frozen", "gas3d"])
def test_velocity_sources(m1mod, name):
    # explicit velocity-dependent sources (c = 1, |u| up to 0.3 c to exercise every term)
    p = CASES[name]()
    rng = np.random.default_rng(13)
    u = []
    for a in range(p.dim):
        shp = list(p.shape)
        shp[p.dim - 1 - a] += 1
        u.append(rng.uniform(-0.3, 0.3, shp))
    ref = Scheme(p).velocity_sources(u)
    ctx = ctx_for(m1mod, p)
    ctx.set_velocity(*[np.ascontiguousarray(x).ravel() for x in u])
    ctx.velocity_sources(p.dt)
    E, F, T = ctx.get_state()
    scale_E = np.abs(ref[0]).max()
    assert np.abs(E - ref[0].ravel()).max() <= 1e-12 * scale_E
    Fr = np.stack([np.asarray(x).ravel() for x in ref[1:1 + p.dim]])
    assert np.abs(np.asarray(F).reshape(p.dim, -1) - Fr).max() <= 1e-12 * p.c * scale_E
    if p.gas:
        assert np.abs(T - ref[1 + p.dim].ravel()).max() <= 1e-12 * np.abs(ref[1 + p.dim]).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_krylov_is_deterministic(m1mod, prec):
    # fixed-order reductions: the same solve twice gives bit-identical results
    p = si.beam_lognormal_2d(96, 70, dt_factor=10.0)
    ctx = ctx_for(m1mod, p)
    b = np.random.default_rng(21).standard_normal(3 * p.ncell)
    opts = m1mod.default_opts(precision=prec, gmres_rtol=1e-8, gmres_max=400)
    x1, i1 = ctx.gmres_solve(p.dt, b, opts=opts, raise_on_fail=False)
    x2, i2 = ctx.gmres_solve(p.dt, b, opts=opts, raise_on_fail=False)
    assert i1.iters == i2.iters
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("prec,pc", [(0, 1), (1, 1), (1, 3)], ids=["fp64-bj", "mixed-bj", "mixed-mg"])
def test_implicit_step_bicgstab(m1mod, prec, pc):
    # the paper's Krylov solver inside the same Newton step meets the implicit parity bar
    p = CASES["beam2d"]()
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    assert ref.converged
    ctx = ctx_for(m1mod, p)
    opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0, precision=prec, precond=pc,
                              krylov=m1mod.KRYLOV_BICGSTAB)
    st, info = ctx.implicit_step(p.dt, opts)
    assert info.converged
    u = ctx.get_solution()
    assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
    errs = rel_by_component(u, ref.u, s.nu, s.N)
    assert max(errs[:1 + p.dim]) < 1e-7, errs


@pytest.mark.parametrize("fixed_eigs", [False, True])
def test_beam_45_sect53(m1mod, fixed_eigs):
    # The Sect. 5.3 beam (128^2, sigma = 0, 45 degrees) marched with the GPU's
    # semi-implicit step: 64 steps against the oracle's march (1e-8 per field: the
    # beam has f = 1, where the eigenvalues go as sqrt(1 - f), so rounding
    # differences of eps in f become sqrt(eps) in lambda and are carried on),
    # then to steady state, where the mid-height width (FWHM) matches the oracle's
    # (22 cells with computed eigenvalues, 27 with fixed +-c; paper 24 and 30).
    from tests.m1_cases import beam_45_oracle, midheight_fwhm
    n = 128
    p = si.beam_45_2d(n, fixed_eigs)
    ctx = ctx_for(m1mod, p)
    for _ in range(64):
        ctx.explicit_step(p.dt)
    ref = beam_45_oracle(n, fixed_eigs, 64 * p.dt)
    E, F, _ = ctx.get_state()
    N = p.ncell
    assert np.abs(E - ref.E.ravel()).max() <= 1e-8 * np.abs(ref.E).max()
    for b in range(2):
        assert np.abs(F[b * N:(b + 1) * N] - ref.F[b].ravel()).max() <= 1e-8 * p.c * np.abs(ref.E).max()
    widths, done = [], 64
    for t_end in (4.0, 5.0):
        for _ in range(int(round(t_end / p.dt)) - done):
            ctx.explicit_step(p.dt)
        done = int(round(t_end / p.dt))
        widths.append(midheight_fwhm(ctx.get_state()[0].reshape(n, n)))
    assert widths[0] == widths[1]  # steady at mid-height
    assert widths[1] == (27 if fixed_eigs else 22)


@pytest.mark.parametrize("periodic,gas,n", [(False, False, 12), (False, True, 12), (True, False, 12),
                                            (False, False, 300)])
@pytest.mark.parametrize("arith", ["native", "double_word"])
def test_line_preconditioner_matches_dense_lu(m1mod, periodic, gas, n, arith):
    # M1_PRECOND_LINE: on a non-periodic 1D grid the preconditioner is J itself, and
    # GMRES takes one step (two at most: the convergence test runs one step behind).
    # The line factors are built with FP64 operations; with the J v in double words
    # the two differ by ~1e-14 relative, and GMRES takes a few more steps to 1e-13.
    from tests.m1_cases import line_case_1d
    p = line_case_1d(periodic, gas, n=n)
    s = Scheme(p)
    u = perturbed_state(p, 64)
    b = np.random.default_rng(65).standard_normal(u.size)
    x_lu = dense_solve(s, u, b)
    ctx = ctx_for(m1mod, p)
    ctx.set_fp64_arithmetic(m1mod.FP64_NATIVE if arith == "native" else m1mod.FP64_DOUBLE_WORD)
    opts = m1mod.default_opts(gmres_rtol=1e-13, gmres_max=300, precond=m1mod.PRECOND_LINE)
    x, info = ctx.gmres_solve(p.dt, b, U=u, opts=opts)
    assert info.converged
    assert np.linalg.norm(x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)
    if not periodic:
        assert info.iters <= (2 if arith == "native" else 10), info.iters


def test_line_preconditioner_rejects_unsupported(m1mod):
    from tests.m1_cases import line_case_1d
    p1 = line_case_1d(False, False)
    ctx = ctx_for(m1mod, p1)
    o = m1mod.default_opts(precision=m1mod.PREC_MIXED, precond=m1mod.PRECOND_LINE, advance=0)
    st, info = ctx.implicit_step(p1.dt, o, raise_on_fail=False)
    assert st == m1mod.M1_ERR_ARG
    p2 = si.beam_lognormal_2d(24, 20, dt_factor=10.0)
    ctx2 = ctx_for(m1mod, p2)
    o = m1mod.default_opts(precision=m1mod.PREC_FP64, precond=m1mod.PRECOND_LINE, advance=0)
    st, info = ctx2.implicit_step(p2.dt, o, raise_on_fail=False)
    assert st == m1mod.M1_ERR_ARG
