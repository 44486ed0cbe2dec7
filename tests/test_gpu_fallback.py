"""GPU parity of the admissibility fallback of the implicit step (realizability = 1).

Sect. 3.1.3 leaves f > 1 possible with the AP + WB scheme and names the centred source
as a remedy; the library flags cells a posteriori (see m1_solver_opts.realizability).
Several flagged sets can be valid (they depend on the Newton iterates, which differ
between the FP64 oracle and the GPU's mixed-precision path), so the tests check what
is unique once the GPU's set is fixed:

* the GPU state is admissible (E > 0, |F| <= cE in every cell);
* it solves the oracle's scheme with the GPU's flagged set: the oracle residual is
  within 1e-8 of ||R(U^n)|| of that scheme;
* on small grids the oracle's own Newton with that set (flagging more only if its
  iterates need it) reaches the same state within 1e-7 per field.

Workloads: the 2D beam (32^2 with 1-cell correlation length, and the full 1024^2
bench grid) at 50 and 100 dt_CFL, where the plain AP + WB solution leaves the
admissible set, and the 512-cell two-slab problem at 50 dt_CFL for its 200 steps.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, newton_solve

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


def _oracle_residual_ratio(p, mask, u):
    s = Scheme(p, fallback=mask.reshape(p.shape))
    r0 = np.linalg.norm(s.residual(p.state_vector()))
    return np.linalg.norm(s.residual(u)) / r0, s


PATHS = {"fp64_bj": dict(precision=0, precond=1), "mixed_mg": dict(precision=1, precond=3, line_search=0)}


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("factor", [50.0, 100.0])
def test_beam_small_fallback_parity(m1mod, factor, path):
    p = si.beam_lognormal_2d(32, ell=1.0, dt_factor=factor)
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(advance=0, realizability=1, newton_rtol=1e-10, gmres_rtol=1e-8, newton_max=80,
                              **PATHS[path])
    st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
    assert st == m1mod.M1_OK and info.converged, info.as_dict()
    u = ctx.get_solution()
    mask = ctx.get_fallback()
    ctx.close()
    assert info.realizability_violations == 0 and info.fallback_cells == int(mask.sum()) > 0
    ratio, s = _oracle_residual_ratio(p, mask, u)
    assert not s.inadmissible(u).any()
    assert ratio <= 1.05e-10, ratio
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8, newton_max=60, realizability=True)
    assert ref.converged
    if ref.fallback.sum() == mask.sum():  # the oracle needed no further cell: one system, one root
        assert _max_rel(u, ref.u, s.nu, s.N) < 1e-7


def test_two_slab_200_steps_at_50(m1mod):
    """The two-slab workload's 200 backward-Euler steps at 50 dt_CFL (FP64 GMRES(30), line preconditioner)."""
    p = si.two_slab_1d(512, dt_factor=50.0)
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(realizability=1, precond=m1mod.PRECOND_LINE, newton_max=60)
    n = p.ncell
    flagged = []
    for step in range(200):
        st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
        assert st == m1mod.M1_OK and info.converged, (step, info.as_dict())
        u = ctx.get_solution()
        mask = ctx.get_fallback()
        assert info.realizability_violations == 0, step
        if step % 20 == 0 or step < 5:
            ratio, s = _oracle_residual_ratio(p, mask, u)
            assert ratio <= 1.05e-8, (step, ratio)
            assert not s.inadmissible(u).any(), step
        flagged.append(int(mask.sum()))
        p.E = u[:n].copy()
        p.F = u[n:].reshape(1, n).copy()
    ctx.close()
    # the flagged cells sit where the pulse streams freely (the thin slab and the fronts)
    assert max(flagged) < n // 2, flagged


@pytest.mark.parametrize("factor", [50.0, 100.0])
def test_beam_1024_fallback(m1mod, factor):
    """The bench grid at 50 and 100 dt_CFL on the bench's path (mixed, multigrid, full steps)."""
    p = si.beam_lognormal_2d(1024, dt_factor=factor)
    ctx = _ctx(m1mod, p)
    opts = m1mod.default_opts(advance=0, realizability=1, precision=m1mod.PREC_MIXED, precond=m1mod.PRECOND_MG,
                              line_search=0, newton_max=60)
    st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
    assert st == m1mod.M1_OK and info.converged, info.as_dict()
    u = ctx.get_solution()
    mask = ctx.get_fallback()
    ctx.close()
    assert info.realizability_violations == 0
    ratio, s = _oracle_residual_ratio(p, mask, u)
    assert ratio <= 1.05e-8, ratio
    assert not s.inadmissible(u).any()
