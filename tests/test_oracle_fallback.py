"""Pins of the oracle's admissibility fallback (CPU only).

Sect. 3.1.3 leaves open whether the AP + WB scheme keeps f = |F|/(cE) <= 1, and
names the centred source of Eq. (wb_naive) as a remedy. The fallback of the
oracle (Scheme(fallback=mask)) gives a flagged cell the centred source, and the
faces of a flagged cell alpha = 1 and the speeds -c, +c. Pinned here:

* with every cell flagged it IS the HLL scheme with fixed speeds and the centred
  source (the flags fixed_eigs, ap_correction = 0, well_balanced = 0);
* the property of the M1 closure behind that scheme's admissibility: for an
  admissible U, U + F_a(U)/c and U - F_a(U)/c are admissible (F_a the physical
  flux along axis a), so the backward-Euler update, (1 + sum_a 2 nu_a) U_i =
  U_i^n + sum_a nu_a [(U + F_a/c)_{i-1} + (U - F_a/c)_{i+1}] + (sources that
  keep the set when sigma_f >= sigma_a, as with the paper's single sigma) with
  nu_a = c dt / (2 dx_a), is a convex combination;
* that update is admissible for any dt (Newton to convergence, dense LU);
* the a posteriori loop of newton_solve(realizability=True) on the 2D beam at
  50 and 100 dt_CFL and on the 1D two-slab problem at 50 dt_CFL: converged, and
  every cell admissible, where the plain AP + WB solution is not.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Closure, Scheme, newton_solve


def random_problem(dim, rng, bc, fmax=0.95):
    n = (9,) if dim == 1 else (7, 6)
    p = si.make_problem(dim, n, bc=bc, dt_factor=30.0)
    p.E = rng.uniform(0.2, 2.0, p.shape)
    d = rng.standard_normal((dim,) + p.shape)
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    p.F = p.c * p.E * rng.uniform(0.0, fmax, p.shape) * d
    p.sigma_a = 10.0 ** rng.uniform(-1.0, 2.5, p.shape)
    p.sigma_f = p.sigma_a + 10.0 ** rng.uniform(-1.0, 2.5, p.shape)  # flux opacity = absorption + scattering
    p.B = rng.uniform(0.0, 1.0, p.shape)
    p.implicit_eigs = False
    if any(k == "dirichlet" for k in bc[0]):
        M = p.ncell // p.n[0]
        fshape = p.shape[:-1]
        p.boundary[(0, 0)] = (np.full(fshape, 1.5), np.stack([np.full(fshape, 1.2)] + [np.zeros(fshape)] * (dim - 1)),
                              (np.arange(M) % 2).reshape(fshape).astype(np.uint8))
    return p


BCS = {1: [[("dirichlet", "outflow")], [("periodic", "periodic")]],
       2: [[("dirichlet", "outflow"), ("periodic", "periodic")], [("outflow", "reflect"), ("outflow", "outflow")]]}


@pytest.mark.parametrize("dim,k", [(1, 0), (1, 1), (2, 0), (2, 1)])
def test_full_fallback_is_hll_fixed_speeds_centred_source(dim, k):
    rng = np.random.default_rng(10 + 2 * dim + k)
    p = random_problem(dim, rng, BCS[dim][k])
    u = p.state_vector() * (1.0 + 0.1 * rng.standard_normal(p.ncell * p.n_u))
    flagged = Scheme(p, fallback=np.ones(p.shape, bool))
    q = p.copy()
    q.fixed_eigs, q.ap_correction, q.well_balanced = True, False, False
    plain = Scheme(q)
    np.testing.assert_allclose(flagged.residual(u), plain.residual(u), rtol=0, atol=1e-13 * np.abs(u).max())
    # an empty mask is the scheme itself
    np.testing.assert_array_equal(Scheme(p, fallback=np.zeros(p.shape, bool)).residual(u), Scheme(p).residual(u))


def test_flagged_cell_changes_only_its_own_stencil():
    rng = np.random.default_rng(3)
    p = random_problem(2, rng, BCS[2][1])
    u = p.state_vector()
    mask = np.zeros(p.shape, bool)
    mask[3, 2] = True
    R0 = Scheme(p).residual(u).reshape(p.n_u, *p.shape)
    R1 = Scheme(p, fallback=mask).residual(u).reshape(p.n_u, *p.shape)
    changed = np.any(R0 != R1, axis=0)
    assert changed[3, 2]
    near = np.zeros(p.shape, bool)  # the cell and its four neighbours (faces shared with it)
    for dy, dx in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
        near[3 + dy, 2 + dx] = True
    assert not np.any(changed & ~near)


@pytest.mark.parametrize("dim", [2, 3])
def test_m1_flux_split_is_admissible(dim):
    """For |f| <= 1: E +- F_a/c >= 0 and |F +- c P_a.| <= c E +- F_a (E = 1, brute force)."""
    g = np.linspace(-1.0, 1.0, 81 if dim == 2 else 25)
    mesh = np.meshgrid(*([g] * dim), indexing="ij")
    f = np.stack([m.ravel() for m in mesh])
    nrm = np.linalg.norm(f, axis=0)
    f = f[:, nrm <= 1.0]
    f = np.concatenate([f, f / np.maximum(np.linalg.norm(f, axis=0), 1e-300) * (1.0 - 1e-12)], axis=1)
    c = 1.0
    E = np.ones(f.shape[1])
    cl = Closure(E, [f[b] for b in range(dim)], c)
    for a in range(dim):
        for sgn in (1.0, -1.0):
            E2 = E + sgn * f[a]
            G = np.stack([f[b] + sgn * c * cl.pressure(a, b) for b in range(dim)])
            assert np.all(E2 >= -1e-12)
            assert np.all(np.linalg.norm(G, axis=0) <= c * E2 + 1e-12)


@pytest.mark.parametrize("dim,k", [(1, 0), (1, 1), (2, 0), (2, 1)])
def test_full_fallback_backward_euler_is_admissible(dim, k):
    rng = np.random.default_rng(20 + 2 * dim + k)
    p = random_problem(dim, rng, BCS[dim][k], fmax=0.99)
    for factor in (1.0, 30.0, 1000.0):
        p.dt = factor * p.dt_cfl
        s = Scheme(p, fallback=np.ones(p.shape, bool))
        r = newton_solve(s, rtol=1e-12, newton_max=40, dense=True)
        assert r.converged
        assert not s.inadmissible(r.u).any(), factor


@pytest.mark.parametrize("factor", [50.0, 100.0])
def test_fallback_loop_beam(factor):
    p = si.beam_lognormal_2d(32, ell=1.0, dt_factor=factor)
    plain = newton_solve(Scheme(p), rtol=1e-8, gmres_rtol=1e-6)
    assert plain.converged and Scheme(p).inadmissible(plain.u).sum() > 50  # the AP + WB solution is not admissible
    r = newton_solve(Scheme(p), rtol=1e-8, gmres_rtol=1e-6, newton_max=60, realizability=True)
    assert r.converged and r.fallback_rounds >= 1
    assert not Scheme(p).inadmissible(r.u).any()
    assert r.fallback.sum() < 0.25 * p.ncell
    # the result solves the flagged scheme from U^n
    s = Scheme(p, fallback=r.fallback)
    R0 = np.linalg.norm(s.residual(p.state_vector()))
    assert np.linalg.norm(s.residual(r.u)) <= 1.0001e-8 * R0


def test_fallback_loop_two_slab_50():
    p = si.two_slab_1d(128, dt_factor=50.0)
    n = p.ncell
    saw_inadmissible = False
    for step in range(10):
        plain = newton_solve(Scheme(p), rtol=1e-8, newton_max=40, dense=True)
        saw_inadmissible |= bool(plain.converged and Scheme(p).inadmissible(plain.u).any())
        r = newton_solve(Scheme(p), rtol=1e-8, newton_max=60, dense=True, realizability=True)
        assert r.converged, step
        assert not Scheme(p).inadmissible(r.u).any(), step
        p.E = r.u[:n].copy()
        p.F = r.u[n:].reshape(1, n).copy()
    assert saw_inadmissible
