"""Pins of the oracle's scheme and solvers (CPU only).

* free streaming: F = cE, dt = dx/c shifts the state by exactly one cell;
  an inflow front moves at c;
* conservation of sum E (sigma_a = 0) and of sum (E + rho c_v T);
* well-balanced steady state across an opacity jump (Sect. 3.1.2): zero flux
  residual with the WB source, an O(1) one with the centred source;
* Appendix B: the WB source solve damps Fourier mode k by exactly
  1/(1 + 2r(1 + cos 2 pi k dx)) and is non-expansive for any sigma >= 0;
* realizability |F| <= cE of the HLL step at the CFL step dx/(c d)
  (alpha = 1, centred source, one opacity);
* asymptotic preservation: one thick implicit step equals the discrete
  diffusion scheme Eq. (discreteDiffusionEqua), HLL without alpha does not;
* J v against central differences, point blocks against the dense Jacobian,
  GMRES against dense LU, Newton's quadratic tail.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, dense_jacobian, dense_solve, gmres, newton_solve
from oracle.solvers import block_jacobi


def random_state(p, rng, fmax=0.9, Elo=0.2, Ehi=2.0):
    E = rng.uniform(Elo, Ehi, p.shape)
    n = rng.standard_normal((p.dim,) + p.shape)
    n /= np.linalg.norm(n, axis=0, keepdims=True)
    f = rng.uniform(0.0, fmax, p.shape)
    p.E = E
    p.F = p.c * E * f * n
    if p.gas:
        p.T = rng.uniform(0.5, 1.5, p.shape)
        p.rho_cv = rng.uniform(0.5, 2.0, p.shape)
    return p


# --------------------------------------------------------------------- transport

@pytest.mark.parametrize("dim", [1, 2])
def test_free_streaming_shift(dim):
    rng = np.random.default_rng(1)
    n = (12,) if dim == 1 else (12, 5)
    p = si.make_problem(dim, n, bc=[("periodic", "periodic")] * dim)
    p.E = rng.uniform(0.5, 2.0, p.shape)
    p.F = np.zeros((dim,) + p.shape)
    p.F[0] = p.c * p.E
    p.B = np.zeros(p.shape)
    p.dt = p.dx[0] / p.c
    out = Scheme(p).explicit_step()
    ax = dim - 1
    assert np.allclose(out[0], np.roll(p.E, 1, axis=ax), rtol=1e-13, atol=0)
    assert np.allclose(out[1], np.roll(p.F[0], 1, axis=ax), rtol=1e-13, atol=0)


def test_front_speed():
    n = 200
    p = si.make_problem(1, (n,), bc=[("dirichlet", "outflow")], well_balanced=False)
    p.boundary[(0, 0)] = (np.array(1.0), np.array([1.0]), np.array(1))
    p.B = np.zeros(n)
    p.dt = 0.5 * p.dx[0] / p.c
    steps = 200
    for _ in range(steps):
        out = Scheme(p).explicit_step()
        p.E, p.F = out[0], np.array([out[1]])
    x = p.centers(0)
    front = x[np.argmin(np.abs(p.E - 0.5))]
    assert abs(front - p.c * steps * p.dt) <= 2 * p.dx[0]


# --------------------------------------------------------------------- conservation

@pytest.mark.parametrize("dim", [1, 2])
def test_energy_conservation_explicit(dim):
    rng = np.random.default_rng(2 + dim)
    n = (16,) if dim == 1 else (10, 7)
    p = si.make_problem(dim, n, bc=[("periodic", "periodic")] * dim, dt_factor=0.5)
    random_state(p, rng)
    p.sigma_f = rng.uniform(0.0, 50.0, p.shape)
    p.sigma_a = np.zeros(p.shape)
    out = Scheme(p).explicit_step()
    assert out[0].sum() == pytest.approx(p.E.sum(), rel=1e-13)


def test_total_energy_conservation_gas():
    rng = np.random.default_rng(5)
    p = si.make_problem(2, (9, 8), bc=[("periodic", "periodic")] * 2, gas=True, dt_factor=0.5)
    random_state(p, rng)
    p.sigma_a = rng.uniform(0.0, 30.0, p.shape)
    p.sigma_f = p.sigma_a.copy()
    tot0 = (p.E + p.rho_cv * p.T).sum()
    out = Scheme(p).explicit_step()
    assert (out[0] + p.rho_cv * out[3]).sum() == pytest.approx(tot0, rel=1e-13)
    # implicit step: the E and T residual rows sum to (E + rho c_v T) - (...)^n
    p.dt = 5 * p.dt_cfl
    s = Scheme(p)
    res = newton_solve(s, rtol=1e-11)
    assert res.converged
    U = s.unpack(res.u)
    assert (U[0] + p.rho_cv * U[3]).sum() == pytest.approx(tot0, rel=1e-10)


# --------------------------------------------------------------------- well-balanced

def _steady_state(sig, F0, dx, c, E_right):
    """E with c (P_xx(E_{i+1}) - P_xx(E_i))/dx = -sigma_{i+1/2} F0 at F = F0 (1D),
    marched from the right end; P_xx from the oracle closure, root by bisection."""
    from oracle.m1 import Closure

    def pxx(E):
        cl = Closure(np.array([E]), [np.array([F0])], c)
        return cl.pressure(0, 0)[0]

    n = sig.size
    E = np.zeros(n)
    E[-1] = E_right
    for i in range(n - 2, -1, -1):
        s_face = 0.5 * (sig[i] + sig[i + 1])
        target = pxx(E[i + 1]) + s_face * F0 * dx / c
        lo, hi = E[i + 1], E[i + 1] + 10 * s_face * F0 * dx / c + 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if pxx(mid) < target:
                lo = mid
            else:
                hi = mid
        E[i] = 0.5 * (lo + hi)
    return E


def test_well_balanced_steady_flux():
    n = 40
    p = si.make_problem(1, (n,), bc=[("dirichlet", "dirichlet")], fixed_eigs=True)
    x = p.centers(0)
    sig = np.where(x < 0.5, 400.0, 0.5)
    p.sigma_a = np.zeros(n)
    p.sigma_f = sig
    F0 = 0.01
    E = _steady_state(np.concatenate([[sig[0]], sig, [sig[-1]]]), F0, p.dx[0], p.c, 1.0)
    p.E = E[1:-1].copy()
    p.F = np.full((1, n), F0)
    p.boundary[(0, 0)] = (np.array(E[0]), np.array([F0]), np.array(1))
    p.boundary[(0, 1)] = (np.array(E[-1]), np.array([F0]), np.array(1))
    p.dt = 10 * p.dt_cfl
    s = Scheme(p)
    R = s.residual_comps(s.Un)
    scale = p.dt * p.c * np.abs(sig * F0).max()
    assert np.abs(R[1]).max() <= 1e-12 * scale
    p.well_balanced = False
    R = Scheme(p).residual_comps(Scheme(p).Un)
    assert np.abs(R[1]).max() >= 0.05 * scale


def test_wb_source_fourier_damping():
    n, sigma, dt = 32, 7.0, 0.3
    p = si.make_problem(1, (n,), bc=[("periodic", "periodic")], dt=dt)
    p.sigma_f[:] = sigma
    s = Scheme(p)
    r = p.c * sigma * dt / 4.0
    for k in (0, 1, 5, 16):
        mode = np.cos(2 * np.pi * k * np.arange(n) / n)
        out = s._wb_implicit_solve(mode, 0)
        amp = 1.0 / (1.0 + 2.0 * r * (1.0 + np.cos(2 * np.pi * k / n)))
        assert np.allclose(out, amp * mode, rtol=1e-12, atol=1e-14)


def test_wb_source_non_expansive():
    rng = np.random.default_rng(9)
    n = 50
    p = si.make_problem(1, (n,), bc=[("periodic", "periodic")], dt=1.0)
    s = Scheme(p)
    for _ in range(20):
        p.sigma_f = rng.uniform(0.0, 1.0, n) ** 4 * 1e3
        Fs = rng.standard_normal(n)
        out = s._wb_implicit_solve(Fs, 0)
        assert np.linalg.norm(out) <= np.linalg.norm(Fs) * (1 + 1e-14)


# --------------------------------------------------------------------- realizability

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_hll_realizability(dim):
    rng = np.random.default_rng(20 + dim)
    n = {1: (30,), 2: (9, 8), 3: (5, 4, 4)}[dim]
    p = si.make_problem(dim, n, bc=[("periodic", "periodic")] * dim, ap_correction=False,
                        well_balanced=False, dt_factor=1.0)
    for _ in range(5):
        random_state(p, rng, fmax=1.0, Elo=1e-3, Ehi=1.0)
        p.sigma_a = rng.uniform(0, 10, p.shape)
        p.sigma_f = p.sigma_a.copy()  # one opacity, as in the model (Sect. 2.1)
        p.B = rng.uniform(0, 1e-3, p.shape)
        out = Scheme(p).explicit_step()
        nF = np.sqrt(sum(out[1 + b] ** 2 for b in range(dim)))
        assert np.all(out[0] > 0)
        assert np.all(nF <= p.c * out[0] * (1 + 1e-12))


# --------------------------------------------------------------------- asymptotic preserving

def _diffusion_step(E0, sig, dx, dt, c):
    """Backward-Euler discrete diffusion Eq. (discreteDiffusionEqua) with
    sigma_a = 0 and periodic ends (cyclic system solved densely)."""
    n = E0.size
    sf = 0.5 * (sig + np.roll(sig, -1))  # sigma_{i+1/2}
    k = c * dt / (3 * dx * dx)
    A = np.eye(n)
    for i in range(n):
        ip, im = (i + 1) % n, (i - 1) % n
        A[i, i] += k / sf[i] + k / sf[im]
        A[i, ip] -= k / sf[i]
        A[i, im] -= k / sf[im]
    return np.linalg.solve(A, E0)


def test_asymptotic_preserving_one_step():
    n = 64
    p = si.make_problem(1, (n,), bc=[("periodic", "periodic")])
    x = p.centers(0)
    p.E = 1.0 + np.exp(-((x - 0.5) ** 2) / (2 * 0.08 ** 2))
    p.sigma_a = np.zeros(n)
    sdx = 1e4
    p.sigma_f = sdx / p.dx[0] * (1.0 + 0.5 * np.sin(2 * np.pi * x))
    p.B = np.zeros(n)
    # a diffusion time step that moves the profile visibly
    D = p.c / (3 * p.sigma_f.min())
    p.dt = 0.2 * (0.08 ** 2) / D
    ref = _diffusion_step(p.E.copy(), p.sigma_f, p.dx[0], p.dt, p.c)
    change = np.abs(ref - p.E).max()
    res = newton_solve(Scheme(p), rtol=1e-12)
    assert res.converged
    err_ap = np.abs(res.u[:n] - ref).max()
    p.ap_correction = False
    res_hll = newton_solve(Scheme(p), rtol=1e-12)
    err_hll = np.abs(res_hll.u[:n] - ref).max()
    assert err_ap <= 1e-3 * change
    assert err_hll >= 0.3 * change


# --------------------------------------------------------------------- linearisation and solvers

def _gas_case(rng, dim):
    n = {1: (7,), 2: (4, 5), 3: (3, 3, 3)}[dim]
    bc = [("dirichlet", "outflow"), ("periodic", "periodic"), ("reflect", "outflow")][:dim]
    p = si.make_problem(dim, n, bc=bc, gas=True, dt_factor=20)
    random_state(p, rng, fmax=0.8)
    p.sigma_a = rng.uniform(0.1, 30, p.shape)
    p.sigma_f = rng.uniform(0.1, 30, p.shape)
    face = p.shape[:-1] if dim > 1 else ()
    Eg = rng.uniform(0.5, 1.5, face)
    Fg = np.zeros((dim,) + face)
    Fg[0] = 0.5 * Eg
    mask = (rng.uniform(size=face) < 0.6).astype(np.uint8) if dim > 1 else np.array(1, np.uint8)
    p.boundary[(0, 0)] = (Eg, Fg, mask)
    p.S = rng.uniform(0, 1, p.shape)
    return p


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("implicit_eigs", [True, False])
def test_jv_matches_central_differences(dim, implicit_eigs):
    rng = np.random.default_rng(30 + dim)
    p = _gas_case(rng, dim)
    p.implicit_eigs = implicit_eigs
    s = Scheme(p)
    u = s.pack(s.Un) * (1 + 0.05 * rng.standard_normal(s.nu * s.N))
    v = rng.standard_normal(u.size)
    jv = s.jv(u, v)
    errs = []
    for h in (1e-4, 1e-5):
        fd = (s.residual(u + h * v) - s.residual(u - h * v)) / (2 * h)
        errs.append(np.abs(jv - fd).max() / np.abs(fd).max())
    assert errs[1] < 1e-7
    assert errs[1] < errs[0] * 0.05  # O(h^2)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_diag_blocks_are_jacobian_diagonal(dim):
    rng = np.random.default_rng(40 + dim)
    p = _gas_case(rng, dim)
    s = Scheme(p)
    u = s.pack(s.Un)
    J = dense_jacobian(s, u)
    B = s.diag_blocks(u)
    N, nu = s.N, s.nu
    for i in range(N):
        idx = [k * N + i for k in range(nu)]
        assert np.allclose(B[i], J[np.ix_(idx, idx)], rtol=0, atol=1e-12 * np.abs(J).max())


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_gmres_matches_dense_lu(dim):
    rng = np.random.default_rng(50 + dim)
    p = _gas_case(rng, dim)
    s = Scheme(p)
    u = s.pack(s.Un)
    b = rng.standard_normal(u.size)
    x_lu = dense_solve(s, u, b)
    Minv = block_jacobi(s.diag_blocks(u), s.N, s.nu)
    res = gmres(lambda v: s.jv(u, v), b, Minv, rtol=1e-13, restart=30, maxiter=5000)
    assert res.converged
    assert np.linalg.norm(res.x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)


@pytest.mark.parametrize("dim", [1, 2])
def test_bicgstab_matches_dense_lu(dim):
    from oracle.solvers import bicgstab
    rng = np.random.default_rng(60 + dim)
    p = _gas_case(rng, dim)
    s = Scheme(p)
    u = s.pack(s.Un)
    b = rng.standard_normal(u.size)
    x_lu = dense_solve(s, u, b)
    Minv = block_jacobi(s.diag_blocks(u), s.N, s.nu)
    res = bicgstab(lambda v: s.jv(u, v), b, Minv, rtol=1e-13, maxiter=5000)
    assert res.converged
    assert np.linalg.norm(res.x - x_lu) <= 1e-9 * np.linalg.norm(x_lu)


def test_bicgstab_exact_preconditioner_takes_one_step():
    # M^-1 = A^-1 makes A M^-1 the identity: the first half step leaves s = 0
    from oracle.solvers import bicgstab
    rng = np.random.default_rng(61)
    A = rng.standard_normal((12, 12)) + 12.0 * np.eye(12)
    Ainv = np.linalg.inv(A)
    b = rng.standard_normal(12)
    res = bicgstab(lambda v: A @ v, b, lambda r: Ainv @ r, rtol=1e-12)
    assert res.converged and res.iters == 1
    assert np.linalg.norm(res.x - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(res.x)


def test_bicgstab_nonsymmetric_dense():
    from oracle.solvers import bicgstab
    rng = np.random.default_rng(62)
    n = 40
    A = rng.standard_normal((n, n)) + 3.0 * np.sqrt(n) * np.eye(n)
    b = rng.standard_normal(n)
    res = bicgstab(lambda v: A @ v, b, lambda r: r, rtol=1e-12, maxiter=500)
    assert res.converged
    assert np.linalg.norm(res.x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(res.x)


def test_newton_quadratic_tail():
    rng = np.random.default_rng(4)
    p = si.make_problem(1, (48,), bc=[("periodic", "periodic")], dt_factor=2.0, gas=True)
    random_state(p, rng, fmax=0.5)
    p.sigma_a = rng.uniform(0.5, 20, p.shape)
    p.sigma_f = p.sigma_a.copy()
    res = newton_solve(Scheme(p), rtol=1e-14, gmres_rtol=1e-13)
    assert res.converged
    h = np.array(res.history) / res.history[0]
    # once below 1e-2 the error squares: r_{k+1} <= C r_k^2 with modest C
    tail = [(h[k], h[k + 1]) for k in range(len(h) - 1) if 1e-12 < h[k] < 1e-2]
    assert len(tail) >= 2, h
    for a, b in tail:
        assert b <= 1e2 * a * a + 1e-14


# --------------------------------------------------------------------- gas advection (frozen flow)

def test_advection_divergence_free_keeps_uniform_and_conserves():
    n = 8
    p = si.make_problem(3, (n, n, n), bc=[("periodic", "periodic")] * 3, gas=True, dt_factor=1.0)
    p.T = np.full(p.shape, 2.0)
    p.rho_cv = np.full(p.shape, 1.5)
    u = si.divergence_free_velocity_3d(n, seed=4, umax=0.3)
    # discrete divergence of the face field vanishes to round-off
    div = (np.diff(u[0], axis=2) + np.diff(u[1], axis=1) + np.diff(u[2], axis=0))
    assert np.abs(div).max() < 1e-15
    T = Scheme(p).advect_internal_energy(u)
    assert np.allclose(T, 2.0, rtol=1e-14)
    rng = np.random.default_rng(6)
    p.T = rng.uniform(0.5, 1.5, p.shape)
    p.rho_cv = rng.uniform(0.5, 2.0, p.shape)
    e0 = (p.rho_cv * p.T).sum()
    T = Scheme(p).advect_internal_energy(u)
    assert (p.rho_cv * T).sum() == pytest.approx(e0, rel=1e-14)


def test_advection_upwind_shift():
    n = 16
    p = si.make_problem(1, (n,), bc=[("periodic", "periodic")], gas=True)
    p.T = np.random.default_rng(7).uniform(0.5, 1.5, n)
    p.rho_cv = np.ones(n)
    p.dt = 0.25
    u = np.full(n + 1, p.dx[0] / p.dt)  # CFL 1 to the right: e moves one cell
    T = Scheme(p).advect_internal_energy([u])
    assert np.allclose(T, np.roll(p.T, 1), rtol=1e-14)


# ------------------------------------------------------------ velocity-dependent sources
def _vel_case(d, gas, rng, F_scale=0.0):
    n = {1: (8,), 2: (6, 5), 3: (4, 3, 3)}[d]
    p = si.make_problem(d, n, bc=[("periodic", "periodic")] * d, gas=gas, dt_factor=3.0)
    p.E = rng.uniform(0.5, 2.0, p.shape)
    p.F = F_scale * p.c * p.E * rng.uniform(-1, 1, (d,) + p.shape) / np.sqrt(d)
    p.sigma_a = 10.0 ** rng.uniform(-1, 1, p.shape)
    p.sigma_f = p.sigma_a.copy()
    if gas:
        p.T = p.E ** 0.25  # a_r = 1: a_r T^4 = E
        p.rho_cv = rng.uniform(0.5, 2.0, p.shape)
    else:
        p.B = p.E.copy()
    return p


def _faces_from_cells(p, ucell):
    """Face velocities whose two-face mean is the given uniform cell velocity."""
    out = []
    for a in range(p.dim):
        shp = list(p.shape)
        shp[p.dim - 1 - a] += 1
        out.append(np.full(shp, ucell[a]))
    return out


@pytest.mark.parametrize("d", [1, 2, 3])
def test_velocity_sources_vanish_at_rest(d):
    rng = np.random.default_rng(70 + d)
    p = _vel_case(d, True, rng, F_scale=0.5)
    s = Scheme(p)
    out = s.velocity_sources(_faces_from_cells(p, [0.0] * d))
    for k in range(s.nu):
        assert np.array_equal(out[k], s.Un[k])


@pytest.mark.parametrize("gas", [False, True])
def test_velocity_sources_isotropic_equilibrium(gas):
    # F = 0, P = E/3 I, a_r T^4 = E: S_E = (4/3)(sigma/c) E |u|^2, S_F = (4/3) sigma E u
    rng = np.random.default_rng(80 + gas)
    p = _vel_case(2, gas, rng)
    s = Scheme(p)
    uc = np.array([3e-3, -2e-3])
    out = s.velocity_sources(_faces_from_cells(p, uc))
    E, sig, c, dt = p.E, p.sigma_f, p.c, p.dt
    SE = 4.0 / 3.0 * sig / c * E * (uc @ uc)
    np.testing.assert_allclose(out[0], E + dt * SE, rtol=1e-14, atol=0)
    for a in range(2):
        np.testing.assert_allclose(out[1 + a], c * dt * 4.0 / 3.0 * sig * E * uc[a], rtol=1e-13, atol=0)
    if gas:  # the matter energy gives what the radiation gains
        np.testing.assert_allclose(p.rho_cv * out[3] + out[0], p.rho_cv * p.T + E, rtol=1e-14)


def test_velocity_sources_free_streaming():
    # f = 1 along x (P = E x x, F = c E x), u = u_x x: S_E = sigma u_x E + 2 (sigma/c) E u_x^2,
    # S_F,x = sigma E u_x + sigma B u_x + sigma u_x^2 E / c, S_F,y = 0
    rng = np.random.default_rng(90)
    p = _vel_case(2, False, rng)
    p.F = np.stack([p.c * p.E, np.zeros(p.shape)])
    s = Scheme(p)
    ux = 2e-3
    out = s.velocity_sources(_faces_from_cells(p, [ux, 0.0]))
    E, B, sig, c, dt = p.E, p.B, p.sigma_f, p.c, p.dt
    np.testing.assert_allclose(out[0], E + dt * (sig * ux * E + 2.0 * sig / c * E * ux ** 2), rtol=1e-13)
    np.testing.assert_allclose(out[1], c * E + c * dt * (sig * E * ux + sig * B * ux + sig * ux ** 2 * E / c),
                               rtol=1e-13)
    np.testing.assert_allclose(out[2], 0.0, atol=1e-300)


def test_velocity_sources_rotate_with_the_state():
    # rotating u and F by 90 degrees in the plane rotates the flux source and keeps S_E
    rng = np.random.default_rng(91)
    p = _vel_case(2, False, rng, F_scale=0.6)
    p.E = np.full(p.shape, 1.3)
    p.sigma_f = np.full(p.shape, 0.7)
    p.sigma_a = p.sigma_f.copy()
    p.B = np.full(p.shape, 0.9)
    F0 = np.array([0.31, -0.17])
    p.F = np.stack([np.full(p.shape, F0[0]), np.full(p.shape, F0[1])])
    uc = np.array([1.5e-3, 0.6e-3])
    out1 = Scheme(p).velocity_sources(_faces_from_cells(p, uc))
    p.F = np.stack([np.full(p.shape, -F0[1]), np.full(p.shape, F0[0])])  # R F, R = rotation by +90
    out2 = Scheme(p).velocity_sources(_faces_from_cells(p, [-uc[1], uc[0]]))
    np.testing.assert_allclose(out2[0], out1[0], rtol=1e-14)
    np.testing.assert_allclose(out2[1], -out1[2], rtol=1e-13)
    np.testing.assert_allclose(out2[2], out1[1], rtol=1e-13)


def test_beam_widths_sect53():
    # Sect. 5.3: the 128^2 beam at 45 degrees enters over 8 cells; at mid-height it
    # is about 24 cells wide with computed eigenvalues and about 30 with fixed +-c.
    # Width here is the FWHM of the horizontal cut (a reading: the paper gives no
    # definition); the oracle gives 22 and 27. The ordering and the ratio are the
    # method's; each width is held to 15 % of the paper's value.
    import json, os
    from tests.m1_cases import beam_45_oracle, midheight_fwhm
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    w = gold["beam_width_cells"]
    p = si.beam_45_2d(128)
    assert int(((p.boundary[(0, 0)][0]) > 1.0).sum()) == w["inflow"]
    wc = midheight_fwhm(beam_45_oracle(128, False, 4.0).E)
    wf = midheight_fwhm(beam_45_oracle(128, True, 4.0).E)
    assert wc < wf
    assert abs(wc - w["computed_eigs_mid"]) <= 0.15 * w["computed_eigs_mid"], wc
    assert abs(wf - w["fixed_eigs_mid"]) <= 0.15 * w["fixed_eigs_mid"], wf
    assert 1.1 <= wf / wc <= 1.4


@pytest.mark.parametrize("gas", [False, True])
def test_1d_jacobian_is_block_tridiagonal(gas):
    # the scheme couples a cell to its two neighbours only (HLL faces, WB face
    # averages, ghosts through the edge cells): on a non-periodic 1D grid the
    # line preconditioner's matrix is J itself, and GMRES with it takes one step
    from oracle import block_tridiagonal_part
    from tests.m1_cases import line_case_1d
    p = line_case_1d(False, gas)
    s = Scheme(p)
    u = s.pack(s.Un)
    J = dense_jacobian(s, u)
    T = block_tridiagonal_part(J, s.nu, s.N)
    assert np.array_equal(T, J)
    b = np.random.default_rng(63).standard_normal(u.size)
    res = gmres(lambda v: s.jv(u, v), b, lambda r: np.linalg.solve(T, r), rtol=1e-12, restart=30, maxiter=10)
    assert res.converged and res.iters == 1


def test_periodic_1d_jacobian_differs_by_the_wrap_corners():
    from oracle import block_tridiagonal_part
    from tests.m1_cases import line_case_1d
    p = line_case_1d(True, False)
    s = Scheme(p)
    u = s.pack(s.Un)
    J = dense_jacobian(s, u)
    D = J - block_tridiagonal_part(J, s.nu, s.N)
    i = np.arange(s.nu * s.N) % s.N
    corner = ((i[:, None] == 0) & (i[None, :] == s.N - 1)) | ((i[:, None] == s.N - 1) & (i[None, :] == 0))
    assert np.all(D[~corner] == 0.0)
    assert np.abs(D[corner]).max() > 0.0
