"""Shared small workloads for the GPU parity tests (seeded, span several
256-thread tiles with ragged tails)."""
import numpy as np

import seeded_inputs as si


def perturbed_state(p, seed, scale=0.05):
    """U^n with a multiplicative perturbation (a generic Newton iterate)."""
    rng = np.random.default_rng(seed)
    u = p.state_vector()
    return u * (1.0 + scale * rng.standard_normal(u.size))


def gas_3d(n=(13, 11, 9), seed=3):
    rng = np.random.default_rng(seed)
    p = si.make_problem(3, n, bc=[("dirichlet", "outflow"), ("periodic", "periodic"), ("reflect", "outflow")],
                        gas=True, dt_factor=20)
    p.E = rng.uniform(0.5, 2.0, p.shape)
    dirs = rng.standard_normal((3,) + p.shape)
    dirs /= np.linalg.norm(dirs, axis=0, keepdims=True)
    p.F = p.c * p.E * rng.uniform(0, 0.8, p.shape) * dirs
    p.T = rng.uniform(0.7, 1.3, p.shape)
    p.rho_cv = rng.uniform(0.5, 2.0, p.shape)
    p.sigma_a = 10.0 ** rng.uniform(-1, 2, p.shape)
    p.sigma_f = 10.0 ** rng.uniform(-1, 2, p.shape)
    face = p.shape[:-1]
    Eg = rng.uniform(0.5, 1.5, face)
    Fg = np.zeros((3,) + face)
    Fg[0] = 0.6 * Eg
    p.boundary[(0, 0)] = (Eg, Fg, (rng.uniform(size=face) < 0.5).astype(np.uint8))
    p.S = rng.uniform(0, 1, p.shape)
    return p


def smooth_2d(n=(40, 33), seed=11):
    """Periodic 2D state away from vacuum with wave speeds at the new time
    level (the Newton system of Sect. 3.3.1 with lambda(U^{n+1}))."""
    p = si.make_problem(2, n, bc=[("periodic", "periodic")] * 2, dt_factor=10.0)
    rng = np.random.default_rng(seed)
    X, Y = p.mesh()
    p.E = 0.1 + np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2) / (2 * 0.1 ** 2))
    p.F = 0.2 * p.E * rng.uniform(-1, 1, (2,) + p.shape)
    p.sigma_a = si.opacity_span(p.shape, 4.0, seed, 1e-1, 1e2, p.dx[0])
    p.sigma_f = p.sigma_a.copy()
    p.B = np.full(p.shape, 0.1)
    p.implicit_eigs = True
    return p


def gas_2d(n=(37, 21), seed=5):
    """2D gas-coupled case with frozen wave speeds, Dirichlet/outflow in x and
    reflecting walls in y (exercises the tiled 2D J v with gas coupling)."""
    rng = np.random.default_rng(seed)
    p = si.make_problem(2, n, bc=[("dirichlet", "outflow"), ("reflect", "reflect")], gas=True, dt_factor=20)
    p.E = rng.uniform(0.5, 2.0, p.shape)
    dirs = rng.standard_normal((2,) + p.shape)
    dirs /= np.linalg.norm(dirs, axis=0, keepdims=True)
    p.F = p.c * p.E * rng.uniform(0, 0.8, p.shape) * dirs
    p.T = rng.uniform(0.7, 1.3, p.shape)
    p.rho_cv = rng.uniform(0.5, 2.0, p.shape)
    p.sigma_a = 10.0 ** rng.uniform(-1, 2, p.shape)
    p.sigma_f = p.sigma_a.copy()
    Eg = rng.uniform(0.5, 1.5, (n[1],))
    Fg = np.zeros((2, n[1]))
    Fg[0] = 0.6 * Eg
    p.boundary[(0, 0)] = (Eg, Fg, (rng.uniform(size=n[1]) < 0.5).astype(np.uint8))
    p.implicit_eigs = False
    return p


def cases():
    """name -> problem factory"""
    return {
        "slab1d": lambda: si.two_slab_1d(300, dt_factor=50.0),
        "beam2d": lambda: si.beam_lognormal_2d(70, 45, dt_factor=10.0),
        "smooth2d_implicit_eigs": smooth_2d,
        "gas3d": gas_3d,
        "gas2d_frozen": gas_2d,
    }


def midheight_fwhm(E2d: np.ndarray) -> int:
    """Width in cells of a beam in a horizontal cut at mid-height (Sect. 5.3):
    the cut is the mean of the two rows next to y = 0; the width counts the cells
    whose excess over the background E = 1 is above half the cut's peak excess."""
    ny = E2d.shape[0]
    ex = 0.5 * (E2d[ny // 2 - 1] + E2d[ny // 2]) - 1.0
    return int((ex > 0.5 * ex.max()).sum())


def beam_45_oracle(n: int, fixed_eigs: bool, t_end: float):
    """March the oracle's semi-implicit step on the Sect. 5.3 beam to t_end;
    returns the problem holding the final state."""
    from oracle import Scheme
    p = si.beam_45_2d(n, fixed_eigs)
    for _ in range(int(round(t_end / p.dt))):
        out = Scheme(p).explicit_step()
        p.E = out[0]
        p.F = np.stack(out[1:3])
    return p


def line_case_1d(periodic: bool, gas: bool, n: int = 12, seed: int = 61):
    """A 1D state away from equilibrium for the line preconditioner (Dirichlet / outflow
    or periodic, radiation only or with gas), dt = 50 dt_CFL."""
    rng = np.random.default_rng(seed)
    bc = [("periodic", "periodic")] if periodic else [("dirichlet", "outflow")]
    p = si.make_problem(1, (n,), bc=bc, gas=gas, dt_factor=50)
    p.E = rng.uniform(0.5, 2.0, p.shape)
    p.F = 0.6 * rng.uniform(-1, 1, (1,) + p.shape) * p.E
    p.sigma_a = 10.0 ** rng.uniform(-1, 2, p.shape)
    p.sigma_f = 10.0 ** rng.uniform(-1, 2, p.shape)
    if gas:
        p.T = rng.uniform(0.7, 1.3, p.shape)
        p.rho_cv = rng.uniform(0.5, 2.0, p.shape)
    if not periodic:
        p.boundary[(0, 0)] = (np.array(1.5), np.array([0.5]), np.array(1))
    return p
