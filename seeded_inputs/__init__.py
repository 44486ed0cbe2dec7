"""Seeded synthetic inputs for the grey M1 radiation step.

This module holds data only: grid descriptions, seeded random fields and the
initial/boundary states of the workloads. It contains none of the method's
arithmetic (no closure, flux, source or solver), so both the CPU oracle and the
CUDA path can consume the same inputs without sharing discretisation code.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), a published
counter-based generator, turned into normals by the Box-Muller transform.
The opacity and density fields of the workloads are lognormal: white noise
smoothed by a periodic Gaussian kernel of standard deviation ``ell`` cells.

Units follow the code convention c = 1, a_r = 1 unless a problem says
otherwise. Arrays are numpy float64 in C order with x fastest: shape (nx,) in
1D, (ny, nx) in 2D and (nz, ny, nx) in 3D. Flux components are stacked as
F[b] for axis b (0 = x, 1 = y, 2 = z).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

BC_KINDS = ("outflow", "periodic", "reflect", "dirichlet")

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Counter-based SplitMix64 outputs 1..count for ``seed`` (uint64 array)."""
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1) from the top 53 bits."""
    z = splitmix64(seed, count) >> np.uint64(11)
    return (z.astype(np.float64) + 0.5) * 2.0 ** -53


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller from one SplitMix64 stream."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:count]


def smooth_periodic(noise: np.ndarray, ell: float) -> np.ndarray:
    """Convolve ``noise`` with a periodic Gaussian kernel of std ``ell`` cells,
    then normalise to zero mean and unit standard deviation."""
    spec = np.fft.fftn(noise)
    mult = np.ones(noise.shape)
    for ax, n in enumerate(noise.shape):
        k = np.fft.fftfreq(n)  # cycles per cell
        shape = [1] * noise.ndim
        shape[ax] = n
        mult = mult * np.exp(-2.0 * np.pi ** 2 * ell ** 2 * k ** 2).reshape(shape)
    g = np.real(np.fft.ifftn(spec * mult))
    g = g - g.mean()
    s = g.std()
    return g / s if s > 0 else g


def lognormal_unit_field(shape, ell: float, seed: int) -> np.ndarray:
    """Smoothed Gaussian random field (zero mean, unit std) on ``shape``."""
    n = int(np.prod(shape))
    return smooth_periodic(normal(seed, n).reshape(shape), ell)


def opacity_span(shape, ell: float, seed: int, lo: float, hi: float, dx: float) -> np.ndarray:
    """Lognormal opacity whose sigma*dx spans exactly [lo, hi] (log-linear min-max rescale)."""
    g = lognormal_unit_field(shape, ell, seed)
    t = (g - g.min()) / max(g.max() - g.min(), 1e-300)
    return 10.0 ** (np.log10(lo) + t * (np.log10(hi) - np.log10(lo))) / dx


@dataclass
class Problem:
    """One grey M1 problem: grid, flags, fields and time step.

    ``n`` is (nx, ny, nz) with unused axes 1. ``bc[a]`` is the (low, high)
    boundary kind along axis a. ``boundary[(a, side)]`` holds Dirichlet ghost
    data for that face: (E_g, F_g, mask), each over the face's cells
    (the grid shape with axis a removed; F_g has a leading component axis).
    mask == 1 selects the given ghost, mask == 0 a zero-gradient copy.
    """

    dim: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    bc: List[Tuple[str, str]]
    E: np.ndarray
    F: np.ndarray
    sigma_a: np.ndarray
    sigma_f: np.ndarray
    dt: float
    c: float = 1.0
    a_r: float = 1.0
    gas: bool = False
    well_balanced: bool = True
    ap_correction: bool = True
    fixed_eigs: bool = False
    lambda_floor: float = 0.0
    wb_boundary: bool = True
    implicit_eigs: bool = True
    T: Optional[np.ndarray] = None
    rho_cv: Optional[np.ndarray] = None
    B: Optional[np.ndarray] = None
    S: Optional[np.ndarray] = None
    boundary: Dict[Tuple[int, int], tuple] = field(default_factory=dict)
    name: str = ""

    @property
    def shape(self) -> tuple:
        return tuple(self.n[a] for a in reversed(range(self.dim)))

    @property
    def ncell(self) -> int:
        return int(np.prod(self.shape))

    @property
    def dx(self) -> Tuple[float, ...]:
        return tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(self.dim))

    @property
    def n_u(self) -> int:
        return 1 + self.dim + (1 if self.gas else 0)

    @property
    def dt_cfl(self) -> float:
        return cfl_dt(self)

    def centers(self, a: int) -> np.ndarray:
        """Cell-centre coordinates along axis a (1D array)."""
        return self.lo[a] + (np.arange(self.n[a]) + 0.5) * self.dx[a]

    def mesh(self) -> List[np.ndarray]:
        """Cell-centre coordinate arrays broadcast to the grid shape, per axis."""
        axes = [self.centers(a) for a in reversed(range(self.dim))]
        grids = np.meshgrid(*axes, indexing="ij")
        return list(reversed(grids))

    def state_vector(self) -> np.ndarray:
        """Flat unknown vector [E, F_0.., (T)], component-major, x fastest."""
        parts = [self.E.ravel()] + [self.F[b].ravel() for b in range(self.dim)]
        if self.gas:
            parts.append(self.T.ravel())
        return np.concatenate(parts)

    def copy(self) -> "Problem":
        import copy as _copy
        return _copy.deepcopy(self)


def cfl_dt(p: Problem) -> float:
    """Explicit CFL time step dx_min / (c d) (the workloads' dt unit)."""
    return min(p.dx) / (p.c * p.dim)


def _grid(dim, n, lo=None, hi=None):
    n3 = tuple(list(n) + [1] * (3 - len(n)))
    lo3 = tuple(list(lo or [0.0] * dim) + [0.0] * (3 - dim))
    hi3 = tuple(list(hi or [1.0] * dim) + [1.0] * (3 - dim))
    return n3, lo3, hi3


def make_problem(dim, n, *, lo=None, hi=None, bc=None, E=None, F=None, sigma_a=None,
                 sigma_f=None, dt=None, dt_factor=1.0, **kw) -> Problem:
    """Build a Problem with defaults: unit box, outflow, E=1e-6, F=0, sigma=0."""
    n3, lo3, hi3 = _grid(dim, n, lo, hi)
    shape = tuple(n3[a] for a in reversed(range(dim)))
    if bc is None:
        bc = [("outflow", "outflow")] * dim
    if E is None:
        E = np.full(shape, 1e-6)
    if F is None:
        F = np.zeros((dim,) + shape)
    if sigma_a is None:
        sigma_a = np.zeros(shape)
    if sigma_f is None:
        sigma_f = sigma_a.copy()
    p = Problem(dim=dim, n=n3, lo=lo3, hi=hi3, bc=list(bc), E=np.array(E, float),
                F=np.array(F, float), sigma_a=np.array(sigma_a, float),
                sigma_f=np.array(sigma_f, float), dt=0.0, **kw)
    p.dt = float(dt) if dt is not None else dt_factor * cfl_dt(p)
    if p.B is None and not p.gas:
        p.B = np.full(shape, 1e-6 if kw.get("a_r", 1.0) == 1.0 else 0.0)
    return p


# ---------------------------------------------------------------------------
# Workloads (grid sizes are arguments so that tests can use small versions)
# ---------------------------------------------------------------------------

def two_slab_1d(n: int = 512, dt_factor: float = 50.0) -> Problem:
    """1D radiation-only two-slab problem: sigma = 1 (x < 0.5) / 100, Gaussian E
    (amplitude 1, width 0.05, centre 0.25) on floor 1e-6, F = 0, outflow."""
    p = make_problem(1, (n,), dt_factor=dt_factor, name=f"two_slab_1d_{n}")
    x = p.centers(0)
    sig = np.where(x < 0.5, 1.0, 100.0)
    p.sigma_a = sig.copy()
    p.sigma_f = sig.copy()
    p.E = 1e-6 + np.exp(-((x - 0.25) ** 2) / (2 * 0.05 ** 2))
    p.B = np.full(p.shape, 1e-6)
    p.implicit_eigs = False  # the pulse front enters the 1e-6 floor (free streaming)
    return p


def beam_lognormal_2d(nx: int = 1024, ny: Optional[int] = None, seed: int = 2,
                      ell: float = 32.0, span=(1e-3, 1e3), dt_factor: float = 50.0) -> Problem:
    """2D radiation-only beam in a lognormal opacity field.

    Periodic in y, outflow in x. sigma*dx spans ``span`` (seeded lognormal,
    correlation length ``ell`` cells). A collimated beam enters through x = 0
    for y in [0.45, 0.55] with E = 1, F = (0.99 c, 0). Initial E = 1e-6, F = 0.
    Frozen gas: emission B = 1e-6 everywhere.
    """
    ny = nx if ny is None else ny
    p = make_problem(2, (nx, ny), bc=[("dirichlet", "outflow"), ("periodic", "periodic")],
                     dt_factor=dt_factor, name=f"beam_lognormal_2d_{nx}x{ny}_dt{dt_factor:g}")
    sig = opacity_span(p.shape, ell, seed, span[0], span[1], p.dx[0])
    p.sigma_a = sig
    p.sigma_f = sig.copy()
    y = p.centers(1)
    mask = ((y >= 0.45) & (y <= 0.55)).astype(np.uint8)
    Eg = np.where(mask == 1, 1.0, 1e-6)
    Fg = np.zeros((2, ny))
    Fg[0] = np.where(mask == 1, 0.99 * p.c * 1.0, 0.0)
    p.boundary[(0, 0)] = (Eg, Fg, mask)
    p.B = np.full(p.shape, 1e-6)
    # Wave speeds frozen at time n: with speeds at the new time level Newton
    # does not converge on this beam-into-vacuum workload (free streaming).
    p.implicit_eigs = False
    return p


def beam_45_2d(n: int = 128, fixed_eigs: bool = False) -> Problem:
    """The 2D beam verification problem of Sect. 5.3 in code units (c = a_r = 1).

    Domain [-1, 1]^2, n x n cells, sigma = 0. Background T = 300 K, F = 0, scaled
    to E = 1; the beam has T = 1000 K, so E = (1000/300)^4, with |F| = cE at 45
    degrees. It enters through x = -1 for y in [-0.875, -0.75] (8 cells at
    n = 128). The rest of the x = -1 side is a background ghost (E = 1, F = 0);
    the other sides are outflow. With sigma = 0 neither the asymptotic
    correction nor the well-balanced source act, so the WB boundary closure is
    off. dt is the explicit CFL step (the semi-implicit scheme).
    """
    p = make_problem(2, (n, n), lo=[-1.0, -1.0], hi=[1.0, 1.0],
                     bc=[("dirichlet", "outflow"), ("outflow", "outflow")],
                     E=np.ones((n, n)), dt_factor=1.0,
                     name=f"beam_45_2d_{n}_{'fixed' if fixed_eigs else 'computed'}")
    p.B = np.ones(p.shape)
    p.fixed_eigs = fixed_eigs
    p.wb_boundary = False
    p.implicit_eigs = False
    y = p.centers(1)
    inside = (y >= -0.875) & (y <= -0.75)
    Eb = (1000.0 / 300.0) ** 4
    Eg = np.where(inside, Eb, 1.0)
    Fg = np.zeros((2, n))
    Fg[0] = np.where(inside, p.c * Eb / np.sqrt(2.0), 0.0)
    Fg[1] = Fg[0].copy()
    p.boundary[(0, 0)] = (Eg, Fg, np.ones(n, np.uint8))
    return p


def marshak_1d(n: int = 400, ap_correction: bool = True, rho_cv: float = 1.0,
               sigma_dx: float = 25.0) -> Problem:
    """The Marshak wave of Sect. 5.1 in code units (c = a_r = 1, domain [0, 1]).

    n cells with sigma dx = ``sigma_dx`` (25 at n = 400, sigma = 1e4), gas coupled
    with constant rho c_v, initial equilibrium T = T_r = 0.3 (300 K scaled by
    1000 K), F = 0. The left side is a Dirichlet ghost at T_r = 1 (E = 1, F = 0),
    the right side outflow. The paper's cgs values (rho c_v = 1 J/K/cm^3,
    sigma = 1e4 /cm) would move the front far less than one cell by its t_f; with
    rho c_v = 1 in code units the front crosses about two thirds of the domain by
    t = 3000. Wave speeds frozen at time n. ``dt`` holds the first step of
    ``marshak_schedule``.
    """
    p = make_problem(1, (n,), bc=[("dirichlet", "outflow")], gas=True, dt=1.0,
                     name=f"marshak_1d_{n}_{'ap' if ap_correction else 'hll'}")
    T0 = 0.3
    p.E = np.full(p.shape, p.a_r * T0 ** 4)
    p.F = np.zeros((1, n))
    p.T = np.full(p.shape, T0)
    p.rho_cv = np.full(p.shape, float(rho_cv))
    p.sigma_a = np.full(p.shape, sigma_dx / p.dx[0])
    p.sigma_f = p.sigma_a.copy()
    p.boundary[(0, 0)] = (np.array(p.a_r * 1.0 ** 4), np.array([0.0]), np.array(1, np.uint8))
    p.ap_correction = ap_correction
    p.implicit_eigs = False
    p.dt = marshak_schedule()[0]
    return p


def marshak_schedule(t_end: float = 3000.0, dt0: float = 0.01, dt_max: float = 10.0,
                     growth: float = 1.2) -> List[float]:
    """Time steps of the Marshak run: from dt0, growing by ``growth`` per step up to
    dt_max, the last one cut to end at t_end (the source is switched on at t = 0)."""
    dts, t, d = [], 0.0, dt0
    while t < t_end * (1.0 - 1e-12):
        d = min(d, t_end - t)
        dts.append(d)
        t += d
        d = min(d * growth, dt_max)
    return dts


def diffusion_gaussian_1d(n: int, sigma: float = 1000.0, width: float = 0.05, floor: float = 1e-6,
                          ap_correction: bool = True) -> Problem:
    """1D Gaussian pulse in a thick, purely scattering medium (the diffusive limit of
    Sect. 2.3): [0, 1], outflow, sigma_a = 0, sigma_f = ``sigma`` everywhere,
    E = floor + exp(-(x - 1/2)^2 / (2 width^2)), F = 0, wave speeds frozen at time n.
    ``dt`` is left at 1; the caller sets it."""
    p = make_problem(1, (n,), bc=[("outflow", "outflow")], dt=1.0, ap_correction=ap_correction,
                     name=f"diffusion_gaussian_1d_{n}")
    x = p.centers(0)
    p.E = floor + np.exp(-((x - 0.5) ** 2) / (2 * width * width))
    p.F = np.zeros((1, n))
    p.sigma_a = np.zeros(p.shape)
    p.sigma_f = np.full(p.shape, float(sigma))
    p.B = np.zeros(p.shape)
    p.implicit_eigs = False
    return p


def opacity_jump_1d(n: int = 100, sigma_dx: float = 100.0, well_balanced: bool = True) -> Problem:
    """The opacity-jump run of Sect. 5.2 in code units (c = a_r = 1, domain [0, 1]).

    sigma_f dx = ``sigma_dx`` for x < 1/2 and 0 beyond (sigma = 1e4 at n = 100, as in the
    paper), sigma_a = 0 (the gas is in equilibrium with the radiation, so the exchange
    vanishes in the steady state), E = 1 (300 K scaled), F = 0. The left side is a
    Dirichlet ghost at 1000 K (E = (10/3)^4, F = 0), the right side outflow. Wave speeds
    frozen at time n; ``dt`` is left at dx / c."""
    p = make_problem(1, (n,), bc=[("dirichlet", "outflow")], well_balanced=well_balanced,
                     name=f"opacity_jump_1d_{n}_{'wb' if well_balanced else 'centred'}")
    x = p.centers(0)
    p.sigma_a = np.zeros(p.shape)
    p.sigma_f = np.where(x < 0.5, sigma_dx / p.dx[0], 0.0)
    p.E = np.ones(p.shape)
    p.F = np.zeros((1, n))
    p.B = np.zeros(p.shape)
    p.boundary[(0, 0)] = (np.array((1000.0 / 300.0) ** 4), np.array([0.0]), np.array(1, np.uint8))
    p.implicit_eigs = False
    p.dt = p.dx[0] / p.c
    return p


def opacity_jump_schedule(dt0: float = 0.01, growth: float = 1.8, dt_max: float = 4000.0,
                          steps: int = 24) -> List[float]:
    """Time steps of the opacity-jump run: from dx / c, growing by ``growth`` up to dt_max."""
    dts, d = [], dt0
    for _ in range(steps):
        dts.append(d)
        d = min(d * growth, dt_max)
    return dts


def gaussian_lognormal_2d(n: int, seed: int, span=(1e-2, 1e3), dt_factor: float = 50.0,
                          ell: Optional[float] = None, center=None) -> Problem:
    """2D radiation-only problem with a Gaussian E pulse in a lognormal opacity
    field, periodic in both axes (learned-preconditioner and batched workloads)."""
    p = make_problem(2, (n, n), bc=[("periodic", "periodic")] * 2, dt_factor=dt_factor,
                     name=f"gaussian_lognormal_2d_{n}_s{seed}")
    ell = n / 32.0 if ell is None else ell
    p.sigma_a = opacity_span(p.shape, ell, seed, span[0], span[1], p.dx[0])
    p.sigma_f = p.sigma_a.copy()
    if center is None:
        u = uniform01(seed + 77_000, 2)
        center = (0.25 + 0.5 * u[0], 0.25 + 0.5 * u[1])
    X, Y = p.mesh()
    p.E = 1e-6 + np.exp(-((X - center[0]) ** 2 + (Y - center[1]) ** 2) / (2 * 0.05 ** 2))
    p.B = np.full(p.shape, 1e-6)
    p.implicit_eigs = False  # the pulse front enters the 1e-6 floor (free streaming)
    return p


def gas_point_source_3d(n: int = 256, seed: int = 3, ell: float = 16.0,
                        dt_factor: float = 50.0) -> Problem:
    """3D radiation + gas energy: rho = exp(s g - s^2/2) (s = 1, std-``ell`` lognormal),
    sigma_a = sigma_f = kappa rho with kappa dx = 1, rho c_v with c_v = 1.5,
    T0 = 1, E0 = a_r T0^4, F = 0, point source S = 10 in the central 2^3 cells,
    outflow boundaries, wave speeds frozen at time n."""
    p = make_problem(3, (n, n, n), dt_factor=dt_factor, gas=True, name=f"gas_point_source_3d_{n}")
    g = lognormal_unit_field(p.shape, ell, seed)
    rho = np.exp(g - 0.5)
    kappa = 1.0 / p.dx[0]
    p.sigma_a = kappa * rho
    p.sigma_f = p.sigma_a.copy()
    p.rho_cv = 1.5 * rho
    p.T = np.ones(p.shape)
    p.E = p.a_r * p.T ** 4
    p.B = None
    S = np.zeros(p.shape)
    h = n // 2
    lo_, hi_ = max(h - 1, 0), min(h + 1, n)
    S[lo_:hi_, lo_:hi_, lo_:hi_] = 10.0
    p.S = S
    # wave speeds frozen at time n, as in every other workload here: the scheme stays
    # linearly implicit in them, and J v is linear in the cells' derivative quantities
    p.implicit_eigs = False
    return p


def divergence_free_velocity_3d(n: int, seed: int, umax: float = 1e-3):
    """Face-centred velocity (ux on x-faces, ...) from the discrete curl of a
    seeded low-k periodic vector potential; max |u| scaled to ``umax``.
    Returns (ux, uy, uz) with shapes (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx)."""
    shape = (n, n, n)
    A = [lognormal_unit_field(shape, n / 8.0, seed * 3 + k) for k in range(3)]

    def wrap(a, ax):  # append the first plane at the end along ax (periodic)
        return np.concatenate([a, np.take(a, [0], axis=ax)], axis=ax)

    # vector potential on cell edges approximated by cell values (periodic differences)
    Ax, Ay, Az = A
    # ux at x-faces (i-1/2): dAz/dy - dAy/dz using forward differences
    ux = (np.roll(Az, -1, axis=1) - Az) - (np.roll(Ay, -1, axis=0) - Ay)
    uy = (np.roll(Ax, -1, axis=0) - Ax) - (np.roll(Az, -1, axis=2) - Az)
    uz = (np.roll(Ay, -1, axis=2) - Ay) - (np.roll(Ax, -1, axis=1) - Ax)
    s = umax / max(np.abs(ux).max(), np.abs(uy).max(), np.abs(uz).max())
    return wrap(ux * s, 2), wrap(uy * s, 1), wrap(uz * s, 0)


def batch_problems(nprob: int = 256, seed0: int = 5000,
                   sizes=(64, 96, 128, 192, 256)) -> List[Problem]:
    """Independent 2D problems: size uniform from ``sizes``, own lognormal
    opacity (ell = n/32) and Gaussian E, dt log-uniform in [10, 100] dt_CFL."""
    out = []
    for k in range(nprob):
        u = uniform01(seed0 + k, 3)
        n = sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]
        dtf = 10.0 ** (1.0 + u[1])
        out.append(gaussian_lognormal_2d(n, seed0 + k, dt_factor=dtf))
    return out
