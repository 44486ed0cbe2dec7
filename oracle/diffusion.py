"""Reference solution of the diffusive limit, Eq. (diffusionEqua): plain FP64 oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

At order 0 of the diffusive limit (Sect. 2.3) the radiation is in equilibrium with
the gas, E = a_r T^4, and the total energy obeys

    d/dt (a_r T^4 + rho c_v T) - d/dx ( c / (3 sigma) d/dx (a_r T^4) ) = 0.

Sect. 5.1 measures the Marshak wave of the M1 scheme against "a standard
discretization" of this equation. The one taken here (a reading; the paper gives
no details): 1D cell-centred finite volumes, backward Euler in time, the face
diffusion coefficient c / (3 sigma_face) with sigma_face the mean of the two
cells, a Dirichlet value E_b on the left face reached over half a cell, no flux
through the right face. Each step is solved for T by Newton's method with the
tridiagonal Jacobian.

Pinned in tests/test_oracle_marshak.py: with rho c_v = 0 the equation is linear
diffusion of E, whose half-space solution E_0 + (E_b - E_0) erfc(x / (2 sqrt(D t)))
it follows to discretisation error; the total energy changes by exactly the
boundary inflow; a long step reaches the uniform steady state T = T_b.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import numpy as np
from scipy.linalg import solve_banded


@dataclass
class DiffusionResult:
    T: np.ndarray          # gas (= radiation) temperature per cell
    E: np.ndarray          # a_r T^4
    inflow: float          # sum over steps of dt * (energy flux through the left face)
    newton_max: int        # most Newton iterations any step needed


def diffusion_reference(T0: np.ndarray, T_b: float, sigma: np.ndarray, rho_cv: float, dx: float,
                        dts: Sequence[float], c: float = 1.0, a_r: float = 1.0,
                        tol: float = 1e-13, max_iter: int = 100) -> DiffusionResult:
    """March Eq. (diffusionEqua) over the steps dts from T0 (one value per cell)."""
    T = np.array(T0, dtype=np.float64)
    n = T.size
    sigma = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (n,))
    E_b = a_r * T_b ** 4
    # diffusion coefficients: left boundary face (half cell), interior faces
    D_left = c / (3.0 * sigma[0])
    D_face = c / (3.0 * 0.5 * (sigma[:-1] + sigma[1:]))
    inflow, newton_max = 0.0, 0
    for dt in dts:
        e_old = a_r * T ** 4 + rho_cv * T
        for it in range(1, max_iter + 1):
            E = a_r * T ** 4
            dE = 4.0 * a_r * T ** 3
            # flux Phi through each face: Phi_left, interior Phi_{i+1/2}, 0 on the right
            phi_left = -D_left * (E[0] - E_b) / (0.5 * dx)
            phi = -D_face * (E[1:] - E[:-1]) / dx
            phi_lo = np.concatenate(([phi_left], phi))   # face i - 1/2 of cell i
            phi_hi = np.concatenate((phi, [0.0]))        # face i + 1/2 of cell i
            R = a_r * T ** 4 + rho_cv * T - e_old + dt * (phi_hi - phi_lo) / dx
            # tridiagonal Jacobian dR/dT
            g_lo = np.concatenate(([D_left / (0.5 * dx)], D_face / dx))  # d(-phi_lo)/dE_i
            g_hi = np.concatenate((D_face / dx, [0.0]))                   # d(phi_hi)/dE_i
            diag = dE + rho_cv + dt / dx * (g_lo + g_hi) * dE
            ab = np.zeros((3, n))
            ab[0, 1:] = -dt / dx * (D_face / dx) * dE[1:]   # dR_i / dT_{i+1}
            ab[1] = diag
            ab[2, :-1] = -dt / dx * (D_face / dx) * dE[:-1]  # dR_i / dT_{i-1}
            dT = solve_banded((1, 1), ab, -R)
            T = T + dT
            if np.abs(dT).max() <= tol * np.abs(T).max():
                break
        newton_max = max(newton_max, it)
        E = a_r * T ** 4
        inflow += dt * (-D_left * (E[0] - E_b) / (0.5 * dx))
    return DiffusionResult(T, a_r * T ** 4, inflow, newton_max)
