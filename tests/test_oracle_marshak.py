"""Pins of the diffusive-limit reference (oracle/diffusion.py, Eq. (diffusionEqua))
that the Marshak wave of Sect. 5.1 is measured against (CPU only).

* rho c_v = 0: linear diffusion of E = a_r T^4 from a Dirichlet wall, against the
  half-space closed form E_0 + (E_b - E_0) erfc(x / (2 sqrt(D t))), D = c / (3 sigma);
* the total energy sum (E + rho c_v T) dx changes by exactly the inflow through the
  left face (the right face is closed);
* one very long step reaches the uniform steady state T = T_b;
* the Marshak problem and its step schedule as the paper states them (400 cells,
  sigma dx = 25, 300 K / 1000 K);
* the oracle's M1 scheme on a coarse Marshak wave: the asymptotic-preserving alpha
  within 3 % of the diffusion reference, plain HLL off by more than 50 % (Sect. 5.1).
"""
import numpy as np
import pytest
from scipy.special import erfc

import seeded_inputs as si
from oracle.diffusion import diffusion_reference


def test_linear_diffusion_matches_erfc():
    n, sigma, t_end, dt = 200, 100.0, 4.0, 0.0025
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    T0, Tb = 0.3, 1.0
    r = diffusion_reference(np.full(n, T0), Tb, sigma, 0.0, dx, [dt] * int(round(t_end / dt)))
    D = 1.0 / (3.0 * sigma)
    E_exact = T0 ** 4 + (Tb ** 4 - T0 ** 4) * erfc(x / (2.0 * np.sqrt(D * t_end)))
    # backward Euler O(dt) dominates (1.5e-4 here); half a cell's shift at the wall
    # or a wrong D is off by more than 1e-2
    assert np.abs(r.E - E_exact).max() <= 3e-4


def test_total_energy_changes_by_inflow():
    n = 64
    rng = np.random.default_rng(7)
    dx = 1.0 / n
    T0 = rng.uniform(0.3, 0.6, n)
    sigma = 10.0 ** rng.uniform(1, 3, n)
    rho_cv = 0.7
    dts = [0.5, 1.0, 2.0, 4.0]
    r = diffusion_reference(T0, 1.0, sigma, rho_cv, dx, dts)
    e0 = np.sum(T0 ** 4 + rho_cv * T0) * dx
    e1 = np.sum(r.E + rho_cv * r.T) * dx
    assert r.inflow > 0
    assert abs((e1 - e0) - r.inflow) <= 1e-12 * e1


def test_long_step_reaches_uniform_state():
    n = 50
    # backward Euler damps the slowest mode by 1 / (1 + dt lambda) per step: two long steps
    r = diffusion_reference(np.full(n, 0.3), 1.0, 1e3, 1.0, 1.0 / n, [1e12, 1e12])
    assert np.abs(r.T - 1.0).max() <= 1e-12


def test_marshak_problem_as_stated():
    p = si.marshak_1d()
    assert p.n[0] == 400
    assert p.sigma_a[0] * p.dx[0] == pytest.approx(25.0)
    assert p.T[0] / 1.0 == pytest.approx(300.0 / 1000.0)
    assert np.allclose(p.E, p.a_r * p.T ** 4, rtol=1e-15, atol=0)  # radiation in equilibrium with the gas
    dts = si.marshak_schedule()
    assert sum(dts) == pytest.approx(3000.0, rel=1e-12)
    assert max(dts) == 10.0 and dts[0] == 0.01


def test_marshak_oracle_ap_against_hll_sect51():
    # Sect. 5.1 on a coarse grid with the paper's sigma dx = 25 (64 cells, t_end = 480 so that
    # the front crosses about half the domain): the asymptotic-preserving alpha follows the
    # diffusion limit (relative L2 error of T about 1 %; paper 1.1 % at 400 cells), plain HLL
    # does not (about 81 %; paper 84 %)
    from oracle import Scheme, newton_solve
    dts = si.marshak_schedule(t_end=480.0)
    p0 = si.marshak_1d(64)
    ref = diffusion_reference(p0.T, 1.0, p0.sigma_a, float(p0.rho_cv[0]), p0.dx[0], dts)
    err = {}
    for ap in (True, False):
        p = si.marshak_1d(64, ap_correction=ap)
        for dt in dts:
            p.dt = dt
            s = Scheme(p)
            r = newton_solve(s, rtol=1e-6, gmres_rtol=1e-4, line_search=False)
            assert r.converged
            N = s.N
            p.E, p.F, p.T = r.u[:N].copy(), r.u[N:2 * N].reshape(1, N).copy(), r.u[2 * N:].copy()
        err[ap] = np.linalg.norm(p.T - ref.T) / np.linalg.norm(ref.T)
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    assert err[True] <= 3.0 * gold["marshak_rel_l2_ap"]["value"], err   # paper 1.1 %
    assert err[False] >= 0.6 * gold["marshak_rel_l2_hll"]["value"], err  # paper 84 %
    assert err[False] >= 20.0 * err[True], err
