"""Pins of the oracle's closure, eigenvalues and AP coefficient (CPU only).

Each check compares the oracle with something the paper or the mathematics
fixes independently of the oracle's own formulas:
* closure limits chi(0) = 1/3, chi(1) = 1 and P -> E/3 I, E n(x)n (Sect. 2.2);
* trace D = 1 in 3D and the paper's (3chi-1)/2 n(x)n form of the tensor;
* the eigenvalue formula against the numerical eigenvalues of the flux
  Jacobian of the M1 system (a library eigen-solver on a finite-difference
  Jacobian of the closure), plus the limits +-c/sqrt(3) (Appendix C) and
  (c, c) at f = 1;
* alpha = 1/(1 + sqrt(3) sigma dx / 2) at f = 0, Eq. (asymptoticCorrectionP1).
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle.m1 import Closure, Scheme, eigenvalues


def closure_of(E, F, c=1.0):
    E = np.atleast_1d(np.asarray(E, float))
    F = [np.atleast_1d(np.asarray(f, float)) for f in F]
    return Closure(E, F, c)


def test_chi_limits():
    cl0 = closure_of(2.0, [0.0, 0.0, 0.0])
    assert cl0.chi[0] == pytest.approx(1.0 / 3.0, abs=1e-15)
    cl1 = closure_of(2.0, [2.0 * 0.6, 2.0 * 0.8, 0.0])  # |F| = cE
    assert cl1.chi[0] == pytest.approx(1.0, abs=1e-15)


def test_pressure_limits():
    E = 3.0
    cl = closure_of(E, [0.0, 0.0, 0.0])
    for a in range(3):
        for b in range(3):
            want = E / 3.0 if a == b else 0.0
            assert cl.pressure(a, b)[0] == pytest.approx(want, abs=1e-15)
    n = np.array([0.36, 0.48, 0.8])  # unit vector
    cl = closure_of(E, list(E * n))  # free streaming, f = 1
    for a in range(3):
        for b in range(3):
            assert cl.pressure(a, b)[0] == pytest.approx(E * n[a] * n[b], rel=1e-13, abs=1e-15)


def test_trace_and_paper_form():
    rng = np.random.default_rng(7)
    c = 2.0
    for _ in range(50):
        E = rng.uniform(0.1, 10.0)
        f = rng.uniform(0.0, 0.999)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        F = c * E * f * n
        cl = closure_of(E, list(F), c)
        D = np.array([[cl.D[a][b][0] for b in range(3)] for a in range(3)])
        assert np.trace(D) == pytest.approx(1.0, abs=1e-14)
        chi = (3 + 4 * f * f) / (5 + 2 * np.sqrt(4 - 3 * f * f))
        paper = (1 - chi) / 2 * np.eye(3) + (3 * chi - 1) / 2 * np.outer(n, n)
        assert np.abs(D - paper).max() < 1e-13


def test_clamp_keeps_direction():
    E = 1.0
    cl = closure_of(E, [3.0, 4.0])  # |F| = 5 cE
    assert cl.f2[0] == 1.0
    assert cl.fvec[0][0] == pytest.approx(0.6)
    assert cl.fvec[1][0] == pytest.approx(0.8)


def _flux_jacobian_eigs(E, F, a, c, h=1e-7):
    """Eigenvalues of d(flux_a)/dU for the M1 system U = (E, F), flux_a = (F_a, c^2 P_{a.})."""
    d = len(F)
    U = np.array([E] + list(F), float)

    def flux(u):
        cl = closure_of(u[0], list(u[1:]), c)
        return np.array([u[1 + a]] + [c * c * cl.pressure(a, b)[0] for b in range(d)])

    J = np.zeros((d + 1, d + 1))
    for k in range(d + 1):
        e = np.zeros(d + 1)
        e[k] = h * max(1.0, abs(U[k]))
        J[:, k] = (flux(U + e) - flux(U - e)) / (2 * e[k])
    return np.sort(np.linalg.eigvals(J).real)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_eigenvalues_match_flux_jacobian(d):
    rng = np.random.default_rng(11 + d)
    c = 1.5
    for _ in range(25):
        E = rng.uniform(0.5, 2.0)
        f = rng.uniform(0.0, 0.95)
        n = rng.standard_normal(d)
        n /= np.linalg.norm(n)
        F = list(c * E * f * n)
        for a in range(d):
            ev = _flux_jacobian_eigs(E, F, a, c)
            cl = closure_of(E, F, c)
            lmax, lmin = eigenvalues(cl, a, c)
            assert lmax[0] == pytest.approx(ev[-1], abs=2e-6 * c)
            assert lmin[0] == pytest.approx(ev[0], abs=2e-6 * c)


def test_eigenvalue_limits_and_bounds():
    c = 1.0
    cl = closure_of(1.0, [0.0, 0.0])
    lmax, lmin = eigenvalues(cl, 0, c)
    assert lmax[0] == pytest.approx(c / np.sqrt(3.0), abs=1e-15)
    assert lmin[0] == pytest.approx(-c / np.sqrt(3.0), abs=1e-15)
    cl = closure_of(1.0, [1.0, 0.0])  # f = 1 along the normal
    lmax, lmin = eigenvalues(cl, 0, c)
    assert lmax[0] == pytest.approx(c) and lmin[0] == pytest.approx(c)
    cl = closure_of(1.0, [0.0, 1.0])  # f = 1 tangential
    lmax, lmin = eigenvalues(cl, 0, c)
    assert lmax[0] == pytest.approx(0.0, abs=1e-15) and lmin[0] == pytest.approx(0.0, abs=1e-15)
    # brute force over the realizable disc: lmin <= lmax, |lambda| <= c
    g = np.linspace(-1, 1, 81)
    FX, FY = np.meshgrid(g, g)
    keep = FX ** 2 + FY ** 2 <= 1.0
    cl = closure_of(np.ones(keep.sum()), [FX[keep], FY[keep]], c)
    lmax, lmin = eigenvalues(cl, 0, c)
    assert np.all(lmin <= lmax + 1e-15)
    assert np.all(np.abs(lmax) <= c + 1e-14) and np.all(np.abs(lmin) <= c + 1e-14)


@pytest.mark.parametrize("sdx", [1e-3, 0.5, 25.0, 1e4])
def test_alpha_p1_limit(sdx):
    # f = 0 everywhere: alpha = 1 / (1 + sqrt(3) sigma dx / 2) on interior faces
    n = 16
    p = si.make_problem(1, (n,), bc=[("periodic", "periodic")], E=np.ones(n))
    p.sigma_f[:] = sdx / p.dx[0]
    s = Scheme(p)
    want = 1.0 / (1.0 + np.sqrt(3.0) * sdx / 2.0)
    assert np.allclose(s.alpha[0], want, rtol=1e-14)


def test_alpha_to_one_and_off():
    n = 8
    p = si.make_problem(1, (n,), bc=[("periodic", "periodic")], E=np.ones(n))
    p.sigma_f[:] = 1e-12 / p.dx[0]
    assert np.allclose(Scheme(p).alpha[0], 1.0, atol=1e-11)
    p.sigma_f[:] = 1e3 / p.dx[0]
    p.ap_correction = False
    assert np.all(Scheme(p).alpha[0] == 1.0)
