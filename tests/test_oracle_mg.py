"""Pins of the aggregation multigrid oracle (oracle/mg.py) against independent computations."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import mg
from oracle.m1 import Scheme
from oracle.solvers import dense_jacobian


def _beam(nx=12, ny=8):
    p = si.beam_lognormal_2d(nx, ny, dt_factor=10.0)
    s = Scheme(p)
    rng = np.random.default_rng(7)
    u = s.pack(s.Un)
    # a state off the initial one, so that every closure derivative is exercised
    u = u * (1.0 + 0.05 * rng.standard_normal(u.size))
    return p, s, u


def _periodic(p):
    return p.bc[0][0] == "periodic", p.bc[1][0] == "periodic"


def test_colouring_separates_stencils():
    # cells of one colour are >= 3 apart along each axis, also across a periodic wrap
    for n in range(3, 40):
        m = mg.colouring(n, True)
        for i in range(n):
            for j in range(n):
                if i != j and i % m == j % m:
                    d = min(abs(i - j), n - abs(i - j))
                    assert d >= 3, (n, m, i, j)


def test_assembled_stencil_reproduces_jv():
    p, s, u = _beam()
    px, py = _periodic(p)
    A = mg.assemble_blocks(lambda v: s.jv(u, v), s.nu, p.n[0], p.n[1], px, py)
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.standard_normal(s.nu * s.N)
        ref = s.jv(u, v)
        got = mg.apply_stencil(A, v, p.n[0], p.n[1], px, py)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_galerkin_is_ptap():
    p, s, u = _beam()
    px, py = _periodic(p)
    nx, ny = p.n[0], p.n[1]
    A = mg.assemble_blocks(lambda v: s.jv(u, v), s.nu, nx, ny, px, py)
    Ac, nxc, nyc = mg.galerkin(A, nx, ny, px, py)
    rng = np.random.default_rng(2)
    xc = rng.standard_normal(s.nu * nxc * nyc)
    ref = mg.restrict(mg.apply_stencil(A, mg.prolong(xc, s.nu, nx, ny), nx, ny, px, py), s.nu, nx, ny)
    got = mg.apply_stencil(Ac, xc, nxc, nyc, px, py)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_cycle_is_linear():
    p, s, u = _beam(16, 8)
    px, py = _periodic(p)
    H = mg.Hierarchy(lambda v: s.jv(u, v), s.nu, p.n[0], p.n[1], px, py, coarsest=4)
    rng = np.random.default_rng(3)
    r1, r2 = rng.standard_normal(s.nu * s.N), rng.standard_normal(s.nu * s.N)
    lhs = H.cycle(2.0 * r1 - 3.0 * r2)
    rhs = 2.0 * H.cycle(r1) - 3.0 * H.cycle(r2)
    assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(rhs)


def test_two_level_cycle_matches_dense_construction():
    # no smoothing: z = P (K damped block-Jacobi sweeps on A_c = P^T J P) P^T r, with A_c,
    # its block diagonal and P built densely from the dense Jacobian
    p, s, u = _beam(8, 8)
    px, py = _periodic(p)
    nx, ny, nu, N = p.n[0], p.n[1], s.nu, s.N
    H = mg.Hierarchy(lambda v: s.jv(u, v), nu, nx, ny, px, py, coarsest=4)
    assert len(H.ops) == 2
    J = dense_jacobian(s, u)
    agg, nxc, nyc = mg.aggregate(nx, ny)
    Nc = nxc * nyc
    P = np.zeros((nu * N, nu * Nc))
    for c in range(nu):
        P[c * N + np.arange(N), c * Nc + agg] = 1.0
    Ac = P.T @ J @ P
    Dc = np.zeros_like(Ac)
    for i in range(Nc):
        idx = i + Nc * np.arange(nu)
        Dc[np.ix_(idx, idx)] = np.linalg.inv(Ac[np.ix_(idx, idx)])
    r = np.random.default_rng(4).standard_normal(nu * N)
    rc = P.T @ r
    zc = np.zeros(nu * Nc)
    for _ in range(mg.COARSE_SWEEPS):
        zc = zc + mg.OMEGA * Dc @ (rc - Ac @ zc)
    ref = P @ zc
    got = H.cycle(r, nu1=0, nu2=0)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [16, 32])
def test_cycle_preconditions_gmres(n):
    # on the beam workload's first Newton system the cycle needs fewer Krylov steps than
    # point-block Jacobi (the reason it exists)
    import scipy.sparse.linalg as spla
    p = si.beam_lognormal_2d(n, n, dt_factor=10.0)
    s = Scheme(p)
    u = s.pack(s.Un)
    px, py = _periodic(p)
    H = mg.Hierarchy(lambda v: s.jv(u, v), s.nu, n, n, px, py, coarsest=4)
    b = -s.residual(u)
    J = spla.LinearOperator((b.size, b.size), matvec=lambda v: s.jv(u, v))
    counts = {}
    for name, M in (("bj", lambda r: mg.apply_blocks(H.dinv[0], r)), ("mg", H.cycle)):
        it = [0]

        def cb(_):
            it[0] += 1
        _, info = spla.gmres(J, b, rtol=1e-6, restart=30, maxiter=400,
                             M=spla.LinearOperator(J.shape, matvec=M), callback=cb, callback_type="pr_norm")
        assert info == 0
        counts[name] = it[0]
    assert counts["mg"] < counts["bj"], counts
