"""Pins of the oracle's learned-preconditioner application forms (oracle/learned.py)
on the Jacobian of a small seeded 2D system: a network equal to the part of the
inverse that point-block Jacobi misses makes both forms exact; a zero network
reduces them to point-block Jacobi and to two Richardson sweeps with it; with
the real U-Net both forms are positively homogeneous and map zero to zero."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, block_jacobi, dense_jacobian, unet
from oracle import learned as ol

H = W = 8


@pytest.fixture(scope="module")
def system():
    p = si.gaussian_lognormal_2d(H, 1000, dt_factor=50.0)
    s = Scheme(p)
    u = p.state_vector()
    J = dense_jacobian(s, u)
    N, nu = s.N, 3
    idx = [[c * N + i for c in range(nu)] for i in range(N)]
    blocks = np.stack([J[np.ix_(ix, ix)] for ix in idx])
    Minv = block_jacobi(blocks, N, nu)
    Mdense = np.stack([Minv(e) for e in np.eye(nu * N)], axis=1)
    return p, s, u, J, Minv, Mdense


def test_block_jacobi_matrix_inverts_the_point_blocks(system):
    _, s, _, J, _, Mdense = system
    N = s.N
    for i in (0, 17, N - 1):
        ix = [c * N + i for c in range(3)]
        assert np.allclose(Mdense[np.ix_(ix, ix)] @ J[np.ix_(ix, ix)], np.eye(3), atol=1e-12)


def test_perfect_network_makes_both_forms_exact(system):
    _, _, _, J, Minv, Mdense = system
    Jinv = np.linalg.inv(J)
    miss = Jinv - Mdense  # what the training pairs target: e - M J e from J e
    net = lambda x: miss @ x  # noqa: E731
    A = lambda x: J @ x  # noqa: E731
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.standard_normal(J.shape[0])
        x = np.linalg.solve(J, v)
        scale = np.abs(x).max()
        assert np.abs(ol.additive(v, Minv, net) - x).max() <= 1e-10 * scale
        assert np.abs(ol.two_stage(v, A, Minv, net) - x).max() <= 1e-10 * scale


def test_zero_network_reduces_to_point_block_jacobi_sweeps(system):
    _, _, _, J, Minv, _ = system
    zero = lambda x: np.zeros_like(x)  # noqa: E731
    A = lambda x: J @ x  # noqa: E731
    v = np.random.default_rng(6).standard_normal(J.shape[0])
    assert np.array_equal(ol.additive(v, Minv, zero), Minv(v))
    # two Richardson sweeps x <- x + M (v - J x) from x = 0
    x = np.zeros_like(v)
    for _ in range(2):
        x = x + Minv(v - J @ x)
    z = ol.two_stage(v, A, Minv, zero)
    assert np.abs(z - x).max() <= 1e-13 * np.abs(x).max()


def test_unet_forms_are_positively_homogeneous_and_zero_preserving(system):
    p, s, u, J, Minv, _ = system
    N = s.N
    planes = unet.input_planes(u[:N], u[N:2 * N], u[2 * N:3 * N], p.sigma_f.ravel(), p.dx[0], p.c)
    net = ol.unet_map(unet.init_params(3), planes, H, W)
    A = lambda x: J @ x  # noqa: E731
    v = np.random.default_rng(7).standard_normal(3 * N)
    for form in (lambda y: ol.additive(y, Minv, net), lambda y: ol.two_stage(y, A, Minv, net)):
        z = form(v)
        assert np.abs(form(2.5 * v) - 2.5 * z).max() <= 1e-12 * np.abs(z).max()
        assert np.abs(form(np.zeros_like(v))).max() == 0.0
        # the network is not linear: the correction of v + w differs from the sum
        w = np.random.default_rng(8).standard_normal(3 * N)
        assert np.abs(form(v + w) - form(v) - form(w)).max() > 1e-6 * np.abs(z).max()


def test_unet_map_matches_the_nhwc_forward(system):
    p, s, u, _, _, _ = system
    N = s.N
    planes = unet.input_planes(u[:N], u[N:2 * N], u[2 * N:3 * N], p.sigma_f.ravel(), p.dx[0], p.c)
    theta = unet.init_params(4)
    x = np.random.default_rng(9).standard_normal(3 * N)
    nhwc = np.concatenate([x.reshape(3, N).T, planes.reshape(N, 4)], axis=1).reshape(1, H, W, unet.CIN)
    y = unet.forward(theta, nhwc).reshape(N, 3)
    got = ol.unet_map(theta, planes, H, W)(x)
    for c in range(3):
        assert np.array_equal(got[c * N:(c + 1) * N], y[:, c])
