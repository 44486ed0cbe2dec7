"""GPU parity of the 3D J v tiled in x-y and marching in z (wave speeds frozen at time n
or fixed), against the oracle's dual-number J v: FP64 within 1e-12 relative per
component, FP32 within 1e-4 in the 2-norm (inputs rounded to FP32).

Grids are ragged against the 32 x 8 x 16 tiles and slabs, and the cases cover every
boundary kind on some axis (Dirichlet with a partial mask, periodic, reflect,
outflow), gas coupling and radiation only, the well-balanced and the centred
source, the boundary closure of Eq. (boundaryCondition) on and off, and fixed
wave speeds. One case runs the whole implicit step on the tiled path against the
oracle's Newton solve (state within 1e-7, oracle residual within 1e-8).
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, newton_solve
from tests.m1_cases import gas_3d, perturbed_state

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


def _rel(a, b, nu, N):
    return max(np.abs(a[k * N:(k + 1) * N] - b[k * N:(k + 1) * N]).max()
               / max(np.abs(b[k * N:(k + 1) * N]).max(), 1e-300) for k in range(nu))


def _case(name):
    if name == "gas_frozen":
        p = gas_3d(n=(37, 13, 19), seed=7)
    elif name == "gas_fixed_centred":
        p = gas_3d(n=(33, 9, 17), seed=8)
        p.fixed_eigs, p.well_balanced = True, False
    elif name == "gas_no_wb_boundary":
        p = gas_3d(n=(35, 10, 18), seed=9)
        p.wb_boundary = False
    else:  # radiation only, periodic in x and y, outflow in z
        rng = np.random.default_rng(10)
        p = si.make_problem(3, (34, 11, 20), bc=[("periodic", "periodic"), ("periodic", "periodic"),
                                                  ("outflow", "reflect")], dt_factor=30)
        p.E = rng.uniform(0.2, 2.0, p.shape)
        d = rng.standard_normal((3,) + p.shape)
        d /= np.linalg.norm(d, axis=0, keepdims=True)
        p.F = p.c * p.E * rng.uniform(0.0, 0.95, p.shape) * d
        p.sigma_a = 10.0 ** rng.uniform(-2, 2, p.shape)
        p.sigma_f = p.sigma_a.copy()
        p.B = rng.uniform(0.0, 1.0, p.shape)
    p.implicit_eigs = False
    return p


CASES = ["gas_frozen", "gas_fixed_centred", "gas_no_wb_boundary", "radiation_periodic"]


@pytest.mark.parametrize("name", CASES)
def test_jv3d_tiled_fp64(m1mod, name):
    p = _case(name)
    s = Scheme(p)
    u = perturbed_state(p, 21)
    v = np.random.default_rng(22).standard_normal(u.size)
    ctx = _ctx(m1mod, p)
    assert _rel(ctx.jv(p.dt, u, v), s.jv(u, v), s.nu, s.N) < 1e-12


@pytest.mark.parametrize("name", CASES)
def test_jv3d_tiled_fp32(m1mod, name):
    p = _case(name)
    s = Scheme(p)
    u = perturbed_state(p, 23)
    v = np.random.default_rng(24).standard_normal(u.size)
    ctx = _ctx(m1mod, p)
    got = ctx.jv(p.dt, u, v, precision=m1mod.PREC_MIXED)
    ref = s.jv(u, v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4


def test_implicit_step_on_the_tiled_path(m1mod):
    p = _case("gas_frozen")
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    assert ref.converged
    for prec in (m1mod.PREC_FP64, m1mod.PREC_MIXED):
        ctx = _ctx(m1mod, p)
        opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0, precision=prec)
        st, info = ctx.implicit_step(p.dt, opts)
        assert info.converged
        u = ctx.get_solution()
        assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
        assert _rel(u, ref.u, s.nu, s.N) < 1e-7
