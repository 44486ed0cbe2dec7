"""The FP64 residual and J v in double-word arithmetic (pairs of FP32 numbers,
m1_set_fp64_arithmetic) against the oracle, beside the same kernels in FP64
operations.

* Both arithmetics meet the FP64 parity bar on every case of the parity suite
  (1D/2D/3D, gas coupling, every boundary kind, frozen, fixed and new-time wave
  speeds, ragged tiles): residual and dual-number J v within 1e-12 relative per
  component. The two differ from each other by a few 1e-14 at most.
* The implicit step in either arithmetic (plain FP64 and mixed) meets the
  implicit bar: the oracle's residual of the GPU state within 1e-8 of
  ||R(U^n)|| and the state within 1e-7 of the oracle's Newton solution.
* Selection: code units (c, a_r, dx near 1) select double words; c = 3e10
  (CGS) keeps FP64 operations. A state whose residual passes 2^100 sends the
  residual back to FP64 (the range guard) and still matches the oracle.
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, newton_solve
from tests.m1_cases import cases, gas_3d, perturbed_state

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


def _ctx(m1mod, p, mode):
    import torch
    ctx = m1mod.context_from_problem(p, stream=torch.cuda.current_stream().cuda_stream, device=True)
    ctx.set_fp64_arithmetic(mode)
    return ctx


def _rel(a, b, nu, N):
    return max(np.abs(a[k * N:(k + 1) * N] - b[k * N:(k + 1) * N]).max()
               / max(np.abs(b[k * N:(k + 1) * N]).max(), 1e-300) for k in range(nu))


CASES = cases()
CASES["gas_3d_tiled"] = lambda: _frozen(gas_3d(n=(35, 10, 18), seed=9))


def _frozen(p):
    p.implicit_eigs = False
    return p


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_jv_in_both_arithmetics(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    u = perturbed_state(p, 31)
    v = np.random.default_rng(32).standard_normal(u.size)
    r_ref, j_ref = s.residual(u), s.jv(u, v)
    got = {}
    for mode in (m1mod.FP64_NATIVE, m1mod.FP64_DOUBLE_WORD):
        ctx = _ctx(m1mod, p, mode)
        assert ctx.fp64_arithmetic() == (mode, 0)
        r, j = ctx.residual(p.dt, u), ctx.jv(p.dt, u, v)
        assert ctx.fp64_arithmetic() == (mode, 0)
        assert _rel(r, r_ref, s.nu, s.N) < 1e-12, (mode, _rel(r, r_ref, s.nu, s.N))
        assert _rel(j, j_ref, s.nu, s.N) < 1e-12, (mode, _rel(j, j_ref, s.nu, s.N))
        got[mode] = (r, j)
        ctx.close()
    rn, jn = got[m1mod.FP64_NATIVE]
    rd, jd = got[m1mod.FP64_DOUBLE_WORD]
    print(name, "double word vs FP64: residual", _rel(rd, rn, s.nu, s.N), "J v", _rel(jd, jn, s.nu, s.N))
    assert _rel(rd, rn, s.nu, s.N) < 1e-12 and _rel(jd, jn, s.nu, s.N) < 1e-12


@pytest.mark.parametrize("name", ["beam2d", "smooth2d_implicit_eigs", "gas2d_frozen", "gas_3d_tiled"])
def test_implicit_step_in_double_words(m1mod, name):
    p = CASES[name]()
    s = Scheme(p)
    ref = newton_solve(s, rtol=1e-10, gmres_rtol=1e-8)
    assert ref.converged
    for prec in (m1mod.PREC_FP64, m1mod.PREC_MIXED):
        ctx = _ctx(m1mod, p, m1mod.FP64_DOUBLE_WORD)
        opts = m1mod.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8, advance=0, precision=prec)
        st, info = ctx.implicit_step(p.dt, opts)
        assert info.converged
        u = ctx.get_solution()
        assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
        assert _rel(u, ref.u, s.nu, s.N) < 1e-7
        assert ctx.fp64_arithmetic() == (m1mod.FP64_DOUBLE_WORD, 0)
        ctx.close()


def test_auto_selection(m1mod):
    import torch
    p = si.make_problem(2, (20, 12), dt_factor=10)
    rng = np.random.default_rng(40)
    p.E = rng.uniform(0.5, 1.5, p.shape)
    p.sigma_a = rng.uniform(0.1, 10.0, p.shape)
    p.sigma_f = p.sigma_a.copy()
    ctx = m1mod.context_from_problem(p, stream=torch.cuda.current_stream().cuda_stream, device=True)
    assert ctx.fp64_arithmetic() == (m1mod.FP64_DOUBLE_WORD, 0)  # code units
    ctx.close()
    q = si.make_problem(2, (20, 12), dt_factor=10, c=3e10)
    q.E = p.E.copy()
    q.sigma_a, q.sigma_f = p.sigma_a.copy(), p.sigma_f.copy()
    ctx = m1mod.context_from_problem(q, stream=torch.cuda.current_stream().cuda_stream, device=True)
    assert ctx.fp64_arithmetic() == (m1mod.FP64_NATIVE, 0)  # c = 3e10 is outside 2^-30 .. 2^30
    ctx.set_fp64_arithmetic(m1mod.FP64_DOUBLE_WORD)
    assert ctx.fp64_arithmetic()[0] == m1mod.FP64_DOUBLE_WORD
    ctx.set_fp64_arithmetic(m1mod.FP64_AUTO)
    assert ctx.fp64_arithmetic()[0] == m1mod.FP64_NATIVE
    ctx.close()


def test_range_guard_returns_to_fp64(m1mod):
    # E of order 1e33 (finite in FP32 and FP64): residuals of order 1e33 exceed
    # the guard's 2^100 ~ 1.3e30, so the implicit step's first residual is computed
    # again in FP64 operations and the context stays there
    p = si.make_problem(2, (24, 16), dt_factor=10)
    rng = np.random.default_rng(41)
    p.E = 1e33 * rng.uniform(0.5, 1.5, p.shape)
    p.F = np.zeros((2,) + p.shape)
    p.sigma_a = rng.uniform(0.1, 10.0, p.shape)
    p.sigma_f = p.sigma_a.copy()
    p.B = np.full(p.shape, 1e33)
    s = Scheme(p)
    ctx = _ctx(m1mod, p, m1mod.FP64_AUTO)
    assert ctx.fp64_arithmetic() == (m1mod.FP64_DOUBLE_WORD, 0)
    opts = m1mod.default_opts(advance=0, precision=m1mod.PREC_FP64)
    st, info = ctx.implicit_step(p.dt, opts)
    assert info.converged
    mode, fallbacks = ctx.fp64_arithmetic()
    assert mode == m1mod.FP64_NATIVE and fallbacks == 1
    u = ctx.get_solution()
    r0 = np.linalg.norm(s.residual(p.state_vector()))
    assert np.linalg.norm(s.residual(u)) <= 1.05e-8 * r0
    ctx.close()


@pytest.mark.parametrize("rtol", [1e-8, 1e-11, 1e-13])
def test_auto_decides_per_step_from_the_measured_floor(m1mod, rtol):
    # M1_FP64_AUTO measures ||R_dw(U^n) - R_fp64(U^n)|| at the start of each step and
    # keeps double words only when the Newton target is 32 times above it
    p = CASES["gas2d_frozen"]()
    ctx = _ctx(m1mod, p, m1mod.FP64_AUTO)
    opts = m1mod.default_opts(newton_rtol=rtol, gmres_rtol=1e-10, advance=0, precision=m1mod.PREC_FP64)
    st, info = ctx.implicit_step(p.dt, opts, raise_on_fail=False)
    d = info.as_dict()
    print(rtol, d["fp64_floor"], d["fp64_double_word"], d["converged"], d["newton_iters"])
    assert 0.0 < d["fp64_floor"] < 1e-12
    assert d["fp64_double_word"] == int(rtol >= 32.0 * d["fp64_floor"])
    if d["fp64_double_word"] == 0:
        assert rtol < 32.0 * d["fp64_floor"]
    assert info.converged
    assert ctx.fp64_arithmetic() == (m1mod.FP64_DOUBLE_WORD, 0)  # outside steps the mode decides
    ctx.close()
