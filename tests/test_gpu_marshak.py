"""The Marshak wave of Sect. 5.1 on the GPU.

The implicit M1 step with gas coupling (FP64, point-block Jacobi) is marched over
the seeded step schedule (dt from 0.01 up to 10, t_end = 3000, code units). The gas
temperature is then compared with the diffusive-limit reference of
oracle/diffusion.py over the same steps, as relative L2 errors. The paper reports
1.1 % with the asymptotic-preserving alpha and 84 % with plain HLL (alpha = 1).

Newton takes full steps here (line_search = 0). On this stiff exchange
(c sigma dt up to 1e5) the monotone Armijo backtracking on ||R||_2 accepts only
theta = 1/32 per iteration and stalls after about ten steps of the schedule,
while the full steps converge. The Newton tolerance of the march is 1e-6: late in
the run the residual's FP64 rounding floor (terms of size c sigma dt E cancel) is
about 1e-8 of ||R(U^n)||.

The first steps are also checked against the oracle's implicit step
(1e-8 relative residual, 1e-7 relative per field).
"""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, newton_solve
from oracle.diffusion import diffusion_reference

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


def _opts(m1mod, **kw):
    return m1mod.default_opts(precision=m1mod.PREC_FP64, precond=m1mod.PRECOND_BJ, line_search=0, **kw)


@pytest.fixture(scope="module")
def reference():
    p = si.marshak_1d()
    return diffusion_reference(p.T, 1.0, p.sigma_a, float(p.rho_cv[0]), p.dx[0], si.marshak_schedule())


def test_first_steps_match_oracle(m1mod):
    p = si.marshak_1d()
    ctx = _ctx(m1mod, p)
    N = p.ncell
    for dt in si.marshak_schedule()[:3]:
        p.dt = dt
        ref = newton_solve(Scheme(p), rtol=1e-10, gmres_rtol=1e-8, line_search=False)
        assert ref.converged
        st, info = ctx.implicit_step(dt, _opts(m1mod, newton_rtol=1e-10, gmres_rtol=1e-8))
        assert info.converged
        E, F, T = ctx.get_state()
        for got, want in ((E, ref.u[:N]), (F, ref.u[N:2 * N]), (T, ref.u[2 * N:])):
            assert np.abs(got - want).max() <= 1e-7 * np.abs(want).max()
        p.E, p.F, p.T = ref.u[:N].copy(), ref.u[N:2 * N].reshape(1, N).copy(), ref.u[2 * N:].copy()


@pytest.mark.parametrize("ap", [True, False])
def test_marshak_wave_sect51(m1mod, reference, ap):
    p = si.marshak_1d(ap_correction=ap)
    ctx = _ctx(m1mod, p)
    o = _opts(m1mod, newton_rtol=1e-6)
    dw = 0
    for k, dt in enumerate(si.marshak_schedule()):
        st, info = ctx.implicit_step(dt, o, raise_on_fail=False)
        assert st == m1mod.M1_OK and info.converged, (k, dt, info.as_dict())
        dw += info.fp64_double_word
    T = ctx.get_state()[2]
    err = np.linalg.norm(T - reference.T) / np.linalg.norm(reference.T)
    # the stiff exchange raises the double-word rounding floor above the 1e-6 target
    # late in the march: those steps take FP64 operations (M1_FP64_AUTO)
    print("relative L2 error of T:", "AP" if ap else "HLL", err, "; steps in double words:", dw,
          "of", len(si.marshak_schedule()))
    if ap:
        assert err <= 0.03
    else:
        assert err >= 0.5
