"""The allocation-free residual (m1_residual_noalloc) against the context
path (m1_residual), through the C ABI on the GPU.

Callers that cannot allocate device memory at the call site use the
allocation-free entry point; its working memory is a static device array of
the library. This file runs last so that a failure here comes after every
other test; it must pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import seeded_inputs as si
from tests.m1_cases import gas_3d, perturbed_state

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2011_13926_gb300 import m1
    return torch, m1


def _device_fields(torch, m1, p):
    keep = []

    def dev(x, dtype=torch.float64):
        if x is None:
            return None
        t = torch.from_numpy(np.array(np.asarray(x).ravel())).to(dtype=dtype).cuda()
        keep.append(t)
        return t.data_ptr()

    f = m1.DeviceFields()
    f.Un = dev(p.state_vector())
    f.sigma_a = dev(p.sigma_a)
    f.sigma_f = dev(p.sigma_f)
    f.B = dev(p.B) if not p.gas else None
    f.S = dev(p.S)
    f.rho_cv = dev(p.rho_cv) if p.gas else None
    for (a, side), (Eg, Fg, mask) in p.boundary.items():
        M = p.ncell // p.n[a]
        f.bE[a][side] = dev(np.broadcast_to(np.asarray(Eg, float).ravel(), (M,)))
        f.bF[a][side] = dev(np.asarray(Fg, float).reshape(p.dim, -1))
        if mask is not None:
            f.bmask[a][side] = dev(np.broadcast_to(np.asarray(mask, np.uint8).ravel(), (M,)), torch.uint8)
    return f, keep


@pytest.mark.parametrize("case", ["beam2d", "gas3d"])
def test_noalloc_matches_context_residual(case):
    torch, m1 = _setup()
    p = si.beam_lognormal_2d(60, 40, dt_factor=10.0) if case == "beam2d" else gas_3d()
    assert p.ncell <= m1.NOALLOC_MAX_CELLS
    ctx = m1.context_from_problem(p)
    f, keep = _device_fields(torch, m1, p)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the static working array
        u = perturbed_state(p, 100 + call)
        r_ctx = ctx.residual(p.dt, u)
        U = torch.from_numpy(u).cuda()
        R = torch.full_like(U, np.nan)
        n2 = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        st = m1.residual_noalloc(ctx.desc, p.dt, f, U.data_ptr(), R.data_ptr(), n2.data_ptr(), stream)
        assert st == m1.M1_OK
        torch.cuda.synchronize()
        r_na = R.cpu().numpy()
        N = p.ncell
        for k in range(p.n_u):
            a, b = r_na[k * N:(k + 1) * N], r_ctx[k * N:(k + 1) * N]
            assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)
        assert float(n2.item()) == pytest.approx(float(np.dot(r_ctx, r_ctx)), rel=1e-12)
    ctx.close()


def test_noalloc_rejects_oversized_grid():
    torch, m1 = _setup()
    d = m1.grid_desc(2, (257, 256))  # 65792 cells > 65536
    f = m1.DeviceFields()
    U = torch.zeros(3 * 257 * 256, dtype=torch.float64, device="cuda")
    f.Un = U.data_ptr()
    f.sigma_a = U.data_ptr()
    st = m1.residual_noalloc(d, 0.1, f, U.data_ptr(), U.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    assert st == m1.M1_ERR_ARG
