"""Batched steps (one persistent launch per size class, replayed from a CUDA
graph) against the FP64 oracle, problem by problem: the same parity bar as the
single-grid implicit path (1e-8 relative residual, 1e-7 in E and F)."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import Scheme, newton_solve

pytestmark = pytest.mark.gpu


def test_batch_matches_oracle_and_tuning_keeps_results():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2011_13926_gb300 import m1
    probs = []
    for k, (n, dtf) in enumerate([(32, 20.0), (48, 10.0), (32, 35.0), (48, 20.0), (32, 10.0)]):
        probs.append(si.gaussian_lognormal_2d(n, 1999 - k, dt_factor=dtf))
    refs = [newton_solve(Scheme(p), rtol=1e-10, gmres_rtol=1e-8) for p in probs]
    B = m1.Batch(probs)
    assert B.num_classes() == 2
    dts = [p.dt for p in probs]
    opts = m1.default_opts(newton_rtol=1e-10, gmres_rtol=1e-8)
    info, ms = B.implicit_step(dts, opts)
    sols = [B.get_solution(k) for k in range(len(probs))]
    for k, (p, ref) in enumerate(zip(probs, refs)):
        assert ref.converged
        assert info[k]["converged"] == 1, info[k]
        u = sols[k]
        s = Scheme(p)
        assert np.linalg.norm(s.residual(u)) <= 1e-8 * ref.res0
        N = p.ncell
        scaleE = np.abs(ref.u[:N]).max()
        for c in range(3):
            a, b = u[c * N:(c + 1) * N], ref.u[c * N:(c + 1) * N]
            # flux components in units of c max|E| (|F| <= cE)
            scale = np.abs(b).max() if c == 0 else max(np.abs(b).max(), p.c * scaleE)
            assert np.abs(a - b).max() <= 1e-7 * scale, (k, c)
    chosen = B.tune(dts, opts)
    assert set(chosen) <= {128, 256, 512}
    info2, ms2 = B.implicit_step(dts, opts)  # re-captured graph with the tuned CTA sizes
    for k in range(len(probs)):
        assert info2[k]["converged"] == 1
        u = B.get_solution(k)
        assert np.abs(u - sols[k]).max() <= 1e-9 * np.abs(sols[k]).max()
