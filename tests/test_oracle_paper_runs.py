"""Oracle pins from two runs the paper describes (CPU only).

* Diffusive limit (Sect. 2.3, Eq. diffusionEqua): in a thick, purely scattering
  medium the M1 solution approaches the heat equation with D = c / (3 sigma). A
  Gaussian of width w then stays Gaussian:
      E(x, t) = w / sqrt(w^2 + 2 D t) exp(-(x - x0)^2 / (2 (w^2 + 2 D t))).
  The oracle's backward-Euler march with the asymptotic correction (Sect. 3.1.3)
  converges to it as dx -> 0 (dt proportional to dx^2); plain HLL (alpha = 1)
  does not, its numerical diffusion is O(sigma dx) times the physical one.
* Opacity jump (Sect. 5.2): marching to the steady state of Eq. steadyState, the
  centred source of Eq. wb_naive produces a flux peak at the jump more than 20
  times the expected constant flux; the well-balanced source of Eq. wb_smart does
  not.
"""
import json
import os

import numpy as np

import seeded_inputs as si
from oracle import Scheme, newton_solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def march(p, dts, **kw):
    n = p.ncell
    for dt in dts:
        p.dt = dt
        r = newton_solve(Scheme(p), **kw)
        assert r.converged, (dt, r.res / r.res0)
        p.E = r.u[:n].reshape(p.shape).copy()
        p.F = r.u[n:2 * n].reshape((1,) + p.shape).copy()
    return p


def gaussian_error(n, ap=True, sigma=1000.0, w=0.05, t_end=3.75, floor=1e-6):
    p = si.diffusion_gaussian_1d(n, sigma=sigma, width=w, floor=floor, ap_correction=ap)
    D = p.c / (3.0 * sigma)
    nst = int(np.ceil(t_end / (p.dx[0] ** 2 / D)))  # dt <= dx^2 / D
    march(p, [t_end / nst] * nst, rtol=1e-10, gmres_rtol=1e-10)
    x = p.centers(0)
    wt2 = w * w + 2.0 * D * t_end
    exact = floor + w / np.sqrt(wt2) * np.exp(-((x - 0.5) ** 2) / (2.0 * wt2))
    return np.sqrt(np.mean((p.E - exact) ** 2)) / np.sqrt(np.mean((exact - floor) ** 2))


def test_diffusion_limit_gaussian_converges():
    # sigma w = 50: the M1 model differs from the heat equation by O(1/(sigma w)^2) = 4e-4
    errs = [gaussian_error(n) for n in (32, 64, 128, 256)]
    for coarse, fine in zip(errs, errs[1:]):
        assert coarse / fine >= 2.0, errs  # at least first order; measured 2.8-3.8
    assert errs[-1] < 2e-3, errs
    # plain HLL at sigma dx = 15.6: O(1) error where the AP scheme is at 1.5 %
    hll = gaussian_error(64, ap=False)
    assert hll > 10.0 * errs[1] and hll > 0.3, (hll, errs)


def test_opacity_jump_flux_spike_sect52():
    golden = json.load(open(GOLDEN))["opacity_jump_naive_spike_factor_min"]["value"]
    peaks = {}
    for wb in (True, False):
        p = march(si.opacity_jump_1d(well_balanced=wb), si.opacity_jump_schedule(), rtol=1e-8,
                  newton_max=40, dense=True)
        F = p.F[0]
        expected = F[-1]  # the constant steady flux, read where the medium is transparent
        assert expected > 0.0
        thin = F[p.ncell // 2 + 2:]
        assert np.all(np.abs(thin / expected - 1.0) < 0.05)  # steady across the transparent half
        peaks[wb] = np.abs(F).max() / expected
        if not wb:
            assert np.argmax(np.abs(F)) in (p.ncell // 2 - 1, p.ncell // 2)  # at the jump
    assert peaks[False] > golden, peaks  # the paper: more than 20x with Eq. wb_naive
    assert peaks[True] < 1.2, peaks      # no peak with Eq. wb_smart
