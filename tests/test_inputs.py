"""The seeded input generators (CPU only): SplitMix64 against the first outputs of its
published definition (Steele, Lea & Flood 2014) for seed 0, uniforms in the open
interval (0, 1), Box-Muller normals with unit moments, the smoothed field's
normalisation, and the opacity fields' exact sigma dx span."""
import numpy as np

import seeded_inputs as si


def test_splitmix64_published_outputs():
    z = si.splitmix64(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_open_interval_and_seed_dependence():
    u = si.uniform01(7, 100_000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    assert not np.array_equal(u[:10], si.uniform01(8, 10))
    assert np.array_equal(u[:10], si.uniform01(7, 10))


def test_normal_moments():
    g = si.normal(11, 200_000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01


def test_smoothed_field_normalised():
    f = si.lognormal_unit_field((64, 48), 4.0, 3)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12


def test_opacity_span_exact():
    dx = 1.0 / 96
    s = si.opacity_span((96, 96), 3.0, 5, 1e-3, 1e3, dx)
    assert np.isclose(s.min() * dx, 1e-3, rtol=1e-12) and np.isclose(s.max() * dx, 1e3, rtol=1e-12)
