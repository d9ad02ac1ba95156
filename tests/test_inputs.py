"""Seeded synthetic inputs: shapes, ranges and determinism of the workloads shaped like the
paper's case studies (Sec. 3)."""
import numpy as np

from paper_2201_06914_gb300 import inputs as I


def test_layered_salt_ranges_and_determinism():
    v = I.layered_salt((81, 161), 25.0, seed=1)
    assert v.shape == (81, 161)
    assert v.max() <= 4725.0 + 1e-9 and v.min() >= 1500.0 * 0.95 - 1e-9
    assert np.array_equal(v, I.layered_salt((81, 161), 25.0, seed=1))
    assert v[40, 80] == 4500.0               # salt at the centre
    assert v[0].mean() < v[-1].mean()        # velocity grows with depth


def test_two_layer_config():
    sv = I.config_two_layer()
    assert sv.shape_padded == (281, 281)
    assert abs(sv.dt - 1.6e-3) < 1e-12      # CFL 0.4 of 2.5 km/s at 10 m
    assert sv.src.shape == (1, 3) and tuple(sv.src[0]) == (1000.0, 0.0, 20.0)
    assert sv.rec.shape == (1, 201, 3)
    m = sv.m_padded("true")
    assert m.dtype == np.float32 and m.shape == (281, 281)


def test_ricker_peak():
    w = I.ricker(400, 1e-3, 10.0)
    assert np.argmax(w) == 150 and abs(w[150] - 1.0) < 1e-12


def test_probes_independent_per_shot():
    Z = I.rademacher_shots(5, 3, 100, 8)
    assert Z.shape == (3, 100, 8)
    assert not np.array_equal(Z[0], Z[1])
    assert np.array_equal(Z[1], I.rademacher(6, 100, 8))


def test_tti_fields_ranges():
    e, d, th, ph = I.tti_fields((12, 14, 16), 12.5)
    assert 0 <= e.min() and e.max() <= 0.25 + 1e-12
    assert 0 <= d.min() and d.max() <= 0.1 + 1e-12
    assert th.max() <= np.radians(40) + 1e-12 and ph.max() <= np.radians(90) + 1e-12
    # delta <= eps everywhere: the pseudo-acoustic system grows where delta > eps
    assert np.all(d <= e)
    assert d.max() > 0.05   # the cap leaves delta its range where eps is large
