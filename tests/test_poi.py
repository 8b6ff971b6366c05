"""Print-quality index (Sec. IV) on threads of known shape. CPU only."""
import numpy as np
import pytest

from paper_2102_02655_gb300 import poi


def _field(nz, nx, inside):
    z, x = np.mgrid[0:nz, 0:nx]
    rn = np.where(inside(z, x), 1.0, -1.0)
    return rn


def test_rectangle_covers_fully():
    rn = _field(40, 200, lambda z, x: (z < 12) & (x >= 50) & (x < 150))
    p = np.full(rn.shape, 0.2)
    p[5, 60] = 0.25
    m = poi.thread_metrics(rn, p, 0, 200, 30, p0=0.2)
    assert m["h"] == 12 and m["A_i"] == 1200 and m["A_r"] == 1200 and m["coverage"] == 1.0
    assert m["dp_max"] == pytest.approx(0.05)
    assert poi.poi(m["coverage"], 60, m["h"], m["dp_max"]) == pytest.approx(60 / (12 * 0.05))


def test_half_disc_covers_pi_over_four():
    R = 40.0
    rn = _field(60, 200, lambda z, x: (x + 0.5 - 100) ** 2 + (z + 0.5) ** 2 < R * R)
    m = poi.thread_metrics(rn, np.zeros(rn.shape), 0, 200, 60, p0=0.0)
    assert m["h"] == 40 and m["A_r"] == 80 * 40
    assert m["coverage"] == pytest.approx(np.pi / 4, rel=0.02)


def test_window_excludes_ink_outside_it():
    rn = _field(40, 200, lambda z, x: ((z < 10) & (x < 100)) | ((z < 30) & (x >= 150)))
    m = poi.thread_metrics(rn, np.zeros(rn.shape), 0, 120, 20, p0=0.0)
    assert m["h"] == 10 and m["A_i"] == 1000
    assert poi.thread_metrics(rn, np.zeros(rn.shape), 100, 150, 20, p0=0.0)["coverage"] is None


def test_normalised_to_the_best_run():
    assert list(poi.normalised([2.0, 4.0, 1.0])) == [0.5, 1.0, 0.25]
