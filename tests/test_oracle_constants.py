"""Pins of the oracle's lattice constants against the values the paper prints
(Sec. II A) and against exact lattice identities. CPU only."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "d2q9_constants.json")))


def _frac(s):
    return float(Fraction(s))


def test_d2q9_weights_and_B_match_paper():
    c, w, B = O.velset(O.D2Q9)
    assert c.shape == (9, 3)
    assert np.all(c[:, 1] == 0)  # laid in the x-z plane
    n2 = (c * c).sum(1)
    for i in range(9):
        assert w[i] == pytest.approx(_frac(GOLD["weights_by_norm2"][str(n2[i])]), abs=1e-16)
        assert B[i] == pytest.approx(_frac(GOLD["B_by_norm2"][str(n2[i])]), abs=1e-15)


@pytest.mark.parametrize("alpha", [4.0 / 9.0, 0.2, 0.9])
def test_d2q9_phi_matches_paper(alpha):
    c, w, B = O.velset(O.D2Q9)
    n2 = (c * c).sum(1)
    for i in range(9):
        expect = {0: alpha, 1: (1 - alpha) / 5, 2: (1 - alpha) / 20}[n2[i]]
        assert O.phi(O.D2Q9, alpha, i) == pytest.approx(expect, abs=1e-16)


def test_phi_reduces_to_weights_at_density_ratio_one():
    for vs in (O.D2Q9, O.D3Q19):
        c, w, B = O.velset(vs)
        for i in range(len(w)):
            assert O.phi(vs, w[0], i) == pytest.approx(w[i], abs=1e-16)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
def test_lattice_isotropy(vs):
    c, w, B = O.velset(vs)
    D = 2 if vs == O.D2Q9 else 3
    axes = [0, 2] if vs == O.D2Q9 else [0, 1, 2]
    cs2 = 1.0 / 3.0
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose((w[:, None] * c).sum(0), 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    for a in axes:
        for b in axes:
            assert M2[a, b] == pytest.approx(cs2 if a == b else 0.0, abs=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    for a in axes:
        for b in axes:
            for cc in axes:
                for d in axes:
                    iso = cs2 * cs2 * ((a == b) * (cc == d) + (a == cc) * (b == d) + (a == d) * (b == cc))
                    assert M4[a, b, cc, d] == pytest.approx(iso, abs=1e-15)
    # opposite of every link present
    s = {tuple(v) for v in c}
    assert all(tuple(-v) in s for v in c)
    assert len(w) == (9 if D == 2 else 19)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
def test_perturbation_B_conditions(vs):
    """sum B = c_s^2 (the perturbation conserves mass) and sum B c c = I/3
    (its stress is proportional to n n - I, which gives sigma = 2 tau A / 9)."""
    c, w, B = O.velset(vs)
    axes = [0, 2] if vs == O.D2Q9 else [0, 1, 2]
    assert B.sum() == pytest.approx(1.0 / 3.0, abs=1e-15)
    M = np.einsum("i,ia,ib->ab", B, c, c)
    for a in axes:
        for b in axes:
            assert M[a, b] == pytest.approx(1.0 / 3.0 if a == b else 0.0, abs=1e-15)


def test_wall_interp_exact_for_quadratics():
    """Three-point extrapolation to the half-way point is exact for any quadratic."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b, cq = rng.normal(size=3)
        f = lambda d: a + b * d + cq * d * d
        assert O.wall_interp(f(0.5), f(1.5), f(2.5)) == pytest.approx(a, abs=1e-13)
