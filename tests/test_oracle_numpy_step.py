"""The C oracle against an independent numpy implementation of the same step
(tests/np_cglbm.py, written separately from the paper's equations) on 4^3 to
8^3 lattices, a few steps, to 1e-13: a transcription slip in either (a wrong
sign, index, weight or dropped term) shows here. CPU only.

Cases cover every rule of the step: periodic mixtures with each ink law,
a moving nozzle (node creation and destruction, the moving-wall and inlet
rules, the open top), a lid with a body force and drag, the paper's D2Q9, and
a density ratio other than one (phi != w)."""
import numpy as np
import pytest

import oracle as O
from np_cglbm import NpLattice

TOL = 1e-13


def _random_fields(shape, seed, u_amp=0.03):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rY = 0.1 + 0.8 * rng.random((nz, ny, nx))
    rB = 0.1 + 0.8 * rng.random((nz, ny, nx))
    u = u_amp * (2 * rng.random((3, nz, ny, nx)) - 1)
    return rY, rB, u


def _compare(shape, params, geom, rheo, steps, init):
    o = O.Oracle(shape, params=params, geom=geom, rheo=rheo)
    n = NpLattice(shape, dict(O.DEFAULT_PARAMS, **params), dict(O.DEFAULT_GEOM, **geom), dict(O.DEFAULT_RHEO, **rheo))
    rY, rB, u = init
    if params.get("velset", 1) == O.D2Q9:
        u = u.copy()
        u[1] = 0.0
    o.set_fields(rY, rB, u)
    n.set_fields(rY, rB, u)
    # the two number the directions differently: match them by their vectors
    co, _, _ = O.velset(params.get("velset", O.D3Q19))
    perm = [int(np.where((co == n.c[j].astype(int)).all(1))[0][0]) for j in range(n.Q)]
    for s in range(steps):
        o.step(1)
        n.step()
        fo = o.populations()[:, perm]
        scale = np.abs(fo).max()
        d = np.abs(fo - n.f).max() / scale
        assert d < TOL, "step %d: populations differ by %.3e" % (s + 1, d)
    f = o.fields()
    for k in ("rho_ink", "rho_amb", "ux", "uy", "uz", "nu", "p", "rhoN", "solid"):
        sc = max(np.abs(f[k]).max(), 1e-2)
        assert np.abs(f[k] - n.fields[k]).max() / sc < TOL, k
    d = o.diag()
    mass = sum(d["mass"])
    for key, nk in (("bc_flux", "bc"), ("created", "created"), ("destroyed", "destroyed")):
        assert np.abs(np.array(d[key]) - n.ledger[nk]).max() < TOL * mass, key
    return o, n


@pytest.mark.parametrize("law", [
    dict(law=O.NEWTONIAN, nu0=0.12, tau_min=0.501, tau_max=5.0),
    dict(law=O.POWER_LAW, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0),
    dict(law=O.CROSS, nu0=0.4, nu_inf=0.02, lam=50.0, n=0.7, tau_min=0.51, tau_max=2.0),
])
def test_periodic_mixture_each_law(law):
    shape = (5, 4, 6)
    _compare(shape, dict(velset=O.D3Q19, tau_amb=0.9, A=0.05, beta=0.6),
             dict(nozzle=0, z_mode=O.Z_PERIODIC), law, 3, _random_fields(shape, 1))


def test_moving_nozzle_inlet_open_top():
    """Head moving 3/8 l.u. per step in x and 1/8 in y: nodes are created and
    destroyed every step; inlet, moving wall, substrate and open top all act."""
    shape = (8, 8, 8)
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, nozzle=1, head_pos=(3.5, 4.25), head_vel=(0.375, 0.125),
                r_inner=1.5, wall_thickness=1.25, gap=3, u_ink=0.0625, rho_top_amb=1.03125)
    o, n = _compare(shape, dict(velset=O.D3Q19, A=0.02, beta=0.7, drag_gamma=0.05),
                    geom, dict(law=O.POWER_LAW, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0), 3,
                    _random_fields(shape, 2))
    d = o.diag()
    assert d["created"][0] > 0 and d["destroyed"][0] > 0 and d["bc_flux"][0] != 0


def test_lid_body_force_and_drag():
    shape = (4, 5, 7)
    geom = dict(nozzle=0, z_mode=O.Z_WALLS, top_mode=O.TOP_WALL, top_vel=(0.02, -0.01, 0.0))
    _compare(shape, dict(velset=O.D3Q19, tau_amb=0.8, A=0.03, beta=0.5, drag_gamma=0.1, drag_height=3.0,
                         body_force=(1e-4, -2e-5, 3e-5), zeta_ink=1.2, zeta_amb=0.9),
             geom, dict(law=O.CROSS, nu0=0.2, nu_inf=0.05, lam=10.0, n=0.5, tau_min=0.51, tau_max=3.0), 3,
             _random_fields(shape, 3))


def test_paper_d2q9_with_nozzle():
    shape = (8, 1, 7)
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, nozzle=1, head_pos=(3.25, 0.0), head_vel=(0.25, 0.0),
                r_inner=1.0, wall_thickness=1.0, gap=3, u_ink=0.0625, rho_top_amb=1.0)
    _compare(shape, dict(velset=O.D2Q9, tau_amb=1.0, A=0.02, beta=0.7), geom,
             dict(law=O.POWER_LAW, n=0.5, K=0.04, tau_min=0.51, tau_max=2.0), 3, _random_fields(shape, 4))


def test_density_ratio_other_than_one():
    """alpha and rho0 differ per component (Eq. 7-9): phi != w, and the phase
    field and partial pressures take their general form."""
    shape = (5, 4, 5)
    _compare(shape, dict(velset=O.D3Q19, alpha_ink=0.2, alpha_amb=0.4, rho0_ink=1.25, rho0_amb=1.0,
                         tau_amb=1.1, A=0.04, beta=0.6),
             dict(nozzle=0, z_mode=O.Z_PERIODIC),
             dict(law=O.POWER_LAW, n=0.7, K=0.06, tau_min=0.51, tau_max=2.0), 3, _random_fields(shape, 5))


def test_print_like_state_with_pure_phases():
    """The print setup's initial state (pure ink in the nozzle, pure ambient
    outside, ledger-tracked inflow), four steps."""
    shape = (8, 8, 8)
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, nozzle=1, head_pos=(3.5, 4.0), head_vel=(0.125, 0.0),
                r_inner=2.0, wall_thickness=1.0, gap=3, u_ink=0.0625, rho_top_amb=1.0)
    from paper_2102_02655_gb300 import inputs as I
    rY, rB = I.nozzle_fill(shape, geom)
    _compare(shape, dict(velset=O.D3Q19), geom, dict(law=O.POWER_LAW, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0),
             4, (rY, rB + 1e-3 * I.uniform_pm(3, 512).reshape(8, 8, 8), np.zeros((3, 8, 8, 8))))
