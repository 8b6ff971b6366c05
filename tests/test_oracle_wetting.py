"""Wetting by the fictitious wall densities (Eq. 18-19), CPU only.

With zeta = 1 for both components the wall holds the weighted mean of its
fluid neighbours, so the wall is neutral and a sessile droplet relaxes to a
90 degree contact angle (the paper's choice, Sec. III). Sessile D2Q9 droplets
(radius 8) start as circular caps at 60, 90 and 120 degrees and must settle
at 90 +- 3 degrees. The angle is read from the cap's height h above the wall
and its half-width a on the first row, tan(theta/2) = h/a; on this lattice the
reading carries 1-2 degrees of discreteness. zeta_ink > 1 (hydrophilic) or
< 1 (hydrophobic) must move the angle below or above 90 degrees."""
import numpy as np
import pytest

import oracle as O


def _cap(shape, R, theta0, width=1.5):
    """A circular cap of ink meeting the wall plane z = -1/2 at theta0."""
    nx, ny, nz = shape
    zc = -0.5 - R * np.cos(np.radians(theta0))
    x = np.arange(nx)[None, None, :] - nx / 2 + 0.5
    z = np.arange(nz)[:, None, None]
    r = np.sqrt(x * x + (z - zc) ** 2)
    c = np.broadcast_to(0.5 * (1 - np.tanh((r - R) / width)), (nz, ny, nx)).copy()
    return c, 1 - c


def contact_angle(rn):
    """Degrees, from the rho^N = 0 level set of a cap centred on the middle
    column: height of the crossing on that column, half-width on row z = 0."""
    nx = rn.shape[1]
    col = rn[:, nx // 2]
    k = int(np.where(col < 0)[0][0])
    h = (k - 1) + col[k - 1] / (col[k - 1] - col[k]) + 0.5
    row = rn[0]
    inside = np.where(row > 0)[0]
    xl, xr = inside[0], inside[-1]
    ar = xr + row[xr] / (row[xr] - row[xr + 1])
    al = xl - row[xl] / (row[xl] - row[xl - 1])
    return 2 * np.degrees(np.arctan(h / ((ar - al) / 2)))


def _run(theta0, steps, zeta_ink=1.0):
    shape = (48, 1, 24)
    o = O.Oracle(shape, params=dict(velset=O.D2Q9, tau_amb=1.0, A=0.01, beta=0.7, zeta_ink=zeta_ink, zeta_amb=1.0),
                 geom=dict(nozzle=0, z_mode=O.Z_WALLS, top_mode=O.TOP_WALL),
                 rheo=dict(law=O.NEWTONIAN, nu0=1 / 6, tau_min=0.501, tau_max=5.0))
    o.set_fields(*_cap(shape, 8.0, theta0))
    th0 = contact_angle(o.fields()["rhoN"][:, 0, :])
    o.step(steps)
    return th0, contact_angle(o.fields()["rhoN"][:, 0, :])


@pytest.mark.parametrize("theta0,steps", [(60, 6000), (90, 4000), (120, 12000)])
def test_neutral_wall_gives_ninety_degrees(theta0, steps):
    start, end = _run(theta0, steps)
    assert abs(start - theta0) < 3
    assert abs(end - 90.0) <= 3.0, (theta0, end)


@pytest.mark.parametrize("zeta_ink,sign", [(1.3, -1), (0.77, +1)])
def test_affinity_moves_the_angle(zeta_ink, sign):
    """Sec. II A: zeta > 1 is hydrophilic, zeta < 1 hydrophobic."""
    _, end = _run(90, 3000, zeta_ink=zeta_ink)
    assert sign * (end - 90.0) > 3.0, end
