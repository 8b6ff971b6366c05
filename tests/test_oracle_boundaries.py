"""Pins of the oracle's boundary and mixing rules against hand computations
(CPU only): node creation (Sec. II B), the fictitious wall densities (Eq. 18),
the harmonic viscosity mix (Eq. 17), the inlet of Eq. 27 inside the moving-wall
rule of Eq. 26, and the anti-bounce-back velocity of Eq. 28.

Each test restates the rule it pins with numpy on a small lattice whose state
makes the expected value computable by hand, so that a plausible slip in the
oracle (a wrong neighbour set, an arithmetic instead of a harmonic mean, a sign
of u_Inlet, a first- instead of second-order extrapolation) fails here."""
import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def _velset():
    c, w, B = O.velset(O.D3Q19)
    opp = np.array([int(np.where((c == -c[i]).all(1))[0][0]) for i in range(len(w))])
    return c, w, opp


def _annulus(shape, geom, n):
    """Nozzle wall nodes at step n (numpy restatement of the 3D reading: the
    vertical annulus r_in <= r <= r_in + t above the gap, around the axis at
    head_pos + n head_vel, x and y periodic). Inputs here are binary fractions,
    so the test's float arithmetic is exact."""
    nx, ny, nz = shape
    hx = geom["head_pos"][0] + n * geom["head_vel"][0]
    hy = geom["head_pos"][1] + n * geom["head_vel"][1]
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    dx = (x - hx) % nx
    dx = np.where(2 * dx >= nx, dx - nx, dx)
    dy = (y - hy) % ny
    dy = np.where(2 * dy >= ny, dy - ny, dy)
    d2 = dx * dx + dy * dy
    rin, rout = geom["r_inner"], geom["r_inner"] + geom["wall_thickness"]
    wall = (d2 >= rin * rin) & (d2 <= rout * rout) & (z >= geom["gap"])
    hole = np.broadcast_to(d2 < rin * rin, (nz, ny, nx))
    return np.broadcast_to(wall, (nz, ny, nx)), hole


def _feq(c, w, rho, u):
    """Eq. 6 at density ratio one (phi = w), with the 2 c_s^4 reading."""
    cu = c @ u
    return rho * w * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - (u @ u) / (2 * CS2))


# --------------------------------------------------------------------------
# node creation (Sec. II B)
# --------------------------------------------------------------------------

def test_created_nodes_take_the_mean_of_fluid_neighbours():
    """A resting uniform mixture (rho_Y = a, rho_B = b) and a head moving at
    v = 0.375 l.u./step: after streaming, a fluid node n next to the wall has
    density rho^k (1 + 6 sum_{wall links i} w_i c_i.v) (each link from a wall
    node returns w_i rho^k - 6 w_i rho^k_w (v.c_opp(i)) with rho_w = rho^k, as
    the extrapolation of a uniform field is uniform), and rho^k elsewhere. A
    node that becomes fluid takes f^eq(rho_bar^k, v), rho_bar^k the plain mean
    over its neighbours fluid at both steps. Checked at every created node,
    component by component."""
    shape = (14, 12, 8)
    nx, ny, nz = shape
    a, b, v = 0.3, 0.7, 0.375
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_WALL, nozzle=1, head_pos=(5.25, 6.5), head_vel=(v, 0.0),
                r_inner=2.0, wall_thickness=1.0, gap=3, u_ink=0.0, top_vel=(0.0, 0.0, 0.0))
    o = O.Oracle(shape, params=dict(A=0.0), geom=geom,
                 rheo=dict(law=O.NEWTONIAN, nu0=0.1, tau_min=0.501, tau_max=5.0))
    o.set_fields(np.full((nz, ny, nx), a), np.full((nz, ny, nx), b))
    o.step(1)
    fp = o.post_stream()
    c, w, opp = _velset()
    wall0, _ = _annulus(shape, geom, 0)
    wall1, _ = _annulus(shape, geom, 1)
    fluid0, fluid1 = ~wall0, ~wall1
    vel = np.array([v, 0.0, 0.0])

    def streamed_factor(z, y, x):
        f = 1.0
        for i in range(1, 19):
            sz, sy, sx = z - c[i, 2], (y - c[i, 1]) % ny, (x - c[i, 0]) % nx
            if 0 <= sz < nz and wall0[sz, sy, sx]:
                f += 6 * w[i] * (c[i] @ vel)
        return f

    created = np.argwhere(fluid1 & ~fluid0)
    assert len(created) >= 4
    ledger = np.zeros(2)
    for z, y, x in created:
        facs = []
        for i in range(1, 19):
            zz, yy, xx = z + c[i, 2], (y + c[i, 1]) % ny, (x + c[i, 0]) % nx
            if 0 <= zz < nz and fluid0[zz, yy, xx] and fluid1[zz, yy, xx]:
                facs.append(streamed_factor(zz, yy, xx))
        assert facs
        mean = np.mean(facs)
        for k, rho in ((0, a), (1, b)):
            expect = _feq(c, w, rho * mean, vel)
            assert np.abs(fp[k, :, z, y, x] - expect).max() < 1e-15, (z, y, x, k)
            ledger[k] += rho * mean
    # the ledger books the created mass
    assert np.allclose(o.diag()["created"], ledger, rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# fictitious wall densities (Eq. 18)
# --------------------------------------------------------------------------

def test_fictitious_wall_densities_eq18():
    """Every solid node (nozzle wall at step n, substrate plane z = -1) holds
    zeta^k sum_i w_i s_i rho^k(x + c_i) / sum_i w_i s_i over its lattice
    neighbours (s_i = 1 where x + c_i is fluid at step n), computed here from
    the fluid densities the oracle reports; zeta differs per component so a
    dropped or swapped affinity shows. Closed form on the substrate: the five
    upward neighbours weigh 1/3 (straight up) and 1/6 (each diagonal)."""
    rng = np.random.default_rng(3)
    shape = (12, 10, 7)
    nx, ny, nz = shape
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, nozzle=1, head_pos=(5.5, 4.75), head_vel=(0.125, 0.0625),
                r_inner=1.5, wall_thickness=1.25, gap=2, u_ink=0.0, rho_top_amb=1.0)
    zeta = (1.3, 0.7)
    o = O.Oracle(shape, params=dict(zeta_ink=zeta[0], zeta_amb=zeta[1]), geom=geom,
                 rheo=dict(law=O.NEWTONIAN, nu0=0.1, tau_min=0.501, tau_max=5.0))
    o.set_fields(0.2 + 0.5 * rng.random((nz, ny, nx)), 0.3 + 0.5 * rng.random((nz, ny, nx)))
    o.step(2)
    rho = o.densities()  # [2, nz + 2, ny, nx], plane z + 1
    c, w, _ = _velset()
    wall, _ = _annulus(shape, geom, 2)
    fluid = ~wall
    checked = 0
    for z in range(-1, nz):
        for y in range(ny):
            for x in range(nx):
                if z >= 0 and fluid[z, y, x]:
                    continue
                num = np.zeros(2)
                den = 0.0
                for i in range(1, 19):
                    zz, yy, xx = z + c[i, 2], (y + c[i, 1]) % ny, (x + c[i, 0]) % nx
                    if 0 <= zz < nz and fluid[zz, yy, xx]:
                        num += w[i] * rho[:, zz + 1, yy, xx]
                        den += w[i]
                for k in range(2):
                    expect = zeta[k] * num[k] / den if den > 0 else 0.0
                    assert rho[k, z + 1, y, x] == pytest.approx(expect, rel=1e-14, abs=1e-300), (k, z, y, x)
                checked += 1
    assert checked > nx * ny
    # substrate, closed form: (rho(x,y,0)/3 + sum of the four side neighbours/6) zeta
    r0 = rho[:, 1]
    side = np.roll(r0, 1, 2) + np.roll(r0, -1, 2) + np.roll(r0, 1, 1) + np.roll(r0, -1, 1)
    expect = np.array(zeta)[:, None, None] * (r0 / 3 + side / 6)
    assert np.allclose(rho[:, 0], expect, rtol=1e-14, atol=0)
    # open top: the ghost plane z = nz copies z = nz - 1
    assert np.array_equal(rho[:, nz + 1], rho[:, nz])


# --------------------------------------------------------------------------
# harmonic viscosity mix (Eq. 17)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cY", [0.3, 0.85])
def test_harmonic_viscosity_mix_eq17(cY):
    """At a mixed site with nu_Y != nu_B the relaxation time is
    1/2 + 3 nu with 1/nu = (rho_Y/rho)/nu_Y + (rho_B/rho)/nu_B, and the
    regularised BGK relaxes the mixture's non-equilibrium stress by exactly
    (1 - 1/tau) (no perturbation, no recolouring, no force)."""
    rng = np.random.default_rng(11)
    tauY, tauB = 0.8, 1.4
    nuY, nuB = (tauY - 0.5) / 3, (tauB - 0.5) / 3
    o = O.Oracle((1, 1, 1), params=dict(tau_amb=tauB, A=0.0, beta=0.0), geom=dict(nozzle=0, z_mode=O.Z_PERIODIC),
                 rheo=dict(law=O.NEWTONIAN, nu0=nuY, tau_min=0.501, tau_max=5.0))
    c, w, _ = _velset()
    u = np.array([0.01, -0.02, 0.015])
    fin = np.stack([_feq(c, w, cY, u), _feq(c, w, 1 - cY, u)])
    pert = rng.normal(size=(2, 19)) * 2e-3 * w
    fin = fin + pert  # a non-equilibrium part (u and rho are recomputed from fin)
    nbr = np.stack([np.full(19, cY), np.full(19, 1 - cY)])
    out, aux = o.collide_one(fin, nbr)
    cYs = fin[0].sum() / fin.sum()  # the site's own colour fraction
    tau = 0.5 + 3.0 / (cYs / nuY + (1 - cYs) / nuB)
    assert aux[0] == pytest.approx(tau, rel=1e-15)
    arith = 0.5 + 3.0 * (cYs * nuY + (1 - cYs) * nuB)
    assert abs(arith - tau) > 0.05  # the pin tells the two means apart
    rho = fin.sum()
    uu = (fin.sum(0) @ c) / rho

    def pineq(f):
        t = f.sum(0)
        return np.einsum("i,ia,ib->ab", t - _feq(c, w, rho, uu), c, c)

    assert np.allclose(pineq(out), (1 - 1 / tau) * pineq(fin), rtol=0, atol=1e-16)


# --------------------------------------------------------------------------
# inlet (Eq. 27 in Eq. 26)
# --------------------------------------------------------------------------

def _inlet_links(shape, geom):
    """(weight sum, count) of the links pulled into the top plane from the
    nozzle's hole: top-plane fluid sites, downward directions whose source
    column lies inside r_in (Eq. 27 applies there)."""
    nx, ny, nz = shape
    c, w, _ = _velset()
    wall, hole = _annulus(shape, geom, 0)
    s, cnt = 0.0, 0
    z = nz - 1
    for y in range(ny):
        for x in range(nx):
            if wall[z, y, x]:
                continue
            for i in range(1, 19):
                if c[i, 2] != -1:
                    continue
                if hole[z, (y - c[i, 1]) % ny, (x - c[i, 0]) % nx]:
                    s += w[i]
                    cnt += 1
    return s, cnt


def test_inlet_flux_first_step_exact():
    """With the nozzle filled with ink at rest, each inlet link returns
    f*_i + 6 w_i rho_w u_ink (Eq. 26 with u_w = u_Inlet = (0, 0, -u_ink),
    Eq. 27, head at rest), with rho_w = 1 (the extrapolation of a uniform ink
    column): the first step's ink inflow is 6 u_ink sum_{inlet links} w_i, and
    no ambient enters through the inlet (its density there is zero)."""
    shape = (16, 16, 12)
    u_ink = 0.05
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, nozzle=1, head_pos=(8.0, 8.0), head_vel=(0.0, 0.0),
                r_inner=3.0, wall_thickness=1.5, gap=4, u_ink=u_ink, rho_top_amb=1.0)
    o = O.Oracle(shape, geom=geom, rheo=dict(law=O.POWER_LAW, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0))
    s, cnt = _inlet_links(shape, geom)
    assert cnt > 100  # the 29 columns inside r_in = 3, five links each (fewer at the rim)
    o.step(1)
    d = o.diag()
    assert d["bc_flux"][0] == pytest.approx(6 * u_ink * s, rel=1e-13)
    # per full column the five links give rho u_ink: 6 (1/18 + 4/36) = 1
    assert 6 * (1 / 18 + 4 / 36) == pytest.approx(1.0, rel=1e-15)


def test_inlet_flux_at_steady_extrusion():
    """After 200 steps of steady extrusion (static head) the ink entering in
    one step is exactly 6 u_ink sum_{inlet links} w_i rho_w,i, with rho_w,i
    the wall density of Eq. 26 extrapolated along +c_i from the previous step's
    densities, (15 rho(x) - 10 rho(x + c_i) + 3 rho(x + 2 c_i))/8, or rho(x)
    where x + c_i or x + 2 c_i is a wall node: rho u_ink per inlet column,
    with rho the ink density at the inlet (here above 1: the extruded ink
    raises the pressure in the small box). Ink that reached the open top
    leaves there by Eq. 28; the ledger books both."""
    shape = (16, 16, 12)
    nx, ny, nz = shape
    u_ink = 0.05
    geom = dict(z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, nozzle=1, head_pos=(8.0, 8.0), head_vel=(0.0, 0.0),
                r_inner=3.0, wall_thickness=1.5, gap=4, u_ink=u_ink, rho_top_amb=1.0)
    o = O.Oracle(shape, geom=geom, rheo=dict(law=O.POWER_LAW, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0))
    o.step(200)
    rho = o.densities()[0, 1:nz + 1]  # ink, planes 0 .. nz-1
    fstar = o.populations()[0]         # ink, post-collision
    b0 = o.diag()["bc_flux"][0]
    o.step(1)
    got = o.diag()["bc_flux"][0] - b0
    c, w, opp = _velset()
    wall, hole = _annulus(shape, geom, 0)
    z = nz - 1
    expect, wsum, outflow = 0.0, 0.0, 0.0
    for y in range(ny):
        for x in range(nx):
            if wall[z, y, x]:
                continue
            for i in range(1, 19):
                if c[i, 2] != -1:
                    continue
                src = (z, (y - c[i, 1]) % ny, (x - c[i, 0]) % nx)
                if not hole[src]:
                    # open top (anti-bounce-back, imposed ink density 0):
                    # -f*_ib(x) replaces f*_ib(x), a change of -2 f*_ib(x)
                    if not wall[src]:
                        outflow += -2.0 * fstar[opp[i], z, y, x]
                    continue
                p1 = (z - 1, (y + c[i, 1]) % ny, (x + c[i, 0]) % nx)
                p2 = (z - 2, (y + 2 * c[i, 1]) % ny, (x + 2 * c[i, 0]) % nx)
                rw = rho[z, y, x]
                if not wall[p1] and not wall[p2]:
                    rw = (15 * rho[z, y, x] - 10 * rho[p1] + 3 * rho[p2]) / 8
                expect += 6 * u_ink * w[i] * rw
                wsum += 6 * u_ink * w[i]
    assert got == pytest.approx(expect + outflow, rel=1e-13)
    assert outflow < 0.0  # some ink already leaves through the open top
    assert 1.0 < expect / wsum < 1.5  # mean inlet ink density: pressurised ink, not a drained nozzle
    # a sign error would drain the nozzle; a missing 1/c_s^2 would be 3x off
    assert got > 0


# --------------------------------------------------------------------------
# anti-bounce-back (Eq. 28)
# --------------------------------------------------------------------------

def test_anti_bounce_back_half_way_velocity_linear_profile():
    """Open top over a flow whose velocity is linear in z, at equilibrium: each
    link through the top takes -f*_ib(x) + 2 rho_w [phi_ib + w_ib((c_ib.u_w)^2
    /(2 c_s^4) - u_w^2/(2 c_s^2))] (Eq. 28) with rho_w = 0 (ink) and rho_top
    (ambient), and u_w = u(nz - 1/2), which the second-order extrapolation
    1.5 u(nz - 1) - 0.5 u(nz - 2) gives exactly for a linear profile."""
    shape = (6, 5, 8)
    nx, ny, nz = shape
    rho_top = 1.02
    U0, U1 = np.array([0.01, -0.004, 0.002]), np.array([0.002, 0.001, -0.0015])
    o = O.Oracle(shape, geom=dict(nozzle=0, z_mode=O.Z_WALLS, top_mode=O.TOP_OPEN, rho_top_amb=rho_top),
                 rheo=dict(law=O.NEWTONIAN, nu0=0.1, tau_min=0.501, tau_max=5.0))
    rY, rB = 0.2, 0.8
    z = np.arange(nz)
    u = (U0[:, None] + U1[:, None] * z[None, :])[:, :, None, None] * np.ones((3, nz, ny, nx))
    o.set_fields(np.full((nz, ny, nx), rY), np.full((nz, ny, nx), rB), u)
    o.step(1)
    fp = o.post_stream()
    c, w, opp = _velset()
    utop = U0 + U1 * (nz - 1)
    uw = U0 + U1 * (nz - 0.5)
    for i in range(19):
        if c[i, 2] != -1:
            continue
        ib = opp[i]
        for k, rho in ((0, rY), (1, rB)):
            fstar = _feq(c, w, rho, utop)[ib]
            rw = 0.0 if k == 0 else rho_top
            cu = c[ib] @ uw
            expect = -fstar + 2 * rw * (w[ib] + w[ib] * (cu * cu / (2 * CS2 * CS2) - (uw @ uw) / (2 * CS2)))
            assert np.abs(fp[k, i, nz - 1] - expect).max() < 1e-16, (i, k)
