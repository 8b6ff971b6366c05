"""A second, independent implementation of one step of the two-component
regularised colour-gradient LB model (Monteferrante et al., arXiv 2102.02655,
Sec. II A-B), in numpy, for cross-checking the C oracle on tiny lattices.

TEST INFRASTRUCTURE, written from the paper's equations and the readings the
library documents, sharing nothing with the oracle's source: its own direction
order, the printed (not the difference) form of the isotropic gradient, the
printed regularisation, and scipy's Brent root finder for the implicit shear
rate. Slow by design (Python loops over sites and links).

Geometry inputs (head position and velocity, radii) must be binary fractions,
so that the float arithmetic here classifies nodes exactly as the fixed-point
rule does.
"""
import numpy as np
from scipy.optimize import brentq

CS2 = 1.0 / 3.0


def velocity_set(vs):
    """(c, w, B, planar): D3Q19 (vs = 1) or the paper's D2Q9 in the x-z
    plane (vs = 0). Order: rest, axes, diagonals (not the oracle's order)."""
    if vs == 1:
        c = [(0, 0, 0)]
        for a in range(3):
            for s in (1, -1):
                v = [0, 0, 0]
                v[a] = s
                c.append(tuple(v))
        for a, b in ((0, 1), (0, 2), (1, 2)):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0]
                    v[a], v[b] = sa, sb
                    c.append(tuple(v))
        c = np.array(c, dtype=float)
        n2 = (c * c).sum(1)
        w = np.where(n2 == 0, 1 / 3, np.where(n2 == 1, 1 / 18, 1 / 36))
        # the D3Q19 perturbation coefficients of the library's reading
        B = np.where(n2 == 0, -2 / 9, np.where(n2 == 1, 1 / 54, 1 / 27))
        return c, w, B, False
    # D2Q9 (Sec. II A), x-z plane; weights and B_i as printed after Eq. 12
    c = np.array([(0, 0, 0), (1, 0, 0), (0, 0, 1), (-1, 0, 0), (0, 0, -1),
                  (1, 0, 1), (-1, 0, 1), (-1, 0, -1), (1, 0, -1)], dtype=float)
    n2 = (c * c).sum(1)
    w = np.where(n2 == 0, 4 / 9, np.where(n2 == 1, 1 / 9, 1 / 36))
    B = np.where(n2 == 0, -4 / 27, np.where(n2 == 1, 2 / 27, 5 / 108))
    return c, w, B, True


class NpLattice:
    """shape = (nx, ny, nz); params / geom / rheo: the test dictionaries."""

    def __init__(self, shape, params, geom, rheo):
        self.nx, self.ny, self.nz = shape
        self.p = dict(params)
        self.g = dict(geom)
        self.r = dict(rheo)
        vs = self.p.get("velset", 1)
        self.c, self.w, self.B, self.planar = velocity_set(vs)
        self.Q = len(self.w)
        ci = self.c.astype(int)
        self.opp = np.array([int(np.where((ci == -ci[i]).all(1))[0][0]) for i in range(self.Q)])
        w0 = self.w[0]
        self.alpha = [self.p.get("alpha_ink") or w0, self.p.get("alpha_amb") or w0]
        # Eq. 7: alpha at rest, the rest of 1 - alpha in proportion to w_i
        self.phi = np.array([[a if i == 0 else (1 - a) * self.w[i] / (1 - w0) for i in range(self.Q)]
                             for a in self.alpha])
        self.pfac = (self.phi * self.c[:, 0] ** 2).sum(1)  # Eq. 9: p^k = pfac_k rho^k
        self.rho0 = [self.p.get("rho0_ink", 1.0), self.p.get("rho0_amb", 1.0)]
        self.zeta = [self.p.get("zeta_ink", 1.0), self.p.get("zeta_amb", 1.0)]
        self.floor = self.p.get("grad_floor") or 2.0 ** -45
        self.walls = self.g.get("z_mode", 1) == 1
        self.lid = self.walls and self.g.get("top_mode", 0) == 1
        self.nozzle = self.walls and bool(self.g.get("nozzle", 0))
        self.n = 0
        self.ledger = {"bc": np.zeros(2), "created": np.zeros(2), "destroyed": np.zeros(2)}

    # ------------------------------------------------------------------ geometry
    def _col(self, x, y, n):
        """(in the wall annulus, inside the hole) for column (x, y) at step n."""
        hx = self.g["head_pos"][0] + n * self.g["head_vel"][0]
        hy = self.g["head_pos"][1] + n * self.g["head_vel"][1]
        dx = (x - hx) % self.nx
        dx = dx - self.nx if 2 * dx >= self.nx else dx
        dy = (y - hy) % self.ny
        dy = dy - self.ny if 2 * dy >= self.ny else dy
        d2 = dx * dx + dy * dy
        ri, ro = self.g["r_inner"], self.g["r_inner"] + self.g["wall_thickness"]
        return (ri * ri <= d2 <= ro * ro), d2 < ri * ri

    def solid(self, x, y, z, n):
        if not self.nozzle or z < self.g["gap"]:
            return False
        return self._col(x, y, n)[0]

    def fluid_mask(self, n):
        m = np.ones((self.nz, self.ny, self.nx), dtype=bool)
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    m[z, y, x] = not self.solid(x, y, z, n)
        return m

    def head_v(self):
        return np.array([self.g["head_vel"][0], self.g["head_vel"][1], 0.0])

    # ------------------------------------------------------------- equilibria
    def feq(self, k, rho, u):
        """Eq. 6 with the 2 c_s^4 reading of the quadratic term."""
        cu = self.c @ u
        return rho * (self.phi[k] + self.w * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - (u @ u) / (2 * CS2)))

    # ----------------------------------------------------------------- state
    def set_fields(self, rY, rB, u=None):
        self.fluid = self.fluid_mask(self.n)
        shp = (self.nz, self.ny, self.nx)
        self.f = np.zeros((2, self.Q) + shp)
        self.rho_prev = np.zeros((2,) + shp)
        self.u_prev = np.zeros((3,) + shp)
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    if not self.fluid[z, y, x]:
                        continue
                    uu = np.zeros(3) if u is None else np.array(u[:, z, y, x], dtype=float)
                    for k, r in enumerate((rY[z, y, x], rB[z, y, x])):
                        self.f[k, :, z, y, x] = self.feq(k, r, uu)
                        self.rho_prev[k, z, y, x] = r
                    self.u_prev[:, z, y, x] = uu

    def _wrap(self, x, y, z):
        """(x, y, z) on the lattice, or None when z leaves it (walls)."""
        x %= self.nx
        y %= self.ny
        if self.walls:
            if z < 0 or z >= self.nz:
                return None
        else:
            z %= self.nz
        return x, y, z

    # ------------------------------------------------------------------ step
    def step(self):
        Q, c, w, opp = self.Q, self.c, self.w, self.opp
        ci = c.astype(int)
        nprev, ncur = self.n, self.n + 1
        fl0 = self.fluid
        fl1 = self.fluid_mask(ncur)
        shp = (self.nz, self.ny, self.nx)
        fs = self.f
        fp = np.zeros((2, Q) + shp)
        v = self.head_v()
        # Eq. 1 with the boundary rules of Eq. 26-28, on the step n-1 geometry
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    if not fl0[z, y, x]:
                        continue
                    for i in range(Q):
                        ib = opp[i]
                        sx, sy, sz = x - ci[i, 0], y - ci[i, 1], z - ci[i, 2]
                        src = self._wrap(sx, sy, sz)
                        kind, uw = "fluid", None
                        if src is None and sz < 0:
                            kind = "rest"
                        elif src is None:
                            if self.lid:
                                kind, uw = "moving", np.array(self.g.get("top_vel", (0, 0, 0)), float)
                            elif self.nozzle:
                                in_wall, in_hole = self._col(sx % self.nx, sy % self.ny, nprev)
                                if in_wall:
                                    kind, uw = "moving", v
                                elif in_hole:  # Eq. 27: u_Inlet = u_ink + v, u_ink along -z
                                    kind, uw = "moving", v + np.array([0.0, 0.0, -self.g["u_ink"]])
                                else:
                                    kind = "open"
                            else:
                                kind = "open"
                        elif not fl0[src[2], src[1], src[0]]:
                            kind, uw = "moving", v
                        for k in range(2):
                            own = fs[k, ib, z, y, x]
                            if kind == "fluid":
                                fp[k, i, z, y, x] = fs[k, i, src[2], src[1], src[0]]
                                continue
                            if kind == "rest":
                                val = own
                            elif kind == "moving":
                                # Eq. 26, wall density extrapolated into the fluid along +c_i
                                rw = self.rho_prev[k, z, y, x]
                                p1 = self._wrap(x + ci[i, 0], y + ci[i, 1], z + ci[i, 2])
                                p2 = self._wrap(x + 2 * ci[i, 0], y + 2 * ci[i, 1], z + 2 * ci[i, 2])
                                if p1 is not None and p2 is not None and fl0[p1[2], p1[1], p1[0]] and \
                                        fl0[p2[2], p2[1], p2[0]]:
                                    r0 = self.rho_prev[k, z, y, x]
                                    r1 = self.rho_prev[k, p1[2], p1[1], p1[0]]
                                    r2 = self.rho_prev[k, p2[2], p2[1], p2[0]]
                                    rw = (15 * r0 - 10 * r1 + 3 * r2) / 8
                                val = own - 2 * w[ib] * rw * (uw @ c[ib]) / CS2
                            else:
                                # Eq. 28, half-way velocity by second-order extrapolation
                                u0 = self.u_prev[:, z, y, x]
                                uw2 = u0.copy()
                                p1 = self._wrap(x + ci[i, 0], y + ci[i, 1], z + ci[i, 2])
                                if p1 is not None and fl0[p1[2], p1[1], p1[0]]:
                                    uw2 = 1.5 * u0 - 0.5 * self.u_prev[:, p1[2], p1[1], p1[0]]
                                rw = 0.0 if k == 0 else self.g.get("rho_top_amb", 1.0)
                                cu = c[ib] @ uw2
                                val = -own + 2 * rw * (self.phi[k, ib] + w[ib] * (
                                    cu * cu / (2 * CS2 * CS2) - (uw2 @ uw2) / (2 * CS2)))
                            fp[k, i, z, y, x] = val
                            self.ledger["bc"][k] += val - own
        # moving boundary (Sec. II B): destroyed and created nodes
        rho = fp.sum(1) * fl0[None]
        for z, y, x in np.argwhere(fl0 & ~fl1):
            self.ledger["destroyed"] += rho[:, z, y, x]
            fp[:, :, z, y, x] = 0.0
        created = np.argwhere(fl1 & ~fl0)
        means = []
        for z, y, x in created:
            acc, cnt = np.zeros(2), 0
            for i in range(1, Q):
                p1 = self._wrap(x + ci[i, 0], y + ci[i, 1], z + ci[i, 2])
                if p1 is None or not (fl0[p1[2], p1[1], p1[0]] and fl1[p1[2], p1[1], p1[0]]):
                    continue
                acc += rho[:, p1[2], p1[1], p1[0]]
                cnt += 1
            means.append(acc / cnt if cnt else np.array([0.0, self.rho0[1]]))
        for (z, y, x), m in zip(created, means):
            for k in range(2):
                fp[k, :, z, y, x] = self.feq(k, m[k], v)
            self.ledger["created"] += m
        rho = fp.sum(1) * fl1[None]
        # densities with the ghost / wall planes z = -1 and z = nz (Eq. 18)
        R = np.zeros((2, self.nz + 2, self.ny, self.nx))
        R[:, 1:-1] = rho
        zl = [-1] if self.walls else []
        zh = [self.nz] if self.lid else []
        for z in zl + list(range(self.nz)) + zh:
            for y in range(self.ny):
                for x in range(self.nx):
                    if 0 <= z < self.nz and fl1[z, y, x]:
                        continue
                    num, den = np.zeros(2), 0.0
                    for i in range(1, Q):
                        p1 = self._wrap(x + ci[i, 0], y + ci[i, 1], z + ci[i, 2])
                        if p1 is None or not fl1[p1[2], p1[1], p1[0]]:
                            continue
                        num += w[i] * rho[:, p1[2], p1[1], p1[0]]
                        den += w[i]
                    R[:, z + 1, y, x] = np.array(self.zeta) * num / den if den > 0 else 0.0
        if self.walls and not self.lid:
            R[:, self.nz + 1] = R[:, self.nz]  # open top: zero normal gradient

        def dens(x, y, z):
            x %= self.nx
            y %= self.ny
            if not self.walls:
                z %= self.nz
            return R[:, z + 1, y, x]

        out = np.zeros_like(fp)
        fields = {k: np.zeros(shp) for k in ("rho_ink", "rho_amb", "ux", "uy", "uz", "nu", "p", "rhoN", "solid")}
        rho_new = np.zeros((2,) + shp)
        u_new = np.zeros((3,) + shp)
        gvec = np.array(self.p.get("body_force", (0.0, 0.0, 0.0)), float)
        for z in range(self.nz):
            for y in range(self.ny):
                for x in range(self.nx):
                    if not fl1[z, y, x]:
                        fields["solid"][z, y, x] = 1.0
                        continue
                    f = fp[:, :, z, y, x]
                    rk = f.sum(1)
                    rt = rk.sum()
                    u = (f.sum(0) @ c) / rt
                    cY, cB = rk / rt
                    nb = np.array([dens(x + ci[i, 0], y + ci[i, 1], z + ci[i, 2]) for i in range(Q)])
                    nt = nb.sum(1)
                    a = nb / np.array(self.rho0)[None]
                    # Eq. 12 in its printed form, sum_i w_i chi(x + c_i) c_i / c_s^2
                    gY = (w * nb[:, 0] / nt) @ c / CS2
                    gB = (w * nb[:, 1] / nt) @ c / CS2
                    gN = 2 * ((w * a[:, 0] / (a[:, 0] + a[:, 1])) @ c) / CS2  # rho^N = 2 a_Y/(a_Y + a_B) - 1
                    F = cB * gY - cY * gB  # Eq. 11
                    gn = np.sqrt(gN @ gN)
                    # Eq. 20: non-equilibrium stress per component
                    fe = np.array([self.feq(k, rk[k], u) for k in range(2)])
                    Pi = np.einsum("ki,ia,ib->kab", f - fe, c, c)
                    tau = self._tau(np.sqrt((Pi[0] ** 2).sum()), rk[0], rt, cY, cB)
                    Fb = rt * gvec
                    if self.walls and self.p.get("drag_gamma", 0.0) and z + 0.5 < self.p.get("drag_height", 4.0):
                        Fb = Fb - self.p["drag_gamma"] * rk[0] * u
                    tot = np.zeros(Q)
                    for k in range(2):
                        Qab = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
                        freg = fe[k] + w / (2 * CS2 * CS2) * np.einsum("iab,ab->i", Qab, Pi[k])
                        fk = freg - (freg - fe[k]) / tau
                        if np.any(Fb != 0):
                            fk = fk + self.feq(k, rk[k], u + Fb / rt) - fe[k]
                        tot += fk
                    # Eq. 10 once on the total
                    if gn > 0 and F @ F > 0:
                        tot += 0.5 * self.p.get("A", 0.01) * gn * (w * (c @ F) ** 2 / (F @ F) - self.B)
                    # Eq. 14-16 with u = 0 in both lines; cos(phi) = 0 at or below the floor
                    cn = np.sqrt((c * c).sum(1))
                    cosp = np.zeros(Q)
                    if gn > self.floor:
                        cosp[1:] = (c[1:] @ gN) / (cn[1:] * gn)
                    e0 = rk[0] * self.phi[0] + rk[1] * self.phi[1]
                    g = self.p.get("beta", 0.7) * rk[0] * rk[1] / rt ** 2 * cosp * e0
                    out[0, :, z, y, x] = cY * tot + g
                    out[1, :, z, y, x] = cB * tot - g
                    uph = u + Fb / (2 * rt)
                    aY, aB = rk[0] / self.rho0[0], rk[1] / self.rho0[1]
                    fields["rho_ink"][z, y, x], fields["rho_amb"][z, y, x] = rk
                    fields["ux"][z, y, x], fields["uy"][z, y, x], fields["uz"][z, y, x] = uph
                    fields["nu"][z, y, x] = CS2 * (tau - 0.5)
                    fields["p"][z, y, x] = self.pfac @ rk
                    fields["rhoN"][z, y, x] = (aY - aB) / (aY + aB)
                    rho_new[:, z, y, x] = rk
                    u_new[:, z, y, x] = uph
        self.f = out
        self.rho_prev = rho_new
        self.u_prev = u_new
        self.fluid = fl1
        self.fields = fields
        self.n = ncur

    def _tau(self, S, rY, rho, cY, cB):
        """Eq. 17, 24-25: the ink's tau from the root of
        g tau_Y(g) = S / (rho_Y c_s^2), mixed harmonically, clamped."""
        r = self.r
        tmin, tmax = r["tau_min"], r["tau_max"]

        def nu_law(g):
            if r["law"] == 1:
                return r["nu_inf"] + (r["nu0"] - r["nu_inf"]) / (1 + (r["lam"] * g) ** r["n"])
            if r["law"] == 2:
                if g <= 0:
                    return np.inf if r["n"] < 1 else (0.0 if r["n"] > 1 else r["K"])
                return r["K"] * g ** (r["n"] - 1)
            return r["nu0"]

        def tau_y(g):
            nu = nu_law(g)
            return tmax if np.isinf(nu) else min(max(0.5 + nu / CS2, tmin), tmax)

        if r["law"] == 0 or not S > 0 or not rY > 1e-12 * rho:
            tY = tau_y(0.0)
        else:
            s = S / (rY * CS2)
            lo, hi = s / tmax, s / tmin
            h = lambda g: g * tau_y(g) - s  # noqa: E731
            if h(lo) >= 0:
                g = lo
            elif h(hi) <= 0:
                g = hi
            else:
                g = brentq(h, lo, hi, xtol=1e-300, rtol=8.9e-16, maxiter=500)
            tY = tau_y(g)
        nuY = CS2 * (tY - 0.5)
        nuB = CS2 * (self.p.get("tau_amb", 1.0) - 0.5)
        nu = 1.0 / (cY / nuY + cB / nuB)
        return min(max(0.5 + nu / CS2, tmin), tmax)
