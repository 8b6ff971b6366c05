"""ctypes wrapper around the plain FP64 CPU oracle (cglbm_oracle.c).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The product path (the
CUDA library and its binding) never imports it and shares no code with it.

The parameter dictionaries use the same keys as the product's binding so that
a test can hand one case to both sides; the oracle keeps its own structs.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

D2Q9, D3Q19 = 0, 1
NEWTONIAN, CROSS, POWER_LAW = 0, 1, 2
Z_PERIODIC, Z_WALLS = 0, 1
TOP_OPEN, TOP_WALL = 0, 1
FIELD_NAMES = ("rho_ink", "rho_amb", "ux", "uy", "uz", "nu", "p", "rhoN", "solid")


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("velset", C.c_int),
                ("tau_amb", C.c_double), ("rho0_ink", C.c_double), ("rho0_amb", C.c_double),
                ("alpha_ink", C.c_double), ("alpha_amb", C.c_double),
                ("A", C.c_double), ("beta", C.c_double),
                ("zeta_ink", C.c_double), ("zeta_amb", C.c_double),
                ("drag_gamma", C.c_double), ("drag_height", C.c_double),
                ("g", C.c_double * 3), ("grad_floor", C.c_double)]


class _Geom(C.Structure):
    _fields_ = [("z_mode", C.c_int), ("top_mode", C.c_int), ("nozzle", C.c_int),
                ("head_pos", C.c_double * 2), ("head_vel", C.c_double * 2),
                ("r_inner", C.c_double), ("wall_thickness", C.c_double),
                ("gap", C.c_int), ("u_ink", C.c_double),
                ("top_vel", C.c_double * 3), ("rho_top_amb", C.c_double)]


class _Rheo(C.Structure):
    _fields_ = [("law", C.c_int), ("nu0", C.c_double), ("nu_inf", C.c_double),
                ("lam", C.c_double), ("n", C.c_double), ("K", C.c_double),
                ("tau_min", C.c_double), ("tau_max", C.c_double)]


class _Diag(C.Structure):
    _fields_ = [("mass", C.c_double * 2), ("momentum", C.c_double * 3),
                ("bc_flux", C.c_double * 2), ("created", C.c_double * 2),
                ("destroyed", C.c_double * 2), ("step", C.c_longlong)]


_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Params)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_geometry.argtypes = [C.c_void_p, C.POINTER(_Geom)]
        L.or_set_rheology.argtypes = [C.c_void_p, C.POINTER(_Rheo)]
        L.or_set_fields.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_fields.argtypes = [C.c_void_p, dp]
        L.or_get_diag.argtypes = [C.c_void_p, C.POINTER(_Diag)]
        L.or_get_populations.argtypes = [C.c_void_p, dp]
        L.or_get_post_stream.argtypes = [C.c_void_p, dp]
        L.or_get_densities.argtypes = [C.c_void_p, dp]
        L.or_velset.argtypes = [C.c_int, C.POINTER(C.c_int), dp, dp]
        L.or_phi.restype = C.c_double
        L.or_phi.argtypes = [C.c_int, C.c_double, C.c_int]
        L.or_solve_tau_ink.restype = C.c_double
        L.or_solve_tau_ink.argtypes = [C.POINTER(_Rheo), C.c_double, C.c_double, dp]
        L.or_wall_interp.restype = C.c_double
        L.or_wall_interp.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_collide_one.argtypes = [C.c_void_p, dp, dp, C.c_double, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# |grad rho^N| at or below which Eq. 16's direction is taken as undefined
# (cos phi_i = 0): 2^8 units of rounding of the arithmetic that computes the
# gradient. A run compared with a path that computes in FP32 (FP32 or 16-bit
# storage) takes that path's level; the oracle itself computes in FP64.
GRAD_FLOOR = {"f64": 2.0 ** -45, "f32": 2.0 ** -16, "f16dev": 2.0 ** -16, "bf16dev": 2.0 ** -16}


def grad_floor(params):
    """The Eq. 16 floor of a parameter dictionary: its "grad_floor" key, else
    the level of its "storage" arithmetic (FP64 when absent)."""
    p = params or {}
    if p.get("grad_floor"):
        return float(p["grad_floor"])
    st = p.get("storage", "f64")
    return GRAD_FLOOR.get(st, GRAD_FLOOR["f64"]) if isinstance(st, str) else GRAD_FLOOR["f64"]


DEFAULT_PARAMS = dict(velset=D3Q19, tau_amb=1.0, rho0_ink=1.0, rho0_amb=1.0,
                      alpha_ink=None, alpha_amb=None, A=0.01, beta=0.7,
                      zeta_ink=1.0, zeta_amb=1.0, drag_gamma=0.0, drag_height=4.0,
                      body_force=(0.0, 0.0, 0.0))
DEFAULT_GEOM = dict(z_mode=Z_WALLS, top_mode=TOP_OPEN, nozzle=1, head_pos=(0.0, 0.0),
                    head_vel=(0.0, 0.0), r_inner=4.0, wall_thickness=2.0, gap=12,
                    u_ink=0.0, top_vel=(0.0, 0.0, 0.0), rho_top_amb=1.0)
DEFAULT_RHEO = dict(law=POWER_LAW, nu0=0.1, nu_inf=0.0, lam=1.0, n=0.6, K=0.05,
                    tau_min=0.51, tau_max=2.0)


def make_rheo(r):
    d = dict(DEFAULT_RHEO, **(r or {}))
    return _Rheo(d["law"], d["nu0"], d["nu_inf"], d["lam"], d["n"], d["K"],
                 d["tau_min"], d["tau_max"])


def velset(vs):
    """Lattice vectors, weights and perturbation coefficients B_i as built by the oracle."""
    c = (C.c_int * (3 * 19))()
    w = np.zeros(19)
    B = np.zeros(19)
    q = lib().or_velset(vs, c, _dp(w), _dp(B))
    return np.array(c[:3 * q]).reshape(q, 3), w[:q].copy(), B[:q].copy()


def phi(vs, alpha, i):
    return lib().or_phi(vs, alpha, i)


def solve_tau_ink(rheo, S, rho_ink):
    g = np.zeros(1)
    r = make_rheo(rheo)
    tau = lib().or_solve_tau_ink(C.byref(r), S, rho_ink, _dp(g))
    return tau, g[0]


def wall_interp(r0, r1, r2):
    return lib().or_wall_interp(r0, r1, r2)


class Oracle:
    """One lattice advanced by the FP64 oracle.

    shape = (nx, ny, nz); fields come back as arrays indexed [z, y, x]."""

    def __init__(self, shape, params=None, geom=None, rheo=None):
        nx, ny, nz = shape
        p = dict(DEFAULT_PARAMS, **(params or {}))
        vs = p["velset"]
        w0 = 4.0 / 9.0 if vs == D2Q9 else 1.0 / 3.0
        a_ink = w0 if p["alpha_ink"] is None else p["alpha_ink"]
        a_amb = w0 if p["alpha_amb"] is None else p["alpha_amb"]
        self.shape = (nx, ny, nz)
        self._p = _Params(nx, ny, nz, vs, p["tau_amb"], p["rho0_ink"], p["rho0_amb"],
                          a_ink, a_amb, p["A"], p["beta"], p["zeta_ink"], p["zeta_amb"],
                          p["drag_gamma"], p["drag_height"], (C.c_double * 3)(*p["body_force"]),
                          grad_floor(p))
        self.Q = 9 if vs == D2Q9 else 19
        self._h = lib().or_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle: invalid lattice parameters")
        self.set_rheology(rheo)
        self.set_geometry(geom)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def set_geometry(self, geom=None):
        d = dict(DEFAULT_GEOM, **(geom or {}))
        g = _Geom(d["z_mode"], d["top_mode"], d["nozzle"], (C.c_double * 2)(*d["head_pos"]),
                  (C.c_double * 2)(*d["head_vel"]), d["r_inner"], d["wall_thickness"], d["gap"],
                  d["u_ink"], (C.c_double * 3)(*d["top_vel"]), d["rho_top_amb"])
        if lib().or_set_geometry(self._h, C.byref(g)) != 0:
            raise ValueError("oracle: invalid geometry")

    def set_rheology(self, rheo=None):
        r = make_rheo(rheo)
        if lib().or_set_rheology(self._h, C.byref(r)) != 0:
            raise ValueError("oracle: invalid rheology")

    def set_fields(self, rho_ink, rho_amb, u=None):
        nx, ny, nz = self.shape
        rY = np.ascontiguousarray(rho_ink, dtype=np.float64).reshape(-1)
        rB = np.ascontiguousarray(rho_amb, dtype=np.float64).reshape(-1)
        assert rY.size == nx * ny * nz and rB.size == nx * ny * nz
        up = None
        if u is not None:
            # u given as [3, nz, ny, nx]; the oracle wants site-major (x fastest) triples
            ua = np.ascontiguousarray(np.moveaxis(np.asarray(u, dtype=np.float64).reshape(3, -1), 0, -1))
            up = _dp(ua)
        if lib().or_set_fields(self._h, _dp(rY), _dp(rB), up) != 0:
            raise ValueError("oracle: set_fields before set_geometry")

    def step(self, n=1):
        if lib().or_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle: step failed (geometry/rheology not set)")

    def fields(self):
        nx, ny, nz = self.shape
        out = np.zeros(len(FIELD_NAMES) * nx * ny * nz)
        lib().or_fields(self._h, _dp(out))
        out = out.reshape(len(FIELD_NAMES), nz, ny, nx)
        return {k: out[i] for i, k in enumerate(FIELD_NAMES)}

    def populations(self):
        nx, ny, nz = self.shape
        out = np.zeros(2 * self.Q * nx * ny * nz)
        lib().or_get_populations(self._h, _dp(out))
        return out.reshape(2, self.Q, nz, ny, nx)

    def post_stream(self):
        """Populations of the last step after streaming and node creation,
        before the collision: [2, Q, nz, ny, nx]."""
        nx, ny, nz = self.shape
        out = np.zeros(2 * self.Q * nx * ny * nz)
        lib().or_get_post_stream(self._h, _dp(out))
        return out.reshape(2, self.Q, nz, ny, nx)

    def densities(self):
        """Densities the last step's colour gradient read: [2, nz + 2, ny, nx],
        plane index z + 1 for z = -1 .. nz (ghost and wall planes included)."""
        nx, ny, nz = self.shape
        out = np.zeros(2 * (nz + 2) * nx * ny)
        lib().or_get_densities(self._h, _dp(out))
        return out.reshape(2, nz + 2, ny, nx)

    def diag(self):
        d = _Diag()
        lib().or_get_diag(self._h, C.byref(d))
        return dict(mass=list(d.mass), momentum=list(d.momentum), bc_flux=list(d.bc_flux),
                    created=list(d.created), destroyed=list(d.destroyed), step=d.step)

    def collide_one(self, fin, nbr, z_wall_dist=-1.0):
        fin = np.ascontiguousarray(fin, dtype=np.float64).reshape(-1)
        nbr = np.ascontiguousarray(nbr, dtype=np.float64).reshape(-1)
        out = np.zeros(2 * self.Q)
        aux = np.zeros(5)
        lib().or_collide_one(self._h, _dp(fin), _dp(nbr), z_wall_dist, _dp(out), _dp(aux))
        return out.reshape(2, self.Q), aux


def threads_used():
    """OpenMP threads the oracle will use (OMP_NUM_THREADS or all cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else os.cpu_count()
