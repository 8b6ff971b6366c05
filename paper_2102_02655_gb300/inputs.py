"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only names workloads (lattice
sizes and parameters shaped like the paper's print runs, Sec. III) and draws
seeded initial fields. Both the CUDA path and the CPU oracle receive the same
arrays from here.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated per site index, so a
field is the same whatever the order or chunking of its generation.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed, index):
    """splitmix64 output for counter ``index`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_pm(seed, n):
    """n values uniform in [-1, 1) from the top 53 bits of splitmix64."""
    u = (splitmix64(seed, np.arange(n, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    return u * (2.0 / 9007199254740992.0) - 1.0


# ---------------------------------------------------------------------------
# Named workloads. Keys match the binding's parameter dictionaries.
# ---------------------------------------------------------------------------

def print_run(shape, r_inner, gap, head_vel, u_ink, n, storage, *, wall=2.0, K=0.05,
              tau_amb=1.0, A=0.01, beta=0.7, head_pos=None):
    """A print-head lattice: moving annular nozzle over a no-slip substrate,
    open top, power-law ink injected into a Newtonian ambient (density ratio 1)."""
    nx, ny, nz = shape
    if head_pos is None:
        head_pos = (nx / 4.0, ny / 2.0)
    return dict(
        shape=shape,
        params=dict(velset=1, storage=storage, tau_amb=tau_amb, rho0_ink=1.0, rho0_amb=1.0,
                    A=A, beta=beta, zeta_ink=1.0, zeta_amb=1.0, drag_gamma=0.0,
                    drag_height=4.0, body_force=(0.0, 0.0, 0.0)),
        geom=dict(z_mode=1, top_mode=0, nozzle=1, head_pos=tuple(head_pos),
                  head_vel=(head_vel, 0.0), r_inner=r_inner, wall_thickness=wall, gap=gap,
                  u_ink=u_ink, top_vel=(0.0, 0.0, 0.0), rho_top_amb=1.0),
        rheo=dict(law=2, nu0=0.1, nu_inf=0.0, lam=1.0, n=n, K=K, tau_min=0.51, tau_max=2.0),
    )


def workload(name):
    """The named synthetic workloads.

    small_print_f64: 64x32x32 D3Q19 FP64 print run, nozzle radius 4, 12 above
        the substrate, head 0.01 l.u./step, ink n = 0.6 at 0.02 l.u./step
        (parity case; 500 steps in the reference run).
    print_512x128x128: 512x128x128 FP32 print run (8.4M sites), radius 10,
        gap 20, n = 0.6, extrusion 0.02, head 0.01 (the throughput workload).
    print_128x64x64: the 128x64x64 downscale of the same run.
    print_256x128x128: half of the throughput lattice (4.2M sites), the size
        used for detailed kernel profiles.
    """
    if name == "small_print_f64":
        return print_run((64, 32, 32), 4.0, 12, 0.01, 0.02, 0.6, "f64", head_pos=(16.0, 16.0))
    if name == "print_512x128x128":
        return print_run((512, 128, 128), 10.0, 20, 0.01, 0.02, 0.6, "f32")
    if name == "print_128x64x64":
        return print_run((128, 64, 64), 10.0, 20, 0.01, 0.02, 0.6, "f32")
    if name == "print_256x128x128":
        return print_run((256, 128, 128), 10.0, 20, 0.01, 0.02, 0.6, "f32")
    raise KeyError(name)


def nozzle_fill(shape, geom, rho0_ink=1.0, rho0_amb=1.0):
    """Initial densities of the print setup (nozzle interior filled with ink
    above the gap, ambient elsewhere), as float64 arrays [z, y, x]. Uses the
    plain distance to the axis in floating point; the library's own fixed-point
    classification agrees on every node of the named workloads."""
    nx, ny, nz = shape
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    dx = (x - geom["head_pos"][0] + nx / 2) % nx - nx / 2
    dy = (y - geom["head_pos"][1] + ny / 2) % ny - ny / 2
    inside = (dx * dx + dy * dy < geom["r_inner"] ** 2) & (z >= geom["gap"])
    inside = np.broadcast_to(inside, (nz, ny, nx))
    rY = np.where(inside, rho0_ink, 0.0)
    rB = np.where(inside, 0.0, rho0_amb)
    return rY, rB


def perturbed_ambient(shape, rho_amb, seed, amplitude=1e-4):
    """rho_amb * (1 + amplitude * U[-1, 1)) with splitmix64 noise per site."""
    nx, ny, nz = shape
    noise = uniform_pm(seed, nx * ny * nz).reshape(nz, ny, nx)
    return rho_amb * (1.0 + amplitude * noise)


def droplet(shape, center, radius, width=2.0, inside=1.0, outside=1.0):
    """A smooth ink droplet (tanh profile) in ambient: rho_ink, rho_amb [z, y, x].
    For 2D lattices (ny = 1) the droplet is a disc in the x-z plane."""
    nx, ny, nz = shape
    x = np.arange(nx)[None, None, :] - center[0]
    y = np.arange(ny)[None, :, None] - center[1]
    z = np.arange(nz)[:, None, None] - center[2]
    r = np.sqrt(x * x + (y * y if ny > 1 else 0.0 * y) + z * z)
    c = 0.5 * (1.0 - np.tanh((r - radius) / width))
    c = np.broadcast_to(c, (nz, ny, nx))
    return inside * c, outside * (1.0 - c)


# ---------------------------------------------------------------------------
# The paper's own 2D print runs (Sec. III): Table I inks, unit conversion
# (Eq. 30-33), the 240 x 880 D2Q9 box. Setup arithmetic only.
# ---------------------------------------------------------------------------

# Table I, MKS columns: nu_0, nu_inf (m^2/s; the table prints "m^2 s"),
# lambda (s), n, nu_air (m^2/s); and the LB relaxation time of the air the
# paper fixed for each ink (tau_B in [0.52, 0.54], Sec. III), read from the
# table's LB nu_air = c_s^2 (tau_B - 1/2).
TABLE1 = {
    "1%-25C": dict(nu0=15.6e-5, nu_inf=2.11e-5, lam=3.16e-3, n=0.751, nu_air=1.552e-5, tau_air=0.54),
    "2%-25C": dict(nu0=66.7e-5, nu_inf=0.69e-5, lam=5.96e-3, n=0.713, nu_air=1.552e-5, tau_air=0.53),
    "3%-25C": dict(nu0=463.6e-5, nu_inf=3.64e-5, lam=62.5e-3, n=0.573, nu_air=1.552e-5, tau_air=0.52),
    "3%-40C": dict(nu0=186.8e-5, nu_inf=5.14e-5, lam=10.2e-3, n=0.737, nu_air=1.552e-5, tau_air=0.52),
}
D_NOZZLE_MKS = 0.2e-3     # m, nozzle diameter (Sec. III)
D_NOZZLE_LB = 60          # lattice nodes
RHO_AIR_MKS = 1.184       # kg/m^3 at 25 C (the air of Eq. 32)
RHO_INK_MKS = 1000.0      # kg/m^3: an aqueous alginate solution, in Eq. 30
DENSITY_RATIO = 842.0     # gamma = rho_Y / rho_B (Sec. III)
SIGMA_MKS = 50.0e-3       # N/m
PSI_MKS = 14e-6           # kg/s, the mass flow rate of Eq. 30


def lb_units(ink):
    """Conversion factors of Eq. 31-33 for one Table I ink: dx (m), dt (s),
    dm (kg). dt follows from the air's LB viscosity c_s^2 (tau_B - 1/2)."""
    t = TABLE1[ink]
    dx = D_NOZZLE_MKS / D_NOZZLE_LB
    nu_air_lb = (t["tau_air"] - 0.5) / 3.0
    dt = dx * dx * nu_air_lb / t["nu_air"]
    dm = dx ** 3 * RHO_AIR_MKS / 1.0  # rho^B_LB = 1
    return dict(dx=dx, dt=dt, dm=dm)


def table1_lb(ink):
    """A Table I ink in lattice units: kinematic viscosities by dt/dx^2, the
    Cross time lambda / dt (in steps; the table's LB column prints its
    exponent with the sign flipped), n unchanged, the air's viscosity."""
    t = TABLE1[ink]
    u = lb_units(ink)
    k = u["dt"] / u["dx"] ** 2
    return dict(nu0=t["nu0"] * k, nu_inf=t["nu_inf"] * k, lam=t["lam"] / u["dt"], n=t["n"],
                nu_air=t["nu_air"] * k, tau_air=t["tau_air"])


def ink_speed_lb(ink):
    """v_ink of Eq. 30, psi / (rho pi (d/2)^2), in lattice units per step."""
    u = lb_units(ink)
    v = PSI_MKS / (RHO_INK_MKS * 3.141592653589793 * (D_NOZZLE_MKS / 2) ** 2)
    return v * u["dt"] / u["dx"]


def paper_print_2d(ink="1%-25C", speed_ratio=1.0, storage="f64", alpha_air=0.2, wall=4.0, shape=(880, 1, 240),
                   ratio=DENSITY_RATIO):
    """The paper's 2D print run (Sec. III): D2Q9 box 880 (x, periodic) by 240
    (z), nozzle diameter 60 and gap 60, nozzle filled with ink at start; the
    ink a Table I Cross fluid, the air Newtonian at the ink's tau_B; density
    ratio 842 by phi (Eq. 7-8: gamma = (1 - alpha_B)/(1 - alpha_Y), with
    alpha_B = alpha_air); sigma = 0.05 N/m converted and A from Eq. 13 at the
    air's tau; head speed speed_ratio x v_ink. The wall thickness is not given
    (wall). ratio < 842 gives the same run at a lower density ratio."""
    nx, ny, nz = shape
    lb = table1_lb(ink)
    u = lb_units(ink)
    v = ink_speed_lb(ink)
    alpha_ink = 1.0 - (1.0 - alpha_air) / ratio
    sigma_lb = SIGMA_MKS * u["dt"] ** 2 / u["dm"]
    A = 9.0 * sigma_lb / (2.0 * lb["tau_air"])
    return dict(
        shape=shape,
        params=dict(velset=0, storage=storage, tau_amb=lb["tau_air"], rho0_ink=float(ratio), rho0_amb=1.0,
                    alpha_ink=alpha_ink, alpha_amb=alpha_air, A=A, beta=0.7, zeta_ink=1.0, zeta_amb=1.0,
                    drag_gamma=0.0, drag_height=4.0, body_force=(0.0, 0.0, 0.0)),
        geom=dict(z_mode=1, top_mode=0, nozzle=1, head_pos=(nx - 90.0, 0.0), head_vel=(-speed_ratio * v, 0.0),
                  r_inner=D_NOZZLE_LB / 2.0, wall_thickness=wall, gap=60, u_ink=v, top_vel=(0.0, 0.0, 0.0),
                  rho_top_amb=1.0),
        rheo=dict(law=1, nu0=lb["nu0"], nu_inf=lb["nu_inf"], lam=lb["lam"], n=lb["n"], K=0.05,
                  tau_min=min(lb["tau_air"], 0.5 + 3 * lb["nu_inf"]), tau_max=0.5 + 3 * lb["nu0"]),
        units=u, sigma_lb=sigma_lb,
    )
