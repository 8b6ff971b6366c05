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
