"""Print-quality index of the deposited thread (Sec. IV), host-side post-processing
of a 2D (x-z) run's fields.

The paper rates a print by POI = (A_i / A_r) d / (h Delta p_m):
  - A_i, the sectional area of the ink thread;
  - A_r, the area of the rectangle circumscribing it (A_i / A_r, the coverage ratio);
  - h, the thread's largest height behind the moving nozzle;
  - Delta p_m, the largest pressure variation in the ink outside the nozzle
    with respect to the equilibrium pressure p_0;
  - d, the nozzle diameter;
and compares runs by POI_i / max_i POI_i.
Ink nodes are those with rho^N > 0. The thread is taken in a window of columns
behind the nozzle and below its tip (the caller gives both); areas are node
counts (one node = one lattice area unit)."""
import numpy as np


def thread_metrics(rho_n, p, x_lo, x_hi, z_top, p0):
    """rho_n, p: [nz, nx] fields of the x-z plane (z = 0 on the substrate).
    Columns x_lo <= x < x_hi, planes z < z_top. Returns h, A_i, A_r, the
    coverage ratio and Delta p_m (None where the window holds no ink)."""
    rho_n = np.asarray(rho_n, dtype=np.float64)[:z_top, x_lo:x_hi]
    p = np.asarray(p, dtype=np.float64)[:z_top, x_lo:x_hi]
    ink = rho_n > 0
    if not ink.any():
        return dict(h=0, A_i=0, A_r=0, coverage=None, dp_max=None)
    zs, xs = np.nonzero(ink)
    h = int(zs.max()) + 1                      # rows 0 .. zmax hold ink
    width = int(xs.max() - xs.min()) + 1
    A_i = int(ink.sum())
    A_r = h * width
    return dict(h=h, A_i=A_i, A_r=A_r, coverage=A_i / A_r, dp_max=float(np.abs(p[ink] - p0).max()))


def poi(coverage, d, h, dp_max):
    """POI = (A_i / A_r) d / (h Delta p_m), up to the paper's proportionality."""
    return coverage * d / (h * dp_max)


def normalised(values):
    """POI_i / max_i POI_i."""
    v = np.asarray(values, dtype=np.float64)
    return v / v.max()
