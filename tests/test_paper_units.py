"""The paper's unit conversion (Sec. III, Eq. 30-33) reproduces the lattice
columns that Table I prints, from its MKS columns, the nozzle diameter (0.2 mm
= 60 nodes), the air's density and the relaxation time fixed for the air
(tau_B = 0.54, 0.53, 0.52, 0.52 for the four inks, read from the printed
nu_air). CPU only."""
import os

import pytest

from paper_2102_02655_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_lb_units.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        ink, nu0, nuinf, lm, le, n, nua = line.split()
        rows[ink] = dict(nu0=float(nu0), nu_inf=float(nuinf), lam_mant=float(lm), lam_exp=int(le), n=float(n),
                         nu_air=float(nua))
    return rows


def _digits(printed):
    """Half a unit in the last printed digit, relative."""
    s = ("%.10g" % printed).rstrip("0")
    dec = len(s.split(".")[1]) if "." in s else 0
    return 0.5 * 10 ** (-dec) / abs(printed)


@pytest.mark.parametrize("ink", list(I.TABLE1))
def test_table1_lattice_columns(ink):
    g = _table()[ink]
    lb = I.table1_lb(ink)
    for k in ("nu0", "nu_inf", "nu_air"):
        assert lb[k] == pytest.approx(g[k], rel=_digits(g[k]) + 1e-3), (k, lb[k], g[k])
    assert lb["n"] == g["n"]
    # lambda: the printed mantissa with the exponent's sign flipped
    lam = g["lam_mant"] * 10.0 ** (-g["lam_exp"])
    assert lb["lam"] == pytest.approx(lam, rel=_digits(g["lam_mant"]) + 1e-3), (lb["lam"], lam)


def test_eq31_33_printed_values():
    dts = sorted(I.lb_units(k)["dt"] for k in I.TABLE1)
    u = I.lb_units("1%-25C")
    assert u["dx"] == pytest.approx(3.333e-6, rel=1e-3)
    assert u["dm"] == pytest.approx(4.39e-17, rel=2e-3)
    assert dts[0] == pytest.approx(4.77e-9, rel=1e-3) and dts[-1] == pytest.approx(9.55e-9, rel=1e-3)


def test_density_ratio_by_alpha():
    """Eq. 8: gamma = (1 - alpha_B) / (1 - alpha_Y) = 842 for the 2D print run."""
    w = I.paper_print_2d("2%-25C")
    p = w["params"]
    assert (1 - p["alpha_amb"]) / (1 - p["alpha_ink"]) == pytest.approx(842.0, rel=1e-12)
    assert p["rho0_ink"] / p["rho0_amb"] == 842.0
    # Eq. 13 at the air's relaxation time gives back sigma (lattice units)
    assert 2 * p["tau_amb"] * p["A"] / 9 == pytest.approx(w["sigma_lb"], rel=1e-12)
    assert w["shape"] == (880, 1, 240) and w["geom"]["gap"] == 60 and 2 * w["geom"]["r_inner"] == 60
