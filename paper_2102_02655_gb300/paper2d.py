"""The paper's 2D print runs (Sec. III-IV) on the GPU: D2Q9 880 x 240, a
Table I ink at density ratio 842, the nozzle moving at speed_ratio x v_ink.
Each run goes until the nozzle has travelled six diameters past the column
where the ink first touched the substrate (the paper's stopping rule), then
reports the thread's height one diameter behind the nozzle (sampled along the
way, to see it settle), its coverage ratio and largest pressure variation over
the whole thread, and POI (paper_2102_02655_gb300.poi).

    python -m paper_2102_02655_gb300.paper2d --ink 1%-25C --speed 1.0 [--storage f64] [--ratio 842]
        [--alpha-air 0.2] [--a-scale 1] [--beta 0.7] [--drag 0]

prints one JSON line per run. The fields are read back every --every steps
(the touch is detected at that granularity)."""
import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import lbm, poi


def run(ink, speed, storage="f64", every=1000, max_steps=3_000_000, travel_d=6.0, device=0, ratio=I.DENSITY_RATIO,
        alpha_air=0.2, a_scale=1.0, beta=None, drag=0.0):
    """One run; alpha_air, a_scale (a factor on the A that Eq. 13 gives),
    beta and the substrate friction gamma of Eq. 29 (drag) change the choices
    the paper does not print."""
    import torch
    w = I.paper_print_2d(ink, speed_ratio=speed, storage=storage, ratio=ratio, alpha_air=alpha_air)
    w["params"]["A"] *= a_scale
    w["params"]["drag_gamma"] = drag
    if beta is not None:
        w["params"]["beta"] = beta
    shape = w["shape"]
    nx, _, nz = shape
    g = w["geom"]
    d = 2 * g["r_inner"]
    r_out = g["r_inner"] + g["wall_thickness"]
    p0 = 0.6 * (1 - w["params"]["alpha_amb"]) * w["params"]["rho0_amb"]  # air at rest (D2Q9 pressure, Eq. 8)
    torch.cuda.set_device(device)
    lat = lbm.Lattice(shape, w["params"], g, w["rheo"], device=device)
    rY, rB = I.nozzle_fill(shape, g, rho0_ink=ratio, rho0_amb=w["params"]["rho0_amb"])
    lat.set_fields(rY, rB)
    head = lambda n: g["head_pos"][0] + g["head_vel"][0] * n  # noqa: E731  (no wrap in these runs)
    # the thread's height is read one diameter behind the nozzle's trailing
    # wall (where it has settled); its coverage and pressure over all of it
    near = lambda rn, p, n: poi.thread_metrics(rn, p, int(np.ceil(head(n) + r_out)),  # noqa: E731
                                                int(np.ceil(head(n) + r_out + d)), int(g["gap"]), p0)
    mask = lbm.LBM_FIELD_PHI | lbm.LBM_FIELD_P
    n, touch, x_touch, series, status = 0, None, None, [], "done"
    t0 = time.perf_counter()
    while n < max_steps:
        try:
            lat.step(every)
            n += every
            f = lat.fields(mask=mask)
        except lbm.LBMError as e:
            status = "unstable: %s" % e
            break
        rn = f["rhoN"][:, 0, :]
        if touch is None and (rn[0] > 0).any():
            touch, x_touch = n, head(n)
        if touch is not None:
            series.append((n, round(x_touch - head(n), 2), near(rn, f["p"][:, 0, :], n)["h"]))
            if x_touch - head(n) >= travel_d * d:
                break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = dict(ink=ink, speed_ratio=speed, density_ratio=ratio, alpha_air=alpha_air, A=w["params"]["A"],
               beta=w["params"]["beta"], drag_gamma=drag, storage=storage, shape=shape, steps=n, status=status,
               mlups=nx * nz * n / wall / 1e6, wall_s=wall, v_ink_lb=g["u_ink"], touch_step=touch)
    if touch is not None and status == "done":
        pp = f["p"][:, 0, :]
        m = poi.thread_metrics(rn, pp, int(np.ceil(head(n) + r_out)), nx, int(g["gap"]), p0)
        h = near(rn, pp, n)["h"]
        out.update(h=h, h_max=m["h"], A_i=m["A_i"], A_r=m["A_r"], coverage=m["coverage"], dp_max=m["dp_max"])
        out["poi"] = poi.poi(m["coverage"], d, h, m["dp_max"]) if m["coverage"] and h else None
        out["height_series"] = series[:: max(1, len(series) // 40)]
    lat.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ink", default="1%-25C", choices=list(I.TABLE1))
    ap.add_argument("--speed", type=float, nargs="+", default=[1.0])
    ap.add_argument("--storage", default="f64")
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--max-steps", type=int, default=3_000_000)
    ap.add_argument("--ratio", type=float, default=I.DENSITY_RATIO, help="density ratio (the paper's: 842)")
    ap.add_argument("--alpha-air", type=float, default=0.2, help="alpha_B (not given in the paper)")
    ap.add_argument("--a-scale", type=float, default=1.0, help="factor on A from Eq. 13")
    ap.add_argument("--beta", type=float, default=None, help="recolouring beta (default 0.7)")
    ap.add_argument("--drag", type=float, default=0.0, help="friction gamma of Eq. 29 within 4 nodes of the substrate")
    a = ap.parse_args()
    res = [run(a.ink, s, a.storage, a.every, a.max_steps, ratio=a.ratio, alpha_air=a.alpha_air, a_scale=a.a_scale,
               beta=a.beta, drag=a.drag) for s in a.speed]
    ok = [r for r in res if r.get("poi")]
    if ok:
        for r, v in zip(ok, poi.normalised([r["poi"] for r in ok])):
            r["poi_norm"] = v
    for r in res:
        print(json.dumps(r))


if __name__ == "__main__":
    main()
