"""Write print_128x64x64_10k.npz: the FP64 oracle's fields after 100, 200,
500, 1,000 and 10,000 steps of the 128x64x64 print run (the downscale of the
512x128x128 throughput lattice), sampled on every 4th site in x, y and z, plus
the diagnostics.

Calls only the oracle. Inputs are the seeded ones every test uses: the nozzle
filled with ink above the gap, ambient elsewhere with a +-1e-4 splitmix64
perturbation (seed 0), rounded to FP32 so that every storage mode starts from
the same values. The file serves the paths that compute in FP32 (FP32 and
16-bit storage), so the oracle takes their rounding floor for the direction
of Eq. 16 (2^-16; the oracle's arithmetic stays FP64).

    python tests/golden/make_print_128x64x64_10k.py   # about 2.5 hours on 4 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2102_02655_gb300 import inputs as I  # noqa: E402

STEPS = 10000
SNAPS = (100, 200, 500, 1000)
SUB = 4
FIELDS = ("rho_ink", "rho_amb", "ux", "uy", "uz", "solid")


def main():
    wl = I.workload("print_128x64x64")
    shape = wl["shape"]
    rY, rB = I.nozzle_fill(shape, wl["geom"])
    rB = I.perturbed_ambient(shape, rB, seed=0)
    rY = rY.astype(np.float32).astype(np.float64)
    rB = rB.astype(np.float32).astype(np.float64)
    ref = O.Oracle(shape, params=dict(wl["params"], storage="f32"), geom=wl["geom"], rheo=wl["rheo"])
    ref.set_fields(rY, rB)
    t0 = time.time()
    done = 0
    out = {}
    while done < STEPS:
        nxt = min([s for s in SNAPS if s > done] + [done + 500, STEPS])
        ref.step(nxt - done)
        done = nxt
        print("step %d  %.0f s" % (done, time.time() - t0), flush=True)
        if done in SNAPS:
            f = ref.fields()
            uscale = np.sqrt(f["ux"] ** 2 + f["uy"] ** 2 + f["uz"] ** 2).max()
            for k in FIELDS:
                out["s%d_%s" % (done, k)] = f[k][::SUB, ::SUB, ::SUB].astype(np.float64)
            out["s%d_speed_max" % done] = np.array(uscale)
            out["s%d_scale_rho_ink" % done] = np.array(np.abs(f["rho_ink"]).max())
            out["s%d_scale_rho_amb" % done] = np.array(np.abs(f["rho_amb"]).max())
    f = ref.fields()
    d = ref.diag()
    out.update({k: f[k][::SUB, ::SUB, ::SUB].astype(np.float64) for k in FIELDS})
    out["speed_max"] = np.array(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2 + f["uz"] ** 2).max())
    out["scale_rho_ink"] = np.array(np.abs(f["rho_ink"]).max())
    out["scale_rho_amb"] = np.array(np.abs(f["rho_amb"]).max())
    out["mass"] = np.array(d["mass"])
    out["steps"] = np.array(STEPS)
    out["snaps"] = np.array(SNAPS)
    out["sub"] = np.array(SUB)
    dst = sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "print_128x64x64_10k.npz")
    np.savez_compressed(dst, **out)


if __name__ == "__main__":
    main()
