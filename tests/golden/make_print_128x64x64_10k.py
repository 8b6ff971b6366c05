"""Write print_128x64x64_10k.npz: the FP64 oracle's fields after 10,000 steps of
the 128x64x64 print run (the downscale of the 512x128x128 throughput lattice),
sampled on every 4th site in x, y and z, plus the diagnostics.

Calls only the oracle. Inputs are the seeded ones every test uses: the nozzle
filled with ink above the gap, ambient elsewhere with a +-1e-4 splitmix64
perturbation (seed 0), rounded to FP32 so that every storage mode starts from
the same values.

    python tests/golden/make_print_128x64x64_10k.py   # about 30 min on 8 cores
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
SUB = 4


def main():
    wl = I.workload("print_128x64x64")
    shape = wl["shape"]
    rY, rB = I.nozzle_fill(shape, wl["geom"])
    rB = I.perturbed_ambient(shape, rB, seed=0)
    rY = rY.astype(np.float32).astype(np.float64)
    rB = rB.astype(np.float32).astype(np.float64)
    ref = O.Oracle(shape, params=dict(wl["params"], storage="f64"), geom=wl["geom"], rheo=wl["rheo"])
    ref.set_fields(rY, rB)
    t0 = time.time()
    done = 0
    while done < STEPS:
        n = min(500, STEPS - done)
        ref.step(n)
        done += n
        print("step %d  %.0f s" % (done, time.time() - t0), flush=True)
    f = ref.fields()
    d = ref.diag()
    out = {k: f[k][::SUB, ::SUB, ::SUB].astype(np.float64) for k in ("rho_ink", "rho_amb", "ux", "uy", "uz", "solid")}
    out["speed_max"] = np.array(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2 + f["uz"] ** 2).max())
    out["scale_rho_ink"] = np.array(np.abs(f["rho_ink"]).max())
    out["scale_rho_amb"] = np.array(np.abs(f["rho_amb"]).max())
    out["mass"] = np.array(d["mass"])
    out["steps"] = np.array(STEPS)
    out["sub"] = np.array(SUB)
    np.savez_compressed(os.path.join(HERE, "print_128x64x64_10k.npz"), **out)


if __name__ == "__main__":
    main()
