"""lbm_step_noalloc: one time step for callers that cannot allocate device
memory (code inside another framework's memory pool or a fixed arena,
real-time loops where an allocation could stall or fail). The call takes the
populations in and out from the caller and keeps its own work space in a
static device array, so it must give the same fields as lbm_step, which
allocates its state in lbm_create.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2102_02655_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
NAMES = ("rho_ink", "rho_amb", "ux", "uy", "uz", "nu", "p", "rhoN", "solid")


def _errors(got, ref):
    us = max(np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2 + ref["uz"] ** 2).max(), 1e-2)
    out = {}
    for k in ("rho_ink", "rho_amb", "ux", "uy", "uz", "nu", "p", "rhoN"):
        scale = us if k in ("ux", "uy", "uz") else np.abs(ref[k]).max()
        out[k] = np.abs(got[k] - ref[k]).max() / scale
    return out


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_step_noalloc_matches_lbm_step_on_two_calls(storage):
    import torch
    from paper_2102_02655_gb300 import build, lbm
    build.build()
    shape = (26, 18, 22)
    nx, ny, nz = shape
    N = nx * ny * nz
    wl = I.print_run(shape, 4.0, 8, 0.03, 0.03, 0.6, storage, head_pos=(9.0, 9.0))
    rY, rB = I.nozzle_fill(shape, wl["geom"])
    rB = I.perturbed_ambient(shape, rB, seed=3)
    npd = np.float64 if storage == "f64" else np.float32
    rY, rB = rY.astype(npd), rB.astype(npd)

    # reference: the handle-based path, two steps
    lat = lbm.Lattice(shape, wl["params"], wl["geom"], wl["rheo"], path="plain")
    lat.set_fields(rY, rB)
    ref = []
    for _ in range(2):
        lat.step(1)
        f = lat.fields()
        ref.append({k: np.asarray(f[k], np.float64) for k in NAMES})
    lat.close()

    # the same initial state in the storage layout: equilibrium at rest with
    # phi = w, slot 0 = w_i rho_ink, slot 1 = w_i (rho_ink + rho_amb - rho0_amb)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=npd)
    f0 = np.empty((2, 19, N), dtype=npd)
    f0[0] = w[:, None] * rY.reshape(-1)[None, :]
    f0[1] = w[:, None] * ((rY + rB).reshape(-1)[None, :] - npd(1.0))
    tdt = torch.float64 if storage == "f64" else torch.float32
    stream = torch.cuda.Stream()
    bufs = [torch.from_numpy(f0).cuda(), torch.empty((2, 19, N), dtype=tdt, device="cuda")]
    fields = torch.empty((9, N), dtype=tdt, device="cuda")
    torch.cuda.synchronize()
    cfg = lbm.make_config(shape, wl["params"], path="plain", stream=stream.cuda_stream)
    geom = lbm.make_geometry(wl["geom"])
    rheo = lbm.make_rheology(wl["rheo"])
    for n in (1, 2):
        d = lbm.lbm_diag()
        src, dst = bufs[(n - 1) % 2], bufs[n % 2]
        st = lbm.lbm_step_noalloc(cfg, geom, rheo, n, src.data_ptr(), dst.data_ptr(), fields.data_ptr(), d)
        assert st == lbm.LBM_OK, lbm.lbm_last_error(None)
        stream.synchronize()
        got = {k: fields[i].double().cpu().numpy().reshape(nz, ny, nx) for i, k in enumerate(NAMES)}
        errs = _errors(got, ref[n - 1])
        tol = TOL[storage]
        assert errs["nu"] <= (5e-5 if storage == "f32" else tol), errs
        errs["nu"] = 0.0
        assert errs["rhoN"] <= 2 * tol, errs
        errs["rhoN"] = 0.0
        assert max(errs.values()) <= tol, (n, errs)
        assert np.array_equal(got["solid"] != 0, ref[n - 1]["solid"] != 0)
        assert d.mass[0] > 0 and d.step == n


def test_step_noalloc_rejects_oversized_lattice():
    from paper_2102_02655_gb300 import build, lbm
    build.build()
    wl = I.print_run((512, 128, 128), 10.0, 20, 0.01, 0.02, 0.6, "f32")
    cfg = lbm.make_config((512, 128, 128), wl["params"])
    st = lbm.lbm_step_noalloc(cfg, lbm.make_geometry(wl["geom"]), lbm.make_rheology(wl["rheo"]), 1,
                              C.c_void_p(1 << 20).value, C.c_void_p(1 << 40).value)
    assert st == lbm.LBM_EINVAL
    assert "static array" in lbm.lbm_last_error(None)
