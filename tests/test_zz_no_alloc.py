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


def _case(name, storage):
    """(shape, workload, initial rho_ink, rho_amb) of each lattice form the call
    serves: the 3D print run, the paper's D2Q9, z-periodic, and a lid."""
    if name == "print":
        shape = (26, 18, 22)
        wl = I.print_run(shape, 4.0, 8, 0.03, 0.03, 0.6, storage, head_pos=(9.0, 9.0))
        rY, rB = I.nozzle_fill(shape, wl["geom"])
        return shape, wl, rY, I.perturbed_ambient(shape, rB, seed=3)
    if name == "d2q9":
        shape = (40, 1, 24)
        wl = I.print_run(shape, 5.0, 8, 0.02, 0.03, 0.6, storage, head_pos=(12.0, 0.0))
        wl["params"] = dict(wl["params"], velset=0)
        rY, rB = I.nozzle_fill(shape, wl["geom"])
        return shape, wl, rY, I.perturbed_ambient(shape, rB, seed=4)
    rheo = dict(law=2, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0)
    if name == "periodic":
        shape = (20, 14, 12)
        rY, rB = I.droplet(shape, (9.5, 7.0, 5.5), 4.0, width=1.5)
        return shape, dict(params=dict(velset=1, storage=storage, A=0.02), rheo=rheo,
                           geom=dict(nozzle=0, z_mode=0)), rY, rB
    # lid: substrate below, a moving lid above, a body force
    shape = (12, 10, 14)
    rY = np.zeros((14, 10, 12))
    rY[4:9] = 1.0
    return shape, dict(params=dict(velset=1, storage=storage, body_force=(1e-5, 0.0, 0.0), tau_amb=0.8),
                       rheo=dict(law=0, nu0=0.1, tau_min=0.501, tau_max=5.0),
                       geom=dict(nozzle=0, z_mode=1, top_mode=1, top_vel=(0.01, 0.002, 0.0))), rY, 1.0 - rY


@pytest.mark.parametrize("name,storage", [("print", "f64"), ("print", "f32"), ("d2q9", "f64"),
                                          ("periodic", "f32"), ("lid", "f64")])
def test_step_noalloc_matches_lbm_step_on_two_calls(name, storage):
    import torch
    from paper_2102_02655_gb300 import build, lbm
    build.build()
    shape, wl, rY, rB = _case(name, storage)
    nx, ny, nz = shape
    N = nx * ny * nz
    npd = np.float64 if storage == "f64" else np.float32
    rY, rB = rY.astype(npd), rB.astype(npd)

    # reference: the handle-based path, three steps
    lat = lbm.Lattice(shape, wl["params"], wl["geom"], wl["rheo"], path="plain")
    lat.set_fields(rY, rB)
    ref, ref_diag = [], [lat.diag()]
    for _ in range(3):
        lat.step(1)
        f = lat.fields()
        ref.append({k: np.asarray(f[k], np.float64) for k in NAMES})
        ref_diag.append(f["diag"])
    lat.close()

    # the same initial state in the storage layout: equilibrium at rest with
    # phi = w, slot 0 = w_i rho_ink, slot 1 = w_i (rho_ink + rho_amb - rho0_amb)
    planar = wl["params"].get("velset", 1) == 0
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4 if planar else [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12,
                 dtype=npd)
    Q = len(w)
    f0 = np.empty((2, Q, N), dtype=npd)
    f0[0] = w[:, None] * rY.reshape(-1)[None, :]
    f0[1] = w[:, None] * ((rY + rB).reshape(-1)[None, :] - npd(1.0))
    tdt = torch.float64 if storage == "f64" else torch.float32
    stream = torch.cuda.Stream()
    bufs = [torch.from_numpy(f0).cuda(), torch.empty((2, Q, N), dtype=tdt, device="cuda")]
    fields = torch.empty((9, N), dtype=tdt, device="cuda")
    torch.cuda.synchronize()
    cfg = lbm.make_config(shape, wl["params"], path="plain", stream=stream.cuda_stream)
    geom = lbm.make_geometry(wl["geom"])
    rheo = lbm.make_rheology(wl["rheo"])
    for n in (1, 2, 3):
        d = lbm.lbm_diag()
        src, dst = bufs[(n - 1) % 2], bufs[n % 2]
        # the third call writes no fields: the diagnostics come without the
        # field sums (mass and momentum 0), the step's boundary flux with them
        fptr = fields.data_ptr() if n < 3 else None
        st = lbm.lbm_step_noalloc(cfg, geom, rheo, n, src.data_ptr(), dst.data_ptr(), fptr, d)
        assert st == lbm.LBM_OK, lbm.lbm_last_error(None)
        stream.synchronize()
        assert d.step == n and d.unstable == 0
        scale = sum(ref_diag[n]["mass"])
        flux = [ref_diag[n]["bc_flux"][k] - ref_diag[n - 1]["bc_flux"][k] for k in range(2)]
        assert max(abs(d.bc_flux[k] - flux[k]) for k in range(2)) <= TOL[storage] * scale
        if n == 3:
            assert list(d.mass) == [0.0, 0.0] and list(d.momentum) == [0.0, 0.0, 0.0]
            continue
        got = {k: fields[i].double().cpu().numpy().reshape(nz, ny, nx) for i, k in enumerate(NAMES)}
        errs = _errors(got, ref[n - 1])
        tol = TOL[storage]
        if planar:
            errs["uy"] = 0.0
        assert max(errs.values()) <= tol, (n, errs)
        assert np.array_equal(got["solid"] != 0, ref[n - 1]["solid"] != 0)
        assert d.mass[0] > 0


def test_step_noalloc_rejects_oversized_lattice():
    from paper_2102_02655_gb300 import build, lbm
    build.build()
    wl = I.print_run((512, 128, 128), 10.0, 20, 0.01, 0.02, 0.6, "f32")
    cfg = lbm.make_config((512, 128, 128), wl["params"])
    st = lbm.lbm_step_noalloc(cfg, lbm.make_geometry(wl["geom"]), lbm.make_rheology(wl["rheo"]), 1,
                              C.c_void_p(1 << 20).value, C.c_void_p(1 << 40).value)
    assert st == lbm.LBM_EINVAL
    assert "static array" in lbm.lbm_last_error(None)
