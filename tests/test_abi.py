"""C ABI checks that need no GPU: the library loads, exports every function
include/lbm.h declares, and rejects invalid arguments on the host before
touching a device."""
import ctypes as C
import os
import re

import pytest

from paper_2102_02655_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2102_02655_gb300 import build
    build.build()
    return lbm.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert "lbm_step" in names and "lbm_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(lbm.EXPORTS) <= set(names)


def _cfg(**kw):
    p = dict(velset=lbm.LBM_D3Q19, storage="f32")
    cfg = lbm.make_config(kw.pop("shape", (8, 8, 8)), p)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 0, "sizes"), ("velset", 7, "velocity set"), ("storage", 9, "storage"),
    ("tau_ambient", 0.5, "tau_ambient"), ("beta", 1.5, "beta"), ("rho0_ink", 0.0, "reference"),
    ("path", 5, "path"),
])
def test_create_rejects_bad_config(L, field, value, msg):
    cfg = _cfg(**{field: value})
    h = C.c_void_p()
    st = L.lbm_create(C.byref(cfg), C.byref(h))
    assert st == lbm.LBM_EINVAL
    assert not h.value
    assert msg in L.lbm_last_error(None).decode()


def test_create_rejects_planar_lattice_with_depth(L):
    cfg = lbm.make_config((8, 2, 8), dict(velset=lbm.LBM_D2Q9))
    h = C.c_void_p()
    assert L.lbm_create(C.byref(cfg), C.byref(h)) == lbm.LBM_EINVAL
    cfg = lbm.make_config((8, 8, 8), dict(velset=lbm.LBM_D2Q9), path="fused")
    assert L.lbm_create(C.byref(cfg), C.byref(h)) == lbm.LBM_EINVAL


def test_calls_on_null_handle(L):
    assert L.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert L.lbm_sync(None, 0) == lbm.LBM_EINVAL
    L.lbm_destroy(None)  # accepted
    assert L.lbm_kernel_launches(None) == 0


def test_python_wrapper_raises_with_message(L):
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(_cfg(nz=0))
    assert e.value.status == lbm.LBM_EINVAL


def _noalloc(L, cfg, geom=None, rheo=None):
    g = lbm.make_geometry(dict(dict(head_pos=(4.0, 4.0), gap=3, r_inner=1.5), **(geom or {})))
    r = lbm.make_rheology(rheo)
    return L.lbm_step_noalloc(C.byref(cfg), C.byref(g), C.byref(r), 1, C.c_void_p(1 << 20), C.c_void_p(1 << 30),
                              None, None)


@pytest.mark.parametrize("geom,rheo,msg", [
    (dict(head_pos=(float("nan"), 4.0)), None, "head position"),
    (dict(head_vel=(0.6, 0.0)), None, "head position"),
    (dict(u_ink=float("inf")), None, "u_ink"),
    (dict(r_inner=1500.0, wall_thickness=600.0), None, "radii"),
    (dict(rho_top_amb=0.0), None, "rho_top_amb"),
    (dict(top_vel=(float("nan"), 0.0, 0.0)), None, "top_vel"),
    (None, dict(law=lbm.LBM_POWER_LAW, K=0.0), "power law"),
    (None, dict(law=lbm.LBM_CROSS, lam=0.0), "Cross"),
    (None, dict(law=lbm.LBM_NEWTONIAN, nu0=float("nan")), "nu0"),
    (None, dict(tau_min=0.5), "tau_min"),
    (None, dict(law=9), "unknown law"),
])
def test_step_noalloc_checks_like_the_handle_calls(L, geom, rheo, msg):
    """lbm_step_noalloc applies the checks of lbm_create, lbm_set_geometry and
    lbm_set_ink_rheology, on the host, before any device work."""
    assert _noalloc(L, _cfg(), geom, rheo) == lbm.LBM_EINVAL
    assert msg in L.lbm_last_error(None).decode()


def test_nozzle_lattice_width_limit(L):
    """The fixed-point nozzle geometry squares half a lattice side in 64-bit
    integers: nozzle runs are limited to nx, ny <= 4000."""
    assert _noalloc(L, _cfg(shape=(4001, 8, 8))) == lbm.LBM_EINVAL
    assert "4000" in L.lbm_last_error(None).decode()


@pytest.mark.parametrize("field,value", [("drag_gamma", float("nan")), ("zeta_ink", float("inf")),
                                         ("A", float("nan")), ("rho0_amb", float("inf"))])
def test_create_rejects_non_finite_constants(L, field, value):
    cfg = _cfg(**{field: value})
    h = C.c_void_p()
    assert L.lbm_create(C.byref(cfg), C.byref(h)) == lbm.LBM_EINVAL
    cfg = _cfg()
    cfg.body_force[1] = float("nan")
    assert L.lbm_create(C.byref(cfg), C.byref(h)) == lbm.LBM_EINVAL
