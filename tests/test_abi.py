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
