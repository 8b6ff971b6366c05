"""Host-side failure handling of the C ABI on a GPU: a device allocator that
fails part-way through lbm_create gives LBM_ENOMEM and gets back every block
it granted; nothing is left allocated and no handle is returned."""
import ctypes as C

import pytest

from paper_2102_02655_gb300 import inputs as I

from test_gpu_parity import _lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fail_at", [0, 1, 4, 9])
def test_create_with_failing_allocator(fail_at):
    import torch
    lbm = _lbm()
    live, granted, freed = {}, [], []

    def alloc(nbytes, ctx):
        if len(granted) == fail_at:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        granted.append(t.data_ptr())
        return t.data_ptr()

    def free(ptr, ctx):
        freed.append(ptr)
        live.pop(ptr, None)

    c_alloc, c_free = lbm.ALLOC_FN(alloc), lbm.FREE_FN(free)
    wl = I.print_run((40, 24, 24), 4.0, 8, 0.01, 0.02, 0.6, "f32")
    cfg = lbm.make_config(wl["shape"], wl["params"])
    cfg.alloc, cfg.free = c_alloc, c_free
    h = C.c_void_p()
    st = lbm.lib().lbm_create(C.byref(cfg), C.byref(h))
    assert st == lbm.LBM_ENOMEM, st
    assert not h.value
    assert "allocation" in lbm.lib().lbm_last_error(None).decode()
    assert len(granted) == fail_at and sorted(freed) == sorted(granted) and not live


def test_create_with_working_allocator_frees_everything_on_destroy():
    import torch
    lbm = _lbm()
    live = {}

    def alloc(nbytes, ctx):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, ctx):
        live.pop(ptr)

    c_alloc, c_free = lbm.ALLOC_FN(alloc), lbm.FREE_FN(free)
    wl = I.print_run((40, 24, 24), 4.0, 8, 0.01, 0.02, 0.6, "f32")
    cfg = lbm.make_config(wl["shape"], wl["params"])
    cfg.alloc, cfg.free = c_alloc, c_free
    h = lbm.lbm_create(cfg)
    n = len(live)
    assert n >= 8
    lbm.lbm_set_ink_rheology(h, lbm.make_rheology(wl["rheo"]))
    lbm.lbm_set_geometry(h, lbm.make_geometry(wl["geom"]))
    lbm.lbm_step(h, 3)
    assert len(live) == n  # steps allocate nothing
    lbm.lbm_destroy(h)
    assert not live
