"""Host logic of the batched step, no GPU: the persistent kernel's work list
covers every site column and plane of every lattice exactly once, and the
batch entry points reject invalid arguments before any device work."""
import ctypes as C

import numpy as np
import pytest

from paper_2102_02655_gb300 import lbm


@pytest.fixture(scope="module")
def L():
    from paper_2102_02655_gb300 import build
    build.build()
    return lbm.lib()


@pytest.mark.parametrize("tile_h", [8, 16])
def test_work_list_covers_each_site_once(L, tile_h):
    rng = np.random.default_rng(7)
    dims = [(int(rng.integers(1, 140)), int(rng.integers(1, 70)), int(rng.integers(1, 50))) for _ in range(7)]
    dims += [(96, 96, 96), (256, 96, 96), (32, 8, 1)]
    zc = [int(rng.integers(1, 40)) for _ in dims]
    items = lbm.lbm_batch_plan(dims, tile_h, zc)
    cover = [np.zeros((nz, ny, nx), dtype=np.int32) for nx, ny, nz in dims]
    for l, x0, y0, za, zb in items:
        nx, ny, nz = dims[l]
        assert x0 % 32 == 0 and y0 % tile_h == 0 and 0 <= za < zb <= nz
        assert zb - za <= zc[l]
        cover[l][za:zb, y0:y0 + tile_h, x0:x0 + 32] += 1
    for c in cover:
        assert np.all(c == 1)
    # each column's planes in ceil(nz / zchunk) chunks of near-equal length
    for l, (nx, ny, nz) in enumerate(dims):
        lens = [zb - za for m, x0, y0, za, zb in items if m == l and x0 == 0 and y0 == 0]
        assert len(lens) == -(-nz // zc[l]) and max(lens) - min(lens) <= 1
    # lattice-major order: the items of one lattice are contiguous
    ls = [it[0] for it in items]
    assert ls == sorted(ls)


def test_work_list_rejects_bad_sizes(L):
    d = (C.c_int * 3)(0, 8, 8)
    z = (C.c_int * 1)(4)
    assert L.lbm_batch_plan(d, 1, 8, z, None, 0) == -1
    d = (C.c_int * 3)(70000, 8, 8)
    assert L.lbm_batch_plan(d, 1, 8, z, None, 0) == -1
    d = (C.c_int * 3)(64, 8, 8)
    assert L.lbm_batch_plan(d, 1, 0, z, None, 0) == -1


def test_batch_create_rejects_bad_arguments(L):
    b = C.c_void_p()
    assert L.lbm_batch_create(None, 0, C.byref(b)) == lbm.LBM_EINVAL
    arr = (C.c_void_p * 2)(None, None)
    assert L.lbm_batch_create(arr, 2, C.byref(b)) == lbm.LBM_EINVAL
    assert "NULL" in L.lbm_batch_last_error(None).decode()
    assert L.lbm_batch_step(None, 1) == lbm.LBM_EINVAL
    L.lbm_batch_destroy(None)
