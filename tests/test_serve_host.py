"""Serving host logic without a GPU: request validation, queueing, and the
device-byte accounting that admission uses."""
import pytest

from paper_2102_02655_gb300 import inputs as I, lbm


@pytest.fixture(scope="module")
def L():
    from paper_2102_02655_gb300 import build
    build.build()
    return lbm.lib()


def test_lattice_bytes_counts_every_buffer(L):
    wl = I.workload("print_128x64x64")
    n = 128 * 64 * 64
    b32 = lbm.lattice_bytes(wl["shape"], dict(wl["params"], storage="f32"))
    b16 = lbm.lattice_bytes(wl["shape"], dict(wl["params"], storage="f16dev"))
    b64 = lbm.lattice_bytes(wl["shape"], dict(wl["params"], storage="f64"))
    # two population buffers dominate: 2 x 38 x N x (4 | 2 + ink fraction | 8)
    assert b32 >= 2 * 38 * n * 4 and b64 >= 2 * 38 * n * 8
    assert b16 >= 2 * (38 * n * 2 + 4 * n)
    assert b16 < b32 < b64
    # plus densities (with ghost planes), top velocities and the 9 field planes
    extra32 = b32 - 2 * 38 * n * 4
    assert extra32 >= 9 * n * 4 + 2 * 2 * n * 4
    assert lbm.lattice_bytes((0, 4, 4), wl["params"]) == -1


def test_server_queues_and_validates(L):
    s = lbm.Server(hbm_budget=1 << 30, storage="f16dev", quantum=10, max_active=2)
    wl = I.workload("print_128x64x64")
    ids = [s.submit(wl["shape"], wl["params"], wl["geom"], wl["rheo"], 5) for _ in range(3)]
    assert ids == sorted(ids) and len(set(ids)) == 3
    st = s.stats()
    assert st["waiting"] == 3 and st["active"] == 0 and st["finished"] == 0 and st["bytes_in_use"] == 0
    with pytest.raises(lbm.LBMError):
        s.submit(wl["shape"], wl["params"], wl["geom"], wl["rheo"], 0)
    with pytest.raises(lbm.LBMError):
        s.submit(wl["shape"], wl["params"], dict(wl["geom"], z_mode=0), wl["rheo"], 5)
    assert s.finished() == []
    s.close()


def test_server_rejects_bad_config(L):
    with pytest.raises(lbm.LBMError):
        lbm.Server(hbm_budget=0)
    with pytest.raises(lbm.LBMError):
        lbm.Server(hbm_budget=1 << 30, quantum=0)
