"""Serving on the GPU: requests admitted as memory and slots free up, advanced
together (continuous batching), each result the same as the request computed
alone, within the storage's parity bar (batched and single-lattice kernels
agree to rounding)."""
import numpy as np
import pytest

import oracle as O
from paper_2102_02655_gb300 import inputs as I

from test_gpu_parity import _lbm, field_errors

pytestmark = pytest.mark.gpu

BAR = {"f32": 1e-5, "f16dev": 1e-3}


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        shape = (int(rng.choice([48, 64, 80])), int(rng.choice([24, 32])), int(rng.choice([24, 32])))
        wl = I.print_run(shape, float(rng.uniform(3.0, 5.0)), int(rng.integers(8, 13)), float(rng.uniform(0.0, 0.02)),
                         float(rng.uniform(0.01, 0.05)), float(rng.uniform(0.3, 1.0)), "f32",
                         head_pos=(shape[0] / 4.0, shape[1] / 2.0))
        out.append((wl, int(rng.integers(20, 90))))
    return out


def _alone(lbm, wl, steps, storage):
    lat = lbm.Lattice(wl["shape"], dict(wl["params"], storage=storage), wl["geom"], wl["rheo"], path="fused")
    lat.step(steps)
    f = lat.fields()
    lat.close()
    return f


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_same_result_alone_and_in_the_mix(storage):
    lbm = _lbm()
    reqs = _requests(7, seed=21)
    srv = lbm.Server(hbm_budget=8 << 30, storage=storage, quantum=16, max_active=3)
    ids = []
    for k, (wl, steps) in enumerate(reqs):
        ids.append(srv.submit(wl["shape"], wl["params"], wl["geom"], wl["rheo"], steps))
        if k % 2 == 1:
            srv.poll()  # later requests arrive while earlier ones run
    results = {}
    for _ in range(1000):
        srv.poll()
        for rid in srv.finished():
            results[rid] = srv.result(rid)
        if len(results) == len(ids):
            break
    st = srv.stats()
    srv.close()
    assert len(results) == len(ids)
    assert st["peak_active"] <= 3 and st["batch_rebuilds"] >= 3
    for rid, (wl, steps) in zip(ids, reqs):
        status, fg, diag, timing = results[rid]
        assert status == 0 and diag["unstable"] == 0
        assert timing["steps"] == steps and timing["t_submit"] <= timing["t_admit"] <= timing["t_done"]
        fo = _alone(lbm, wl, steps, storage)
        e = field_errors(fg, fo, ("rho_ink", "rho_amb", "ux", "uy", "uz"))
        assert max(e.values()) <= BAR[storage], (rid, e)
        assert diag["step"] == steps
        assert np.allclose(diag["mass"], fo["diag"]["mass"], rtol=BAR[storage])


def test_budget_limits_the_active_set():
    lbm = _lbm()
    reqs = [(I.print_run((64, 32, 32), 4.0, 10, 0.01, 0.02, 0.6, "f32", head_pos=(16.0, 16.0)), 40 + 10 * k)
            for k in range(5)]
    # room for two requests at a time
    big = max(lbm.lattice_bytes(wl["shape"], dict(wl["params"], storage="f32")) for wl, _ in reqs)
    srv = lbm.Server(hbm_budget=2 * big + 1, storage="f32", quantum=32, max_active=8)
    for wl, steps in reqs:
        srv.submit(wl["shape"], wl["params"], wl["geom"], wl["rheo"], steps)
    # and one that can never fit
    huge = srv.submit((512, 256, 256), reqs[0][0]["params"], dict(reqs[0][0]["geom"], gap=20), reqs[0][0]["rheo"], 5)
    peak_bytes = 0
    done = {}
    for _ in range(1000):
        srv.poll()
        peak_bytes = max(peak_bytes, srv.stats()["bytes_in_use"])
        for rid in srv.finished():
            done[rid] = srv.result(rid, fields=False)[0]
        if len(done) == len(reqs) + 1:
            break
    st = srv.stats()
    srv.close()
    assert len(done) == len(reqs) + 1
    assert done[huge] == lbm.LBM_ENOMEM
    assert all(v == 0 for k, v in done.items() if k != huge)
    assert peak_bytes <= 2 * big + 1 and st["peak_active"] <= 2


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_served_requests_against_oracle(storage):
    """Requests served together (continuous batching, arrivals interleaved
    with rounds) against the FP64 oracle after 100-150 steps each, at the
    storage's stated bar: 1e-5 (FP32), 1e-3 (FP16 deviations)."""
    lbm = _lbm()
    rng = np.random.default_rng(31)
    reqs = []
    for _ in range(3):
        shape = (int(rng.choice([48, 64])), 32, 32)
        wl = I.print_run(shape, float(rng.uniform(3.0, 5.0)), 10, float(rng.uniform(0.005, 0.02)),
                         float(rng.uniform(0.02, 0.05)), float(rng.uniform(0.4, 0.8)), storage,
                         head_pos=(shape[0] / 4.0, shape[1] / 2.0))
        reqs.append((wl, int(rng.integers(100, 151))))
    srv = lbm.Server(hbm_budget=8 << 30, storage=storage, quantum=40, max_active=2)
    ids = []
    for k, (wl, steps) in enumerate(reqs):
        ids.append(srv.submit(wl["shape"], wl["params"], wl["geom"], wl["rheo"], steps))
        srv.poll()
    results = {}
    for _ in range(1000):
        srv.poll()
        for rid in srv.finished():
            results[rid] = srv.result(rid)
        if len(results) == len(ids):
            break
    srv.close()
    assert len(results) == len(ids)
    for rid, (wl, steps) in zip(ids, reqs):
        status, fg, diag, _ = results[rid]
        assert status == 0 and diag["unstable"] == 0
        ref = O.Oracle(wl["shape"], params=wl["params"], geom=wl["geom"], rheo=wl["rheo"])
        ref.step(steps)
        e = field_errors(fg, ref.fields(), ("rho_ink", "rho_amb", "ux", "uy", "uz"))
        assert max(e.values()) <= BAR[storage], (rid, storage, e)
