"""Batched lattices on the GPU: many lattices of uneven size and parameters in
one persistent, graph-captured launch per step compute what each computes
alone through lbm_step.

The batched kernels run the same source arithmetic as the single-lattice ones
but are separate compiled kernels, and the compiler may fuse multiply-adds
differently in each: the results agree to rounding (1 ulp per step at most),
so a batch is compared with lone runs at a bar a little above that (the
16-bit bar for 16-bit storage, where a 1-ulp FP32 difference can flip a
16-bit rounding).
Within one compiled kernel the work decomposition (z-planes per column) does
not change a single bit."""
import numpy as np
import pytest

import oracle as O
from paper_2102_02655_gb300 import inputs as I

from test_gpu_parity import TOL, _lbm, assert_close, f32_exact, field_errors

# FP32: lone and batched kernels differ by an ulp here and there (1e-7 after
# tens of steps); the bar sits well below what a site left out of a step
# would cost
BAR = {"f32": 2e-6, "f16dev": 1e-3}
LEDGER_BAR = {"f32": 1e-6, "f16dev": 1e-4}

pytestmark = pytest.mark.gpu


def _sweep(n, seed, storage="f32"):
    """n print runs of uneven size and parameters (a small sweep)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.choice([40, 48, 64, 72, 96]))
        ny = int(rng.choice([24, 32, 40]))
        nz = int(rng.choice([24, 32, 36]))
        r = float(rng.uniform(3.0, 5.0))
        wl = I.print_run((nx, ny, nz), r, int(rng.integers(8, 14)), float(rng.uniform(0.0, 0.02)),
                         float(rng.uniform(0.01, 0.05)), float(rng.uniform(0.3, 1.0)), storage,
                         head_pos=(float(rng.uniform(8, nx - 8)), float(rng.uniform(8, ny - 8))))
        out.append(wl)
    return out


def _make(lbm, wl, seed):
    shape = wl["shape"]
    lat = lbm.Lattice(shape, wl["params"], wl["geom"], wl["rheo"], path="fused")
    rY, rB = I.nozzle_fill(shape, wl["geom"])
    lat.set_fields(rY, I.perturbed_ambient(shape, rB, seed=seed))
    return lat


def _fields(lat):
    f = lat.fields()
    return {k: np.asarray(v).copy() for k, v in f.items() if k != "diag"}, f["diag"]


def _assert_same(a, b, label):
    """bit for bit (fields and, up to the order of the atomic sums, ledger)"""
    for k in a[0]:
        assert np.array_equal(a[0][k], b[0][k]), (label, k, float(np.abs(a[0][k] - b[0][k]).max()))
    for k in ("mass", "momentum", "bc_flux", "created", "destroyed"):
        assert np.allclose(a[1][k], b[1][k], rtol=1e-12, atol=1e-12), (label, k)
    assert a[1]["step"] == b[1]["step"]


def _assert_close(a, b, label, storage="f32", bar=BAR):
    """the batch against a lone run: the storage's parity bar"""
    e = field_errors(a[0], b[0], ("rho_ink", "rho_amb", "ux", "uy", "uz", "p", "rhoN"))
    bad = {k: v for k, v in e.items() if not v <= bar[storage]}
    assert not bad, (label, bad)
    assert np.array_equal(a[0]["solid"], b[0]["solid"]), label
    # ledger terms on the mass scale (small differences of large sums)
    scale = sum(abs(v) for v in b[1]["mass"])
    for k in ("mass", "bc_flux", "created", "destroyed"):
        d = max(abs(x - y) for x, y in zip(a[1][k], b[1][k]))
        assert d <= LEDGER_BAR[storage] * scale, (label, k, a[1][k], b[1][k])
    assert a[1]["step"] == b[1]["step"] and a[1]["unstable"] == 0


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_batch_equals_lone_runs(storage):
    lbm = _lbm()
    wls = _sweep(5, seed=11, storage=storage)
    steps = 37  # two full graphs of 16 steps and a remainder
    lone = []
    for k, wl in enumerate(wls):
        lat = _make(lbm, wl, seed=k)
        lat.step(steps)
        lone.append(_fields(lat))
        lat.close()
    lats = [_make(lbm, wl, seed=k) for k, wl in enumerate(wls)]
    batch = lbm.Batch(lats)
    batch.step(20)
    batch.step(steps - 20)
    for k, lat in enumerate(lats):
        _assert_close(_fields(lat), lone[k], "lattice %d" % k, storage)
    info = batch.info()
    assert info["steps"] == steps and info["n_lattices"] == 5
    assert info["launches"] == 6 * steps  # column flags, four box phases, bulk
    batch.close()
    for lat in lats:
        lat.close()


def test_zchunk_plan_is_bitwise_invariant():
    lbm = _lbm()
    wls = _sweep(3, seed=8)
    got = []
    for zc in ([16, 16, 16], [5, 9, 40]):
        lats = [_make(lbm, wl, seed=k) for k, wl in enumerate(wls)]
        batch = lbm.Batch(lats)
        batch.set_plan(0, zc)
        batch.step(21)
        got.append([_fields(lat) for lat in lats])
        batch.close()
        for lat in lats:
            lat.close()
    for k in range(len(wls)):
        _assert_same(got[0][k], got[1][k], "lattice %d" % k)


def test_plan_and_autotune_keep_results():
    lbm = _lbm()
    wls = _sweep(3, seed=5)
    lats = [_make(lbm, wl, seed=k) for k, wl in enumerate(wls)]
    batch = lbm.Batch(lats)
    batch.set_plan(0, [7, 5, 40])  # uneven z-chunks
    batch.step(9)
    tune = batch.autotune(trial_steps=2)
    assert tune["variant"] == 0 and tune["zchunk"] >= 1
    assert len(tune["tried"]) >= 4 and all(ms > 0 for _, _, ms in tune["tried"])
    total = batch.info()["steps"]
    batch.step(5)
    total += 5
    got = [_fields(lat) for lat in lats]
    batch.close()
    for lat in lats:
        lat.close()
    for k, wl in enumerate(wls):
        lat = _make(lbm, wl, seed=k)
        lat.step(total)
        _assert_close(got[k], _fields(lat), "lattice %d" % k)
        lat.close()


def test_lattice_steps_alone_between_batch_steps():
    """lbm_step on a member between batch steps is ordered with the batch."""
    lbm = _lbm()
    wls = _sweep(2, seed=3)
    lats = [_make(lbm, wl, seed=k) for k, wl in enumerate(wls)]
    batch = lbm.Batch(lats)
    batch.step(4)
    lats[0].step(3)
    batch.step(4)
    got = [_fields(lat) for lat in lats]
    batch.close()
    for lat in lats:
        lat.close()
    for k, (wl, n) in enumerate(zip(wls, (11, 8))):
        lat = _make(lbm, wl, seed=k)
        lat.step(n)
        _assert_close(got[k], _fields(lat), "lattice %d" % k)
        lat.close()


def test_batch_members_against_oracle():
    """Members of a batch (FP32, uneven sizes and parameters) after 120 steps
    against the FP64 oracle at the FP32 parity bar, 1e-5."""
    lbm = _lbm()
    wls = _sweep(3, seed=17)
    inits = []
    lats = []
    for k, wl in enumerate(wls):
        rY, rB = I.nozzle_fill(wl["shape"], wl["geom"])
        init = f32_exact(rY, I.perturbed_ambient(wl["shape"], rB, seed=k))
        lat = lbm.Lattice(wl["shape"], wl["params"], wl["geom"], wl["rheo"], path="fused")
        lat.set_fields(*init)
        inits.append(init)
        lats.append(lat)
    batch = lbm.Batch(lats)
    batch.step(120)
    got = [lat.fields() for lat in lats]
    batch.close()
    for lat in lats:
        lat.close()
    for k, wl in enumerate(wls):
        ref = O.Oracle(wl["shape"], params=wl["params"], geom=wl["geom"], rheo=wl["rheo"])
        ref.set_fields(*inits[k])
        ref.step(120)
        assert_close(got[k], ref.fields(), TOL["f32"], label="batch member %d vs oracle" % k)
