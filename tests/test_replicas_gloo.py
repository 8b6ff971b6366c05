"""Host logic of the N > 1 benchmark (one independent lattice per rank, no
data-path collective), exercised on CPU with two gloo ranks.

Each rank advances its own seeded lattice; the only cross-rank traffic is the
barrier around the timed region and the maximum of the per-rank times. The
per-rank stepping here uses the CPU oracle, so the test checks that a replica
computes exactly what a lone run with the same seed computes.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (16, 8, 8)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_run(seed, steps=3):
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2102_02655_gb300 import inputs as I
    wl = I.print_run(SHAPE, 2.0, 4, 0.01, 0.02, 0.6, "f64", wall=1.0, head_pos=(4.0, 4.0))
    ref = O.Oracle(SHAPE, params=wl["params"], geom=wl["geom"], rheo=wl["rheo"])
    rY, rB = I.nozzle_fill(SHAPE, wl["geom"])
    ref.set_fields(rY, I.perturbed_ambient(SHAPE, rB, seed=seed))
    ref.step(steps)
    return ref.fields()["rho_amb"], ref.diag()["mass"]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.replica_barrier(ws)
        rho, mass = _replica_run(seed=rank)
        ms_local = [12.5, 20.0][rank]
        ms = bench.replica_max(ms_local, ws, "cpu")
        value = bench.aggregate_mlups(ws, SHAPE[0] * SHAPE[1] * SHAPE[2], 10, ms)
        bench.replica_barrier(ws)
        q.put((rank, ms, value, rho, mass))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=180)
        res[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sites = SHAPE[0] * SHAPE[1] * SHAPE[2]
    for r in range(2):
        ms, value, rho, mass = res[r]
        # the slowest rank's time, and the rate over both ranks' sites
        assert ms == 20.0
        assert value == pytest.approx(2 * sites * 10 / 20.0e-3 / 1e6, rel=0, abs=1e-12)
        # a replica computes exactly what a lone run with its seed computes
        rho1, mass1 = _replica_run(seed=r)
        assert np.array_equal(rho, rho1)
        assert list(mass) == list(mass1)
    # different seeds give different replicas (no accidental sharing)
    assert not np.array_equal(res[0][2], res[1][2])


def test_single_rank_bookkeeping():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(3.5, 1, "cpu") == 3.5
    assert bench.aggregate_mlups(1, 8388608, 200, 1000.0) == pytest.approx(1677.7216, rel=1e-12)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
