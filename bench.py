"""Throughput benchmark of the two-component colour-gradient LB step on GB300.

One step = one pass of the whole hot path (streaming with boundary rules,
node flips, moments, wall densities, colour gradient, local relaxation time,
regularised collision, perturbation, recolouring) over the synthetic print
lattice 512x128x128 (8.4M sites, D3Q19, FP32 storage and arithmetic), inputs
resident in HBM. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent lattice per rank (replicas; the method has no
exchange step between lattices), launched with torch.distributed.run.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-component MLUPS & %HBM roofline; sweep sims/h, p50/p99 vs plain at same err"
WORKLOAD = "print_512x128x128"
REF_SAMPLE = "print_128x64x64"
# read + write of the populations; 16-bit storage adds the FP32 ink fraction
# per site (read and written once per site)
BYTES_PER_SITE = {"f32": 2 * 19 * 2 * 4, "f64": 2 * 19 * 2 * 8, "f16dev": 2 * 19 * 2 * 2 + 8,
                  "bf16dev": 2 * 19 * 2 * 2 + 8}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Replica bookkeeping for N > 1 (one independent lattice per rank, no
# data-path collective): a barrier around the timed region, the slowest
# rank's time, and the whole-job rate over every rank's sites.

def replica_barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_max(v, ws, device):
    """Maximum of a per-rank float over all ranks (the slowest rank's time)."""
    if ws == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(ws, sites_per_rank, steps, ms):
    """Whole-job site updates per second (millions) when each of ws ranks
    advances its own lattice of sites_per_rank sites by steps steps and the
    slowest rank took ms milliseconds."""
    return ws * sites_per_rank * steps / (ms * 1e-3) / 1e6


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _fused_source_sha():
    """Key of the committed ncu traffic figure: every source of the FP32 fused
    kernel's translation unit and its build flags."""
    from paper_2102_02655_gb300 import build
    h = hashlib.sha256()
    for f in ("lbm_fused_f32.cu", "lbm_fused_impl.cuh", "lbm_launch.h", "lbm_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2102_02655_gb300", "csrc", f), "rb").read())
    h.update(" ".join(build.ARCH + build.FLAGS[:6] + build.FILE_FLAGS["lbm_fused_f32.cu"]).encode())
    return h.hexdigest()[:16]


def _traffic_per_site():
    """DRAM bytes per site update of the fused kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_fused_print_traffic.json")) as f:
            d = json.load(f)
        if d.get("kernel_sha") == _fused_source_sha():
            return float(d["dram_bytes_per_site"])
    except Exception:
        pass
    return None


def oracle_mlups(name, steps, threads=None):
    """Time the FP64 CPU oracle as it stands on `steps` steps of a workload."""
    import oracle as O
    from paper_2102_02655_gb300 import inputs as I
    wl = I.workload(name)
    shape = wl["shape"]
    ref = O.Oracle(shape, params=dict(wl["params"], storage="f64"), geom=wl["geom"], rheo=wl["rheo"])
    rY, rB = I.nozzle_fill(shape, wl["geom"])
    ref.set_fields(rY, I.perturbed_ambient(shape, rB, seed=0))
    ref.step(1)  # warm-up
    t0 = time.perf_counter()
    ref.step(steps)
    dt = time.perf_counter() - t0
    n = shape[0] * shape[1] * shape[2]
    return n * steps / dt / 1e6, dt, n


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from paper_2102_02655_gb300 import inputs as I
    shape = I.workload(REF_SAMPLE)["shape"]
    n = shape[0] * shape[1] * shape[2]
    if args.warmup:
        oracle_mlups(REF_SAMPLE, args.warmup)
    mlups, dt, _ = oracle_mlups(REF_SAMPLE, args.steps)
    cores = O.threads_used()
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "D3Q19", "sites": 512 * 128 * 128},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "%s (%d sites, same print parameters), %d steps per timed run"
                                       % (REF_SAMPLE, n, args.steps)},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_2102_02655_gb300 import build, inputs as I, lbm

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    wl = I.workload(args.workload)
    if args.storage:
        wl["params"]["storage"] = args.storage
    shape = wl["shape"]
    nsites = shape[0] * shape[1] * shape[2]
    storage = wl["params"]["storage"]
    rY, rB = I.nozzle_fill(shape, wl["geom"])
    rB = I.perturbed_ambient(shape, rB, seed=rank)
    lat = lbm.Lattice(shape, wl["params"], wl["geom"], wl["rheo"], path="fused", device=local)
    lat.set_fields(rY, rB)
    stream = lat.stream

    def barrier():
        replica_barrier(ws)

    def max_over_ranks(v):
        return replica_max(v, ws, "cuda")

    # untimed spin-up: the extruded ink thread forms before anything is
    # timed (a step costs more once ink has left the nozzle), then warm-up
    lat.step(args.spinup)
    lat.step(args.warmup)
    torch.cuda.synchronize()

    # timed region: device-resident inputs, K steps, CUDA events on the stream
    lat.profile(True)
    launches0 = lat.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = lat.kernel_launches() - launches0
    tm = lat.timings()
    lat.profile(False)
    ms = max_over_ranks(ms)
    value = aggregate_mlups(ws, nsites, args.steps, ms)

    # roofline of the dominant kernel (fused bulk kernel)
    peak, peak_kind = _peaks()
    bulk_ms_launch = tm["bulk_ms"] / max(1, tm["bulk_launches"])
    bulk_sites_launch = tm["bulk_sites"] / max(1, tm["bulk_launches"])
    bps = BYTES_PER_SITE[storage]
    achieved = bps * bulk_sites_launch / (bulk_ms_launch * 1e-3) / 1e9
    tps = _traffic_per_site()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": tps * bulk_sites_launch if tps is not None else None,
            "kernel": "k_fused", "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": bps * bulk_sites_launch,
            "kernel_ms_per_launch": bulk_ms_launch,
            # the bulk kernel's own duration over the step's wall time (the
            # nozzle-box kernels run beside it on a second stream)
            "kernel_share_of_step": bulk_ms_launch / (ms / args.steps),
            "box_kernels_ms_per_step": tm["plain_ms"] / max(1, tm["plain_groups"])}

    # optional: MLUPS over a long run, in windows, from the fresh nozzle fill
    trace = None
    if args.mlups_trace > 0:
        trace = run_trace(args, wl, rY, rB, lat)

    # config 2's range of ink laws (n = 0.4, 0.6, 0.8), each from its own
    # spun-up state, same lattice and timing
    points = None
    if not args.no_points:
        points = run_points(args, wl, rY, rB, local, lat)

    # end to end through the C ABI with pinned host buffers: upload the
    # initial fields, K steps, read back densities, velocity and diagnostics
    esz = 8 if storage == "f64" else 4
    e2e, unstable = None, 0
    if not args.no_e2e:
        e2e, unstable = run_e2e(lat, rY, rB, storage, nsites, args, barrier, max_over_ranks, ws)
    sweep = None
    if rank == 0 and not args.no_sweep:
        lat.close()
        lat = None
        torch.cuda.empty_cache()
        with Clocks(local) as clk_w:
            sweep = run_sweep(args, local)
        sweep["clocks"] = clk_w.summary()
    serving = None
    if rank == 0 and not args.no_serve:
        if lat is not None:
            lat.close()
            lat = None
        torch.cuda.empty_cache()
        with Clocks(local) as clk_s:
            serving = run_serving(args, local)
        serving["clocks"] = clk_s.summary()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        cs = max(1, args.cpu_steps)
        mlups, dt, n = oracle_mlups(args.workload, cs)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": O.threads_used(), "kind": "oracle",
               "sample": "%s full lattice (%d sites), %d steps after 1 untimed, %.1f s" % (args.workload, n, cs, dt)}

    if lat is not None:
        lat.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if storage == "f64" else "f32", "data": "synthetic",
                "config": {"workload": args.workload, "lattice": "D3Q19", "sites": nsites, "storage": storage,
                           "path": "fused bulk kernel + phase-by-phase nozzle box",
                           "nozzle": "r 10, gap 20, head 0.01 l.u./step, power-law n 0.6, extrusion 0.02",
                           "l2": "inputs larger than L2 (populations %.2f GB)" % (BYTES_PER_SITE[storage] * nsites / 1e9),
                           "spinup_steps": args.spinup,
                           "parallelism": "replicas" if ws > 1 else "single"},
                "ink_law_points": points,
                "mlups_trace": trace,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "unstable": unstable, "sweep": sweep,
                "serving": serving}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_trace(args, wl, rY, rB, lat0, window=500):
    """MLUPS of each window of `window` steps over args.mlups_trace steps from
    the seeded initial state (how a step's cost changes as the ink thread
    grows)."""
    import torch
    shape = wl["shape"]
    nsites = shape[0] * shape[1] * shape[2]
    lat0.set_geometry(wl["geom"])
    lat0.set_fields(rY, rB)
    out = []
    done = 0
    while done < args.mlups_trace:
        n = min(window, args.mlups_trace - done)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(lat0.stream)
        lat0.step(n)
        ev1.record(lat0.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / n
        done += n
        out.append({"steps": done, "ms_per_step": ms, "mlups": nsites / (ms * 1e-3) / 1e6})
    out[-1]["unstable"] = lat0.diag()["unstable"]
    lat0.set_geometry(wl["geom"])
    lat0.set_fields(rY, rB)
    return out


def run_points(args, wl, rY, rB, device, lat0):
    """MLUPS of the throughput lattice for power-law indices n = 0.4, 0.6, 0.8
    (config 2's range; extrusion 0.02, head 0.01 l.u./step), each timed over
    args.point_steps steps after the same spin-up as the headline."""
    import torch
    from paper_2102_02655_gb300 import lbm
    shape = wl["shape"]
    nsites = shape[0] * shape[1] * shape[2]
    out = []
    for n in (0.4, 0.6, 0.8):
        lat0.set_geometry(wl["geom"])
        lat0.set_rheology(dict(wl["rheo"], n=n))
        lat0.set_fields(rY, rB)
        lat0.step(args.spinup + args.warmup)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(lat0.stream)
        lat0.step(args.point_steps)
        ev1.record(lat0.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.point_steps
        out.append({"n": n, "ms_per_step": ms, "mlups": nsites / (ms * 1e-3) / 1e6,
                    "unstable": lat0.diag()["unstable"]})
    lat0.set_geometry(wl["geom"])
    lat0.set_rheology(wl["rheo"])
    lat0.set_fields(rY, rB)
    return out


def sweep_workloads(n=64, seed=2024):
    """The batched parameter sweep: n print runs from 96^3 to 256x96x96, nozzle
    radius 4-12, power-law n in [0.3, 1.0], extrusion 0.01-0.05, head speed
    0-0.02 l.u./step, drawn from the seed (FP32)."""
    import numpy as np
    from paper_2102_02655_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.choice([96, 128, 160, 192, 224, 256]))
        shape = (nx, 96, 96)
        out.append(I.print_run(shape, float(rng.uniform(4.0, 12.0)), 20, float(rng.uniform(0.0, 0.02)),
                               float(rng.uniform(0.01, 0.05)), float(rng.uniform(0.3, 1.0)), "f32",
                               head_pos=(nx / 4.0, 48.0)))
    return out


def run_sweep(args, device):
    """Batched sweep vs the plain one-lattice-at-a-time form on the same
    lattices, each form timed from the same seeded initial state (the cost of a
    step grows as the extruded ink accumulates): whole-sweep MLUPS and
    simulations per hour at 10k steps each."""
    import torch
    from paper_2102_02655_gb300 import inputs as I, lbm
    wls = sweep_workloads(args.sweep_n)
    lats = []
    for wl in wls:
        lats.append(lbm.Lattice(wl["shape"], wl["params"], wl["geom"], wl["rheo"], path="fused", device=device))

    def reset():
        # geometry (step counter back to 0) and the seeded fields of each lattice
        for k, (lat, wl) in enumerate(zip(lats, wls)):
            lat.set_geometry(wl["geom"])
            rY, rB = I.nozzle_fill(wl["shape"], wl["geom"])
            lat.set_fields(rY, I.perturbed_ambient(wl["shape"], rB, seed=k))
        torch.cuda.synchronize()

    sites = sum(w["shape"][0] * w["shape"][1] * w["shape"][2] for w in wls)
    K = args.sweep_steps
    S = args.sweep_spinup
    # autotuned plan; the batch also runs the untimed spin-up of both forms
    # (the same state to rounding), so that both are timed past the fresh
    # nozzle fill, where a step is cheaper
    batch = lbm.Batch(lats)
    tune = batch.autotune(trial_steps=4)
    # plain form: one lattice after another, each K steps on its own stream
    reset()
    batch.step(1 + S)
    batch.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for lat in lats:
        lat.step(K)
        lat.stream.synchronize()
    t_plain = time.perf_counter() - t0
    # batched form: graphs of this call's sizes captured first, then K steps
    # from the same spun-up state
    reset()
    batch.step(1 + S)
    batch.step(K)
    batch.sync()
    reset()
    batch.step(1 + S)
    batch.sync()
    t0 = time.perf_counter()
    batch.step(K)
    batch.sync()
    t_batch = time.perf_counter() - t0
    info = batch.info()
    bad = sum(lat.diag()["unstable"] for lat in lats)
    batch.close()
    for lat in lats:
        lat.close()
    steps_per_sim = 10000
    return {"lattices": len(wls), "sites": sites, "steps_timed": K,
            "plain_mlups": sites * K / t_plain / 1e6, "batched_mlups": sites * K / t_batch / 1e6,
            "speedup": t_plain / t_batch,
            "plain_sims_per_hour": len(wls) * 3600.0 / (t_plain / K * steps_per_sim),
            "batched_sims_per_hour": len(wls) * 3600.0 / (t_batch / K * steps_per_sim),
            "sims_per_hour_note": "10k-step simulations; plain = one after another, batched = all together",
            "autotune": {"variant": tune["variant"], "zchunk": tune["zchunk"], "ctas_per_sm": tune["ctas_per_sm"],
                         "ms_per_step": tune["ms_per_step"], "candidates": len(tune["tried"])},
            "graph_steps": info["steps_per_graph"], "work_items": info["n_items"], "grid": info["grid"],
            "unstable": bad,
            "spinup_steps": S,
            "what": "64 print runs 96^3..256x96x96 (seeded parameters), wall time of K steps after the same "
                    "untimed spin-up for each form, host-synchronised"}


def serve_requests(n, steps_max, seed=5):
    """Print-run requests shaped like the downscaled runs: 96x48x48 to 128x64x64,
    nozzle radius 4-10, power-law n in [0.4, 0.8], extrusion 0.02-0.05, head
    speed 0.005-0.02 l.u./step, steps uniform in [steps_max / 20, steps_max]."""
    import numpy as np
    from paper_2102_02655_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.choice([96, 112, 128]))
        shape = (nx, nx // 2, nx // 2)
        wl = I.print_run(shape, float(rng.uniform(4.0, 10.0)), 16, float(rng.uniform(0.005, 0.02)),
                         float(rng.uniform(0.02, 0.05)), float(rng.uniform(0.4, 0.8)), "f16dev",
                         head_pos=(nx / 4.0, nx / 4.0))
        out.append((wl, int(rng.integers(max(1, steps_max // 20), steps_max + 1))))
    return out


def run_serving(args, device):
    """Poisson arrivals (mean rate args.serve_rate per s) of print-run
    requests, FP16-deviation storage. Continuous batching (lbm_server_*,
    admission against an HBM budget) vs the serial plain path (each request
    alone through lbm_create + lbm_step, first come first served), on the same
    arrival times: latency from arrival to result on the host, p50/p99, and
    simulations per hour over the makespan."""
    import numpy as np
    import torch
    from paper_2102_02655_gb300 import lbm
    reqs = serve_requests(args.serve_n, args.serve_steps)
    rng = np.random.default_rng(11)
    arrive = np.cumsum(rng.exponential(1.0 / args.serve_rate, len(reqs)))
    arrive -= arrive[0]
    work = sum(wl["shape"][0] * wl["shape"][1] * wl["shape"][2] * s for wl, s in reqs)

    # continuous batching
    srv = lbm.Server(hbm_budget=int(args.serve_budget_gb * 1e9), storage="f16dev", quantum=args.serve_quantum,
                     max_active=args.serve_max_active, device=device)
    lat_b = {}
    ids = {}
    nxt = 0
    t0 = time.perf_counter()
    while len(lat_b) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrive[nxt] <= now:
            wl, steps = reqs[nxt]
            ids[srv.submit(wl["shape"], wl["params"], wl["geom"], wl["rheo"], steps)] = nxt
            nxt += 1
        st = srv.stats()
        if st["waiting"] + st["active"] == 0:
            time.sleep(max(0.0, min(0.01, arrive[nxt] - now)) if nxt < len(reqs) else 0.0)
            continue
        srv.poll()
        for rid in srv.finished():
            status, _, diag, _ = srv.result(rid, fields=False)
            k = ids[rid]
            lat_b[k] = (time.perf_counter() - t0 - arrive[k], status, diag["unstable"])
    make_b = time.perf_counter() - t0
    sst = srv.stats()
    srv.close()
    torch.cuda.synchronize()

    # serial plain path on the same arrival times
    lat_s = {}
    t0 = time.perf_counter()
    for k, (wl, steps) in enumerate(reqs):
        now = time.perf_counter() - t0
        if arrive[k] > now:
            time.sleep(arrive[k] - now)
        lat = lbm.Lattice(wl["shape"], wl["params"], wl["geom"], wl["rheo"], path="fused", device=device)
        lat.step(steps)
        d = lat.diag()
        lat.close()
        lat_s[k] = (time.perf_counter() - t0 - arrive[k], 0, d["unstable"])
    make_s = time.perf_counter() - t0

    def pct(d, q):
        return float(np.percentile([v[0] for v in d.values()], q))
    return {"requests": len(reqs), "steps_range": [max(1, args.serve_steps // 20), args.serve_steps],
            "rate_per_s": args.serve_rate, "storage": "f16dev", "budget_gb": args.serve_budget_gb,
            "batched": {"p50_s": pct(lat_b, 50), "p99_s": pct(lat_b, 99), "makespan_s": make_b,
                        "sims_per_hour": len(reqs) * 3600.0 / make_b, "mlups": work / make_b / 1e6,
                        "peak_active": sst["peak_active"], "rounds": sst["rounds"],
                        "batch_rebuilds": sst["batch_rebuilds"],
                        "failed": sum(1 for v in lat_b.values() if v[1] != 0 or v[2])},
            "serial": {"p50_s": pct(lat_s, 50), "p99_s": pct(lat_s, 99), "makespan_s": make_s,
                       "sims_per_hour": len(reqs) * 3600.0 / make_s, "mlups": work / make_s / 1e6,
                       "failed": sum(1 for v in lat_s.values() if v[2])},
            "what": "latency = arrival to result on the host; sims/hour over the makespan; same requests and "
                    "arrival times for both forms"}


def run_e2e(lat, rY, rB, storage, nsites, args, barrier, max_over_ranks, ws):
    import numpy as np
    import torch
    from paper_2102_02655_gb300 import lbm
    tdt = torch.float64 if storage == "f64" else torch.float32
    # the request's input is the spun-up print state the headline is timed on
    # (its densities and velocity, read back untimed into pinned memory), so
    # that both numbers time the same kind of step
    mask = lbm.LBM_FIELD_RHO_INK | lbm.LBM_FIELD_RHO_AMB | lbm.LBM_FIELD_U
    ins = [torch.empty(rY.shape, dtype=tdt).pin_memory() for _ in range(5)]
    lat.fields(mask=mask, out=[t.numpy() for t in ins])
    h_u = torch.stack(ins[2:5]).pin_memory()
    outs = [torch.empty(rY.shape, dtype=tdt).pin_memory() for _ in range(5)]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.set_fields(ins[0].numpy(), ins[1].numpy(), h_u.numpy())
    ev0.record(lat.stream)
    lat.step(args.steps)
    ev1.record(lat.stream)
    res = lat.fields(mask=lbm.LBM_FIELD_RHO_INK | lbm.LBM_FIELD_RHO_AMB | lbm.LBM_FIELD_U,
                     out=[o.numpy() for o in outs])
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    esz = 8 if storage == "f64" else 4
    e2e = {"value": aggregate_mlups(ws, nsites, args.steps, e2e_s * 1e3), "unit": "MLUPS",
           "h2d_bytes_per_step": 5 * nsites * esz / args.steps,
           "d2h_bytes_per_step": (5 * nsites * esz + 120) / args.steps,
           "what": "per request: pinned H2D of a spun-up state's rho_ink, rho_amb, u; K steps; D2H of rho_ink, "
                   "rho_amb, u, diag",
           # the same request's K steps timed on the device alone: the request
           # restarts from the equilibrium of those fields, whose first steps
           # cost less than the headline's (no non-equilibrium stress yet)
           "request_steps_device_mlups": aggregate_mlups(ws, nsites, args.steps, max_over_ranks(ev0.elapsed_time(ev1)))}
    return e2e, res["diag"]["unstable"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--spinup", type=int, default=2000,
                    help="untimed steps before the warm-up (the ink thread forms)")
    ap.add_argument("--point-steps", type=int, default=100, help="timed steps per ink-law point")
    ap.add_argument("--no-points", action="store_true", help="skip the n = 0.4/0.6/0.8 points")
    ap.add_argument("--mlups-trace", type=int, default=0,
                    help="also time this many steps from the fresh state in windows of 500")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched parameter sweep")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-n", type=int, default=40)
    ap.add_argument("--serve-steps", type=int, default=4000, help="largest step count of a request")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="mean arrivals per second")
    ap.add_argument("--serve-quantum", type=int, default=200)
    ap.add_argument("--serve-max-active", type=int, default=32)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--sweep-n", type=int, default=64)
    ap.add_argument("--sweep-steps", type=int, default=20)
    ap.add_argument("--sweep-spinup", type=int, default=1000, help="untimed sweep steps before timing")
    ap.add_argument("--storage", choices=["f64", "f32", "f16dev", "bf16dev"], default=None,
                    help="population storage (default: the workload's, FP32)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="throughput workload (default: the 512x128x128 print lattice)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
