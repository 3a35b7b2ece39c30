"""Benchmark of the fused multilayer shallow-water LBM step on GB300.

Workload: the three-layer pseudo-3D spinodal film (D2Q9, 1024 x 1024
periodic cells, means 1.0 / 0.8 / 0.6 plus seeded Gaussian noise 1e-3,
gamma 0.01 / 0.008 / 0.006, mu = (1, 2, 4) / 6, slip 1, wetting exponents
(3, 2), h* = 0.07, contact angle 20 degrees), FP32 populations.

A benchmark step is one LBM time step (one fused kernel launch) over the
whole lattice. Metric: layer-site updates per second,
LSU/s = n_layers * nx * ny * steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Own arm: inputs resident in HBM; K back-to-back steps on the solver's
stream, bracketed by CUDA events (one before the first step, then one after
every 50 steps, which also gives the spread). The two population buffers (2 x 113 MB) exceed
the 129 MB L2, so no flush is needed; a step's dirty lines that the L2
still holds when it ends are written back inside the next step, as in a
long run. For context the line also reports single steps with the L2
flushed before each (a 256 MiB write and read): those exclude that
write-back and read lower.
The e2e figure goes through the public API with host buffers: every step
uploads the heights from pinned memory (mlswlbm_set_heights), advances one
step and reads the heights back (mlswlbm_get_heights).

Two more workloads are reported beside the main line, under "workloads"
(rank 0, after the timed region; --no-extra skips them):
  * two-layer pseudo-2D film, D1Q3, 512 cells: time to solution of 10 000
    steps through mlswlbm_step (one persistent launch holds the lattice on
    chip) and heights read back, wall clock;
  * three-layer lens field, D2Q9, 2048 x 2048, lenses of radius 200 (the
    droplet/lens equilibrium workload): LSU/s over event-timed
    back-to-back steps (its 2 x 906 MB working set exceeds the L2), then
    the run until the kinetic energy falls below 1e-12 (at most 500 000
    steps) with the lenses' Neumann angles;
  * batched stability sweep: 512 instances (2..5 layers, sides 64..512,
    ~142 M layer-sites per step) in one batch with the tile-height
    autotuner: LSU/s of the batched step, the time to solution of 2000
    steps with the perturbed mode measured every 200 steps and a growth
    rate fitted per instance, and the same steps run instance by instance
    with one solver each (20 steps per instance, scaled to 2000);
  * analysis on the device, 1024^2 film: radial power spectra of the layers
    and ring means of the interfaces, wall time per call;
  * the U-Net surrogate of 64 LBM steps on the 256^2 three-layer film:
    training on 20 000 solver trajectories, held-out errors against the LBM
    and the identity map, tensor-core throughput, and the time to solution
    of 64 instances judged by the LBM against batched and per-instance LBM.

Reference arm (--impl reference): the FP64 CPU oracle on the host cores, one
oracle step per benchmark step on a 128 x 128 patch with the same recipe.
Under torchrun only rank 0 runs it.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

NX = NY = 1024
N_LAYERS = 3
Q = 9
BYTES_PER_LSU = 2 * Q * 4          # read + write of every FP32 population
METRIC = "layer-site updates/s"
UNIT = "LSU/s"
WORKLOAD = "3-layer D2Q9 spinodal film, 1024x1024 periodic, FP32 populations"
FALLBACK_HBM_GBS = 6800.0
CHUNK = 50                         # timed steps between two events
KERNEL_SOURCES = ["paper_2409_16659_gb300/csrc/step_kernels.cu",
                  "paper_2409_16659_gb300/csrc/d2q9_tile.cuh",
                  "paper_2409_16659_gb300/csrc/physics.cuh",
                  "paper_2409_16659_gb300/csrc/tma.cuh"]


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def config_dict(extra=None):
    c = {"workload": WORKLOAD, "n_layers": N_LAYERS, "lattice": "D2Q9", "nx": NX, "ny": NY,
         "cells": NX * NY, "layer_sites_per_step": N_LAYERS * NX * NY,
         "l2": "inputs larger than L2: back-to-back steps over two 113 MB population "
               "buffers (226 MB > 129 MB L2), no flush",
         "parallelism": "replicas (one independent lattice per GPU)"}
    if extra:
        c.update(extra)
    return c


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (no MEASURED_PEAKS.json)"


def ncu_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == "step_d2q9_film3_1024" \
                and parts[1] == want:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, device):
    """Each value's maximum over the ranks of the default process group (the
    job's time is its slowest rank's); unchanged in a single process."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_rate(world_size, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (every rank runs its own lattice, weak scaling)."""
    return world_size * units_per_rank / seconds


def cpu_model():
    """Host CPU description and core count, from /proc/cpuinfo."""
    model, parts = None, set()
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k == "model name" and not model:
                    model = v
                elif k == "CPU part":
                    parts.add(v)
    except OSError:
        pass
    if not model and parts:
        model = "Arm CPU part " + "/".join(sorted(parts))
    return {"model": model or "unknown", "nproc": os.cpu_count()}


def _oracle_lsu(oracle, side, seconds, threads):
    oracle.set_threads(threads)
    p = workloads.film3_d2q9_params(side, side)
    f = oracle.init(p, workloads.film3_d2q9_heights(side, side).ravel())
    steps, t0 = 0, time.perf_counter()
    while True:
        f = oracle.step(p, f)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return N_LAYERS * side * side * steps / dt, steps, dt


def cpu_oracle_sample(seconds=8.0, side=256):
    """The FP64 oracle on a bounded patch of the same workload recipe, on all
    host cores (OpenMP over the cells) and on one thread."""
    import oracle
    cores = os.cpu_count() or 1
    lsu, steps, dt = _oracle_lsu(oracle, side, seconds, cores)
    lsu1, steps1, dt1 = _oracle_lsu(oracle, side, seconds, 1)
    cpu = cpu_model()
    return {"value": lsu, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "FP64 C oracle, %d OpenMP threads, %d steps on a %dx%d patch of the "
                      "3-layer D2Q9 film (same parameters), %.1f s" % (cores, steps, side, side, dt),
            "single_thread": {"value": lsu1, "unit": UNIT, "cores": 1,
                              "sample": "same, 1 thread, %d steps, %.1f s" % (steps1, dt1)},
            "cpu": cpu}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    side = 128
    p = workloads.film3_d2q9_params(side, side)
    f = oracle.init(p, workloads.film3_d2q9_heights(side, side).ravel())
    for _ in range(args.warmup):
        f = oracle.step(p, f)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.step(p, f)
    dt = time.perf_counter() - t0
    lsu = N_LAYERS * side * side * args.steps / dt
    sample = ("FP64 C oracle, %d OpenMP threads, one oracle step per benchmark step on a "
              "%dx%d patch of the 3-layer D2Q9 film (same parameters)" % (cores, side, side))
    line = {"impl": "reference", "metric": METRIC, "value": lsu, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict({"sample_nx": side, "sample_ny": side}),
            "cpu_baseline": {"value": lsu, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": lsu, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_own(args):
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2409_16659_gb300 import mlswlbm as B

    p = workloads.film3_d2q9_params(NX, NY)
    h0 = workloads.film3_d2q9_heights(NX, NY, seed=2 + rank).astype(np.float32)
    stream = torch.cuda.current_stream()
    solver = B.Solver(p, h0, stream=stream)
    lsu_step = N_LAYERS * NX * NY

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- warm-up ----------------------------------------------------------
    for _ in range(args.warmup):
        solver.step(1)
    torch.cuda.synchronize()

    # ---- timed region: K back-to-back steps ---------------------------------
    # Events only every CHUNK steps: an event recorded between two launches
    # keeps the second from starting while the first drains (programmatic
    # dependent launch), so per-step events would time a slower loop than a
    # long run is. The spread is that of the chunk means.
    chunk = min(CHUNK, args.steps)
    bounds = list(range(0, args.steps, chunk)) + [args.steps]
    evs = [torch.cuda.Event(enable_timing=True) for _ in bounds]
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = solver.launch_count()
    barrier()
    evs[0].record(stream)
    for j in range(1, len(bounds)):
        solver.step(bounds[j] - bounds[j - 1])
        evs[j].record(stream)
    barrier()
    launches = solver.launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    total_s = evs[0].elapsed_time(evs[-1]) / 1e3
    step_ms = np.array([evs[j - 1].elapsed_time(evs[j]) / (bounds[j] - bounds[j - 1])
                        for j in range(1, len(bounds))])

    # ---- context: single steps from a flushed L2 ----------------------------
    flush_w = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB
    flush_r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device="cuda")    # 256 MiB
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")

    def flush(i):
        flush_w.fill_(float(i & 1023))
        sink.add_(flush_r.sum())

    k_fl = min(args.steps, 200)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(k_fl)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(k_fl)]
    barrier()
    for i in range(k_fl):
        flush(i)
        starts[i].record(stream)
        solver.step(1)
        ends[i].record(stream)
    barrier()
    flushed_ms = np.array([a.elapsed_time(b) for a, b in zip(starts, ends)])

    # ---- e2e through the public API with pinned host buffers ---------------
    h_host = torch.from_numpy(h0.reshape(-1)).pin_memory()
    h_out = torch.empty(h_host.numel(), dtype=torch.float32).pin_memory()
    h_host_np, h_out_np = h_host.numpy(), h_out.numpy().reshape(N_LAYERS, NY, NX)
    k_e2e = max(3, min(args.steps, 200))
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        solver.set_heights(h_host_np)
        solver.step(1)
        solver.get_heights(h_out_np)
    t1 = time.perf_counter()
    e2e_s = t1 - t0
    assert np.isfinite(h_out_np).all()
    status = solver.status()
    solver.close()

    total_s, e2e_s = max_over_ranks([total_s, e2e_s], "cuda")

    if rank == 0:
        value = job_rate(ws, lsu_step * args.steps, total_s)
        avg_launch_s = total_s / args.steps
        bytes_alg = BYTES_PER_LSU * lsu_step
        peak, peak_src = hbm_peak()
        achieved = bytes_alg / avg_launch_s / 1e9
        traffic = ncu_traffic()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * avg_launch_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "step_d2q9_tma<3,kFast>",
                         "bytes_per_launch_algorithmic": bytes_alg, "peak_source": peak_src},
            "e2e": {"value": job_rate(ws, lsu_step * k_e2e, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": int(h_host.numel() * 4),
                    "d2h_bytes_per_step": int(h_out.numel() * 4), "steps": k_e2e,
                    "api": "mlswlbm_set_heights + mlswlbm_step(1) + mlswlbm_get_heights"},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "step_ms": {"min": float(step_ms.min()), "p10": float(np.percentile(step_ms, 10)),
                        "p50": float(np.median(step_ms)),
                        "p90": float(np.percentile(step_ms, 90)), "max": float(step_ms.max()),
                        "chunks": int(len(step_ms)),
                        "note": "mean time per step of each chunk of %d timed steps" % chunk},
            "flushed_l2": {"ms_per_step_mean": float(flushed_ms.mean()),
                           "ms_per_step_p50": float(np.median(flushed_ms)), "steps": k_fl,
                           "note": "context only: one step after a 256 MiB L2 flush; the "
                                   "step's dirty lines are written back outside the events"},
            "status": B.mlswlbm_strerror(status),
        }
        if not args.no_extra:
            line["workloads"] = extra_workloads(B, torch)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_sample()
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def extra_workloads(B, torch):
    """Time to solution of the D1Q3 film, LSU/s of the 2048^2 lens field and
    of the batched sweep, and the analysis calls on the 1024^2 film."""
    out = {}
    p = workloads.film2_d1q3_params(512)
    h0 = workloads.film2_d1q3_heights(512)
    with B.Solver(p, h0) as s:
        s.step(100)
        torch.cuda.synchronize()
        l0 = s.launch_count()
        t0 = time.perf_counter()
        s.step(10000)
        h = s.get_heights()
        t1 = time.perf_counter()
        out["film2_d1q3_512"] = {
            "steps": 10000, "ms_to_solution": 1e3 * (t1 - t0),
            "steps_per_s": 10000 / (t1 - t0), "gpu_launches": int(s.launch_count() - l0),
            "note": "mlswlbm_step(10000) + mlswlbm_get_heights, wall clock",
            "finite": bool(np.isfinite(h).all())}
    out["lens3_d2q9_2048"] = lens_workload(B, torch)
    out["stability_sweep_512"] = sweep_workload(B, torch)
    out["analysis_film3_1024"] = analysis_workload(B)
    out["unet_surrogate_film3_256"] = unet_workload(B, torch)
    return out


def lens_workload(B, torch, max_steps=500000, check_every=5000, ke_stop=1e-12):
    """The droplet/lens equilibrium workload: four three-layer lenses of
    base radius 200 on the 2048^2 D2Q9 lattice. LBM throughput over 100
    back-to-back steps, then the run to equilibrium: mlswlbm_step_until
    until the kinetic energy falls below 1e-12 or 500 000 steps, wall clock,
    and the upper and lower Neumann angles of every lens from the device's
    ring means and the library's arc fit (target 20 degrees; the FP64
    oracle's 128^2 version of the workload gives 18.7-19.3)."""
    side, radius, steps = 2048, 200.0, 100
    p = workloads.lens3_params(side, side, radius)
    h0 = workloads.lens3_heights(side, side, radius)
    st = torch.cuda.current_stream()
    lsu = 3 * side * side
    peak, _ = hbm_peak()
    res = {}
    with B.Solver(p, h0, stream=st) as s:
        s.step(5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) * 1e-3 / steps
        res.update({"value": lsu / dt, "unit": UNIT, "ms_per_step": 1e3 * dt, "steps": steps,
                    "roofline_frac": BYTES_PER_LSU * lsu / dt / 1e9 / peak,
                    "l2": "back-to-back steps; 2 x 906 MB working set > 129 MB L2"})
        t0 = time.perf_counter()
        done, ke = s.step_until(max_steps, check_every, ke_stop)
        t1 = time.perf_counter()
        nb = int(1.6 * radius)
        upper, lower = [], []
        for c in workloads.lens3_centres(side, side, radius):
            prof, cnt = s.radial_profile(c, nb)
            up = prof[3] - prof[3][-3:].mean()
            lo = prof[2][-3:].mean() - prof[2]
            upper.append(B.fit_cap_angle(up, cnt, 0.0))
            lower.append(B.fit_cap_angle(lo, cnt, 0.0))
        res["to_equilibrium"] = {
            "steps": int(done + steps + 5), "seconds": t1 - t0, "kinetic_energy": ke,
            "stopped_by": "kinetic energy" if ke < ke_stop else "step cap",
            "ke_threshold": ke_stop, "step_cap": max_steps,
            "upper_angles_deg": [a for a, _ in upper], "lower_angles_deg": [a for a, _ in lower],
            "arc_fit_errors": [e for _, e in upper + lower],
            "neumann_angle_deg": 20.0}
        res["status"] = B.mlswlbm_strerror(s.status())
    return res


def unet_workload(B, torch):
    """The U-Net surrogate of 64 LBM steps on the three-layer spinodal film
    (the 1024^2 benchmark recipe at 256^2; 3 height planes and 5 parameter
    planes):
      * training on 20 000 seeded trajectories of 4 windows each, made by the
        batched solver 250 at a time and dropped after their Adam steps;
      * errors of 64 held-out trajectories over 16 windows against the LBM,
        next to the identity map's (the window's own change);
      * tensor-core throughput of prediction and training;
      * time to solution of 64 instances over 16 windows (1024 steps): the
        U-Net judged by the LBM every 4th window (bound 1e-3), the batched
        solver, and one solver per instance, each timed five times (medians
        and ranges), with the largest height difference from the batched
        solver's result."""
    from paper_2409_16659_gb300 import surrogate as S
    side, n = 256, 3
    p = workloads.film3_d2q9_params(side, side)
    extra = workloads.film3_unet_planes(p)
    ntraj, chunk, windows, batch = 20000, 250, 4, 32
    nchunks = ntraj // chunk
    steps_per_chunk = chunk * windows // batch
    st = torch.cuda.current_stream()
    res = {"trajectories": nchunks * chunk, "windows_per_trajectory": windows,
           "train_batch": batch}
    with B.UNet(n, side, side, batch, extra=extra, seed=1, in_scale=1.0, out_scale=4.0,
                stream=st) as u:
        stream_t = S.TrajectoryStream([p] * chunk,
                                      workloads.film3_d2q9_heights_device(side, side, chunk, 1),
                                      windows, stream=st)
        gen_s = [0.0]

        def make_chunk(k):
            t0 = time.perf_counter()
            tr = stream_t(workloads.film3_d2q9_heights_device(side, side, chunk, 1000 + k))
            torch.cuda.synchronize()
            gen_s[0] += time.perf_counter() - t0
            return tr

        t0 = time.perf_counter()
        losses = S.train_streaming(u, make_chunk, nchunks, steps_per_chunk, batch, 2e-3, 2e-4,
                                   seed=5)
        torch.cuda.synchronize()
        res["train_s"] = time.perf_counter() - t0 - gen_s[0]
        res["trajectories_s"] = gen_s[0]
        stream_t.close()
        res["loss_start_end"] = [float(losses[:20].mean()), float(losses[-50:].mean())]
        # held-out trajectories: other seeds, 16 windows
        hold = S.TrajectoryStream([p] * 64, workloads.film3_d2q9_heights_device(side, side, 64, 7),
                                  16, stream=st)
        traj = hold(workloads.film3_d2q9_heights_device(side, side, 64, 99991))
        hold.close()
        err, ident = S.unet_window_errors(u, traj)
        res["held_out"] = {
            "max_err_per_window": [float(v) for v in err.max(axis=0)],
            "identity_max_err_per_window": [float(v) for v in ident.max(axis=0)],
            "median_err_over_identity": float(np.median(err / ident)),
            "frac_windows_err_le_1e-3": float((err <= 1e-3).mean()),
            "identity_frac_le_1e-3": float((ident <= 1e-3).mean())}
        # throughput of the tensor-core kernels
        h = traj[:batch, 0].contiguous()
        t = traj[:batch, 1].contiguous()
        o = torch.empty_like(h)
        for _ in range(3):
            u.predict(h, o)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(st)
        for _ in range(10):
            u.predict(h, o)
        e[1].record(st)
        for _ in range(10):
            u.train_step(h, t, 0.0)
        e[2].record(st)
        torch.cuda.synchronize()
        fwd_flop = 22.347e9 * batch   # the 15 convolutions of one 256^2 sample, x batch
        pm, tm = e[0].elapsed_time(e[1]) / 10, e[1].elapsed_time(e[2]) / 10
        res["tensor_cores"] = {"predict_ms_batch32": pm, "train_step_ms_batch32": tm,
                               "predict_tflops": fwd_flop / pm / 1e9,
                               "train_tflops": 3 * fwd_flop / tm / 1e9,
                               "note": "22.35 GFLOP per sample forward; training counted as 3x"}
        # time to solution, 64 instances x 16 windows, each arm timed five
        # times in turn (median and range)
        params = [p] * 64
        h0s = [np.asarray(workloads.film3_d2q9_heights(side, side, seed=50000 + j), np.float32)
               for j in range(64)]
        reps, tb, tp, ts = 5, [], [], []
        for _ in range(reps):
            ref, t = S.lbm_batched(params, h0s, 16, stream=st)
            tb.append(t)
            tp.append(S.lbm_per_instance(params, h0s, 16, stream=st)[1])
            hr, info = S.judged_rollout(u, params, h0s, 16, audit_every=4, bound=1e-3, stream=st)
            ts.append(info["seconds"])
        med = lambda v: float(np.median(v))
        res["time_to_solution"] = {
            "instances": 64, "windows": 16, "steps": 1024, "repeats": reps,
            "surrogate_judged_s": med(ts), "lbm_batched_s": med(tb), "lbm_per_instance_s": med(tp),
            "surrogate_judged_range_s": [min(ts), max(ts)], "lbm_batched_range_s": [min(tb), max(tb)],
            "lbm_per_instance_range_s": [min(tp), max(tp)],
            "speedup_vs_per_instance": med(tp) / med(ts),
            "speedup_vs_batched": med(tb) / med(ts),
            "speedup_vs_batched_worst_case": min(tb) / max(ts),
            "surrogate_windows": info["surrogate_windows"],
            "audited_windows": info["audited_windows"],
            "fallback_instances": info["fallback_instances"],
            "max_audit_err": float(max(info["audit_errors"])) if info["audit_errors"] else None,
            "final_max_height_diff_vs_lbm": float(
                B.max_abs_diff(hr.contiguous(), ref.contiguous()).cpu().numpy().max()),
            "note": "every 4th window and the last judged by the batched LBM from the same "
                    "heights; an instance beyond 1e-3 returns to its last passed audit and "
                    "finishes on the LBM; medians of the repeats"}
        res["status"] = u.status()
    return res


def analysis_workload(B):
    """Wall time of the on-device analysis calls on the 1024^2 three-layer
    film: radial power spectra of the three layers (512 bins) and the ring
    means of the four interfaces around the centre (300 rings), each call
    including its read-back."""
    p = workloads.film3_d2q9_params(NX, NY)
    h0 = workloads.film3_d2q9_heights(NX, NY, seed=2)
    with B.Solver(p, h0) as s:
        s.step(100)
        s.spectrum(NX // 2)
        s.radial_profile((NX / 2, NY / 2), 300)
        reps = 10
        t0 = time.perf_counter()
        for _ in range(reps):
            s.spectrum(NX // 2)
        t1 = time.perf_counter()
        for _ in range(reps):
            s.radial_profile((NX / 2, NY / 2), 300)
        t2 = time.perf_counter()
        return {"spectrum_ms": 1e3 * (t1 - t0) / reps, "radial_profile_ms": 1e3 * (t2 - t1) / reps,
                "note": "mlswlbm_get_spectrum(512 bins) and mlswlbm_get_radial_profile(300 rings), "
                        "wall clock per call, results on the host",
                "status": B.mlswlbm_strerror(s.status())}


def sweep_workload(B, torch):
    inst = workloads.sweep_instances()
    params = [p for p, _, _, _ in inst]
    heights = [h for _, h, _, _ in inst]
    kx = [m[0] for _, _, m, _ in inst]
    ky = [m[1] for _, _, m, _ in inst]
    lsu = sum(p["n"] * p["nx"] * p["ny"] for p in params)
    st = torch.cuda.current_stream()
    res = {"instances": len(inst), "layer_sites_per_step": lsu}
    t0 = time.perf_counter()
    with B.Batch(params, heights, flags=B.MLSW_BATCH_AUTOTUNE, stream=st) as b:
        torch.cuda.synchronize()
        res["create_s"] = time.perf_counter() - t0
        rows = [b.tile_rows(j) for j in range(len(inst))]
        res["groups"] = b.groups()
        l0 = b.launch_count()
        b.step(1)
        res["launches_per_step"] = b.launch_count() - l0
        res["tile_rows_16"] = rows.count(16)
        res["tile_rows_8"] = rows.count(8)
        b.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 40
        e0.record(st)
        b.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) * 1e-3 / steps
        peak, _ = hbm_peak()
        res.update({"value": lsu / dt, "unit": UNIT, "ms_per_step": 1e3 * dt,
                    "roofline_frac": BYTES_PER_LSU * lsu / dt / 1e9 / peak})
        # time to solution: 2000 steps, the perturbed mode every 200 steps,
        # one growth rate per instance fitted to ln |hhat| of its top layer
        t1 = time.perf_counter()
        amp = [np.abs(b.modes(kx, ky))]
        for _ in range(10):
            b.step(200)
            amp.append(np.abs(b.modes(kx, ky)))
        amp = np.array(amp)  # [sample][instance][layer]
        tt = 200.0 * np.arange(amp.shape[0])
        rates = []
        for j, p in enumerate(params):
            a = amp[:, j, p["n"] - 1]
            rates.append(float(np.polyfit(tt[5:], np.log(np.maximum(a[5:], 1e-300)), 1)[0]))
        res["time_to_solution_s"] = time.perf_counter() - t1
        res["growth_rate_range"] = [min(rates), max(rates)]
        res["status"] = B.mlswlbm_strerror(b.status())
    # the same work one solver per instance, one launch per step
    t2 = time.perf_counter()
    solvers = [B.Solver(p, h, stream=st) for p, h in zip(params, heights)]
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    per = 20
    for s in solvers:
        s.step(per)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    for s in solvers:
        s.close()
    res["per_instance"] = {"create_s": t3 - t2, "ms_per_step": 1e3 * (t4 - t3) / per,
                           "steps_timed": per, "note": "one Solver per instance, "
                           "mlswlbm_step(20) each in turn, wall clock"}
    res["speedup_vs_per_instance"] = res["per_instance"]["ms_per_step"] / res["ms_per_step"]
    return res


def run_profile_batch(args):
    """Warm-up then --steps steps of the first 64 sweep instances (~1.4 GB)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2409_16659_gb300 import mlswlbm as B
    inst = workloads.sweep_instances()[:64]
    with B.Batch([p for p, _, _, _ in inst], [h for _, h, _, _ in inst],
                 stream=torch.cuda.current_stream()) as b:
        b.step(args.warmup)
        b.step(args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"profile_batch_run": True, "groups": b.groups(),
                          "launches": b.launch_count(),
                          "status": B.mlswlbm_strerror(b.status())}), flush=True)
    return 0


def run_profile(args):
    """Warm-up then --steps back-to-back steps; no flush, e2e or CPU leg."""
    import torch
    torch.cuda.set_device(0)
    from paper_2409_16659_gb300 import mlswlbm as B
    p = workloads.film3_d2q9_params(NX, NY)
    h0 = workloads.film3_d2q9_heights(NX, NY).astype(np.float32)
    with B.Solver(p, h0, stream=torch.cuda.current_stream()) as s:
        s.step(args.warmup)
        s.step(args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "launches": s.launch_count(),
                          "status": B.mlswlbm_strerror(s.status())}), flush=True)
    return 0


def run_profile_unet(args):
    """The U-Net surrogate at 256^2, batch 8: --warmup predictions, then
    --steps predictions and one training step (for ncu captures of the
    convolution kernels: 15 launches of conv_tc per prediction, the
    13th being the largest level-0 one, 96 -> 32 channels)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2409_16659_gb300 import mlswlbm as B
    side, batch = 256, 8
    p = workloads.film3_d2q9_params(side, side)
    st = torch.cuda.current_stream()
    with B.UNet(3, side, side, batch, extra=workloads.film3_unet_planes(p), seed=1,
                in_scale=1.0, out_scale=4.0, stream=st) as u:
        h = workloads.film3_d2q9_heights_device(side, side, batch, 5)
        out = torch.empty_like(h)
        for _ in range(args.warmup + args.steps):
            u.predict(h, out)
        u.train_step(h, out, 0.0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_unet_run": True, "status": u.status()}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the D1Q3 film and 2048^2 lens workloads")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up + --steps back-to-back steps (for ncu captures)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="the same for a 64-instance batch of the stability sweep")
    ap.add_argument("--profile-unet", action="store_true",
                    help="U-Net predictions at 256^2 (for ncu captures of its convolutions)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.profile_unet:
        return run_profile_unet(args)
    return run_own(args)


if __name__ == "__main__":
    sys.exit(main())
