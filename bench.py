#!/usr/bin/env python
"""Benchmark of the event-to-flow path: flow frames/s at 1280x720.

Workload: the 1280x720 synthetic stream (201 windows of 10 ms, 150k-400k
events each, 12 rigid objects with their own affine motion, 3 % noise,
seed 1 + rank), i.e. 200 flow frames per step.  One step = one pass of the
whole path (edge image, denoise, exact EDT, surface, pyramid, inverse
search, densification, variational refinement) over every window of the
stream, with all events resident in HBM before the timed region (715 MB
of events per step, larger than the 129 MB L2).

Prints one JSON line (rank 0).  `value` is one window per call through the
pipelined ebof_process_window_async (a window's front end overlaps the
previous window's flow levels; CUDA events on the caller's stream, the step
closed by ebof_stream_join); `in_order` the same windows through
ebof_process_window (every stage of a window in order on the caller's
stream), which also gives the per-window latencies; `batched` is the same stream through
ebof_process_windows; `e2e` streams the windows through
ebof_process_window_host_async with the events in pinned host memory and
every window's flow written back into a pinned host buffer (page-locked
buffers are addressed by the kernels over the host link, so the events cross
it inside the scatter and the flow inside the last kernel), one
ebof_stream_sync per step; `e2e.synchronous_per_window` is the same through
ebof_process_window_host, which synchronises after every window;
`roofline` covers the dominant step, the variational refinement at level 0,
by its algorithmic bytes (24 B per pixel per outer iteration: I0, I1, U in,
U out) over its kernels' time, with every stage's fraction and the patch
search against the FP32 ALU beside it; `config0_346x260` is the 346x260
single-window workload; `cpu_baseline` is the FP64 oracle on a bounded sample
of the same stream, on this host's cores, and alone on one core.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flow frames/s at 1280x720 (batched vs plain), p99 latency, EPE vs FP64 oracle"
UNIT = "frames/s"
W_, H_ = 1280, 720
N_WINDOWS = 201


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--windows", type=int, default=N_WINDOWS)
    ap.add_argument("--batch", type=int, default=40, help="windows per batched call")
    ap.add_argument("--cpu-frames", type=int, default=0,
                    help="oracle sample size (default: one frame per worker)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-multistream", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-config0", action="store_true")
    ap.add_argument("--c0-windows", type=int, default=400,
                    help="windows of the 346x260 single-window line")
    ap.add_argument("--sv-seconds", type=float, default=0.5,
                    help="arrival span of each timed serving run")
    ap.add_argument("--sv-warmup", type=float, default=0.3)
    ap.add_argument("--sv-windows", type=int, default=12,
                    help="generated windows per serving sequence")
    ap.add_argument("--sv-workers", type=int, default=8)
    ap.add_argument("--sv-max-batch", type=int, default=16,
                    help="windows of one stream the server may batch into one launch")
    ap.add_argument("--sv-scales", type=lambda v: [float(x) for x in v.split(",")],
                    default=[1.0, 0.8, 0.65, 0.5, 0.42, 0.35],
                    help="arrival-rate scales of the serving runs")
    ap.add_argument("--sv-p99-bound-ms", type=float, default=10.0,
                    help="p99 latency bound of the sustainable-rate search (one window)")
    ap.add_argument("--ms-windows", type=int, default=11,
                    help="windows per stream in the multi-stream run")
    return ap.parse_args()


# ---------------------------------------------------------------- oracle leg
def _oracle_frame(args):
    """FP64 oracle for one frame pair (previous window, current window)."""
    import oracle
    (w0, w1, prm) = args
    s0 = oracle.surface_from_events(W_, H_, *w0, connectivity=prm["connectivity"],
                                    n_d=prm["n_d"], n_f=prm["n_f"], alpha=prm["alpha"])
    s1 = oracle.surface_from_events(W_, H_, *w1, connectivity=prm["connectivity"],
                                    n_d=prm["n_d"], n_f=prm["n_f"], alpha=prm["alpha"])
    U = oracle.flow(255.0 * s0["S"], 255.0 * s1["S"], levels=prm["levels"],
                    patch=prm["patch"], stride=prm["stride"], gn_iters=prm["gn_iters"],
                    gn_damping=prm["gn_damping"],
                    var_outer=prm["var_outer"], var_sor=prm["var_sor"],
                    var_delta=prm["var_delta"], var_gamma=prm["var_gamma"],
                    var_alpha=prm["var_alpha"], sor_omega=prm["sor_omega"])
    return U.astype(np.float32)


def _params_dict(p):
    return {k: getattr(p, k) for k, _ in type(p)._fields_}


def _window_tuple(stream, k):
    x, y, t, _, tb, te = stream.window(k)
    return (np.ascontiguousarray(x), np.ascontiguousarray(y), np.ascontiguousarray(t), tb, te)


def oracle_sample(stream, prm, frames, workers):
    """Time the oracle on `frames` frame pairs spread over `workers` processes."""
    import oracle
    oracle.build()
    tasks = [(_window_tuple(stream, k), _window_tuple(stream, k + 1), prm)
             for k in range(frames)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_noop, range(workers))  # start the workers outside the timed region
        t0 = time.perf_counter()
        flows = pool.map(_oracle_frame, tasks, chunksize=1)
        dt = time.perf_counter() - t0
    return flows, dt


def _oracle_noop(_):
    import oracle  # noqa: F401
    return 0


def _oracle_frame_timed(args):
    """One frame pair in a fresh single-threaded process: (front end of both
    windows, flow) wall seconds."""
    import oracle
    (w0, w1, prm) = args
    t0 = time.perf_counter()
    kw = dict(connectivity=prm["connectivity"], n_d=prm["n_d"], n_f=prm["n_f"],
              alpha=prm["alpha"])
    s0 = oracle.surface_from_events(W_, H_, *w0, **kw)
    s1 = oracle.surface_from_events(W_, H_, *w1, **kw)
    t1 = time.perf_counter()
    oracle.flow(255.0 * s0["S"], 255.0 * s1["S"], levels=prm["levels"], patch=prm["patch"],
                stride=prm["stride"], gn_iters=prm["gn_iters"], gn_damping=prm["gn_damping"],
                var_outer=prm["var_outer"], var_sor=prm["var_sor"], var_delta=prm["var_delta"],
                var_gamma=prm["var_gamma"], var_alpha=prm["var_alpha"],
                sor_omega=prm["sor_omega"])
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def oracle_single_thread(stream, prm):
    """The oracle alone on one core: one frame pair (windows 0 and 1) in one
    process with nothing else running.  Per window: the front end of one
    window plus the flow of one pair."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        pool.map(_oracle_noop, [0])
        front2, flow = pool.map(_oracle_frame_timed,
                                [(_window_tuple(stream, 0), _window_tuple(stream, 1), prm)])[0]
    return {"ms_per_window": 1000.0 * (0.5 * front2 + flow),
            "front_end_ms_per_window": 500.0 * front2, "flow_ms_per_frame": 1000.0 * flow,
            "threads": 1,
            "sample": "windows 0 and 1 of the 1280x720 stream: both front ends, one flow"}


def cpu_workers():
    """Processes of the oracle sample: every host core, at most 16."""
    n = os.cpu_count() or 1
    return max(1, min(n, 16))


def workload_name(nwin):
    return ("1280x720 single stream, %d windows of 10 ms (%d flow frames), 150k-400k "
            "events/window, 12 affine objects, 3%% noise, seed 1+rank" % (nwin, nwin - 1))


def bench_config(prm, nwin, world):
    """The workload and method parameters, identical in both arms."""
    return {"workload": workload_name(nwin),
            "levels": prm["levels"], "patch": prm["patch"], "stride": prm["stride"],
            "gn_iters": prm["gn_iters"], "var": "%dx%d" % (prm["var_outer"], prm["var_sor"]),
            "l2": "inputs larger than L2: the events of every window of a step (about "
                  "0.7 GB) resident in HBM",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank):
    """The reference arm: the FP64 oracle, as it stands, on this host's cores."""
    if rank != 0:
        return
    import ctypes  # noqa: F401
    from paper_2112_10591_gb300 import synth
    stream = synth.workload_1280x720(seed=1, n_windows=3)
    prm = _reference_params()
    workers = cpu_workers()
    frames_per_step = workers
    times = []
    for i in range(args.warmup + args.steps):
        k = [j % 2 for j in range(frames_per_step)]
        tasks = [(_window_tuple(stream, kk), _window_tuple(stream, kk + 1), prm) for kk in k]
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            pool.map(_oracle_noop, range(workers))
            t0 = time.perf_counter()
            pool.map(_oracle_frame, tasks, chunksize=1)
            dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = frames_per_step * len(times) / total
    world = int(os.environ.get("WORLD_SIZE", "1"))
    sample = ("each step times %d frame pairs of the workload, one per process on %d host "
              "cores (of %d): windows 0->1 and 1->2 of a 3-window draw of the same "
              "1280x720 generator, alternating" % (frames_per_step, workers,
                                                   os.cpu_count() or 1))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(prm, args.windows, world),
        "path": "FP64 oracle (plain C, one window pair per process), as it stands",
        "sample": sample,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "host_cores": os.cpu_count(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def _reference_params():
    # the library's defaults for a 1280x720 sensor, written out (no library load)
    return dict(connectivity=8, n_d=1, n_f=9, alpha=1.08, levels=5, patch=12, stride=4,
                gn_iters=12, gn_damping=0.1, var_outer=5, var_sor=5, var_delta=5.0, var_gamma=10.0,
                var_alpha=20.0, sor_omega=1.6)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline
def algorithmic_bytes_per_launch(stage, level, geo, n_events_per_window, P):
    """Algorithmic bytes of ONE launch of a stage for one window: each
    kernel's inputs read once and outputs written once, by the per-stage
    formulas below.  geo: [(w, h, npx, npy)] per pyramid level."""
    if level >= 0:
        w, h, npx, npy = geo[level]
        Pl, npl = w * h, npx * npy
        Pc = geo[level + 1][0] * geo[level + 1][1] if level + 1 < len(geo) else 0
    per = {
        "scatter": lambda: 13.0 * n_events_per_window,
        "denoise_fill": lambda: 2.0 * P,          # per kernel: read one byte image, write one
        "edt_cols": lambda: 5.0 * P,              # E_df bytes in, int32 g out
        "edt_rows_surface": lambda: 8.0 * P,      # int32 g in, float intensity out
        "pyramid": lambda: 12.0 * Pl,             # gradients: I in, Ix and Iy out
        "patch_search": lambda: 16.0 * Pl + 8.0 * npl + 8.0 * Pc,
        "densify": lambda: 16.0 * Pl + 8.0 * npl,
        "var_coeff": lambda: 52.0 * Pl,           # U, I1, I0, I0x, I0y in; 7 planes out
        "var_sor": lambda: 44.0 * Pl,             # 7 planes and U in, U out
        "flow_out": lambda: 16.0 * P,
    }
    f = per.get(stage)
    return float(f()) if f else 0.0


PER_LEVEL = ("pyramid", "patch_search", "densify", "var_coeff", "var_sor")


def stage_hbm_fractions(ms_per_frame, P, n_events, n_levels, var_outer, peak):
    """HBM fraction of each hot-path stage with the stage's algorithmic bytes
    per flow frame: its own inputs read once and outputs written once, the
    variational stage once per outer iteration (I0, I1, U in, U out: 24 B per
    pixel of every level) with its SOR sweeps on chip; c_L = sum of 4^-l over
    the levels.  ms_per_frame: stage times per frame from the stage profile."""
    cL = sum(4.0 ** -l for l in range(n_levels))
    rows = (
        ("A1 scatter", 12.0 * n_events + P + n_events, ("scatter",)),
        ("A2 denoise_fill", 2.0 * P, ("denoise_fill",)),
        ("A3+A4 edt_surface", 17.0 * P, ("edt_cols", "edt_rows_surface")),
        ("A5 pyramid", 22.0 * P, ("pyramid",)),
        ("A6 patch_search", 17.0 * P * cL, ("patch_search",)),
        ("A7 densify", 16.0 * P * cL, ("densify",)),
        ("A8 variational", var_outer * 24.0 * P * cL, ("var_coeff", "var_sor")),
    )
    out, tb, tt = {}, 0.0, 0.0
    for name, nbytes, stages in rows:
        t = sum(ms_per_frame.get(k, 0.0) for k in stages)
        if t <= 0.0:
            continue
        gbs = nbytes / (t / 1000.0) / 1e9
        out[name] = {"bytes_per_frame": nbytes, "ms_per_frame": t,
                     "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
        tb += nbytes
        tt += t
    if tt > 0.0:
        gbs = tb / (tt / 1000.0) / 1e9
        out["all stages"] = {"bytes_per_frame": tb, "ms_per_frame": tt,
                             "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    return out


def a8_outer_iteration_roofline(by_level, P0, var_outer, frames, peak, traffic_coeff,
                                traffic_sor):
    """Headline roofline of the dominant hot-path step, the variational
    refinement (A8) at level 0.  Unit: one outer iteration, whose algorithmic
    bytes are I0, I1, U in and U out, 24 B per pixel (its SOR sweeps run on
    chip); its time is the level's coefficient and SOR launches of that
    iteration.  by_level: stage ms per frame at level 0."""
    t_ms = by_level.get("var_coeff", 0.0) + by_level.get("var_sor", 0.0)
    if t_ms <= 0.0 or var_outer <= 0:
        return None
    per_iter_s = t_ms / 1000.0 / var_outer
    nbytes = 24.0 * P0
    achieved = nbytes / per_iter_s / 1e9
    traffic = None
    if traffic_coeff is not None and traffic_sor is not None:
        traffic = traffic_coeff + traffic_sor
    return {"bound": "hbm", "kernel": "A8 variational refinement at level 0: var_coeff + "
                                      "var_sor launches of one outer iteration",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "bytes_per_unit": nbytes,
            "unit_def": "one outer iteration at level 0 (24 B per pixel: I0, I1, U in, U out)",
            "us_per_unit": per_iter_s * 1e6, "frames_profiled": frames}


FP32_LANES_PER_SM = 128   # four sub-partitions of 32 FP32 lanes
N_SMS = 152


def a6_flop_roof(by_level_all, geo, ps, iters, sm_mhz):
    """A6 (patch inverse search) against the FP32 ALU: 25 flop per patch pixel
    and Gauss-Newton iteration (bilinear sample, residual, two products and
    sums), summed over the patches of every level, over the search time.
    Peak = SMs x FP32 lanes x 2 (FMA) x SM clock."""
    flops = sum(25.0 * ps * ps * iters * npx * npy for (_, _, npx, npy) in geo)
    t_ms = sum(v.get("patch_search", 0.0) for k, v in by_level_all.items() if k != "all")
    if t_ms <= 0.0:
        return None
    clock = sm_mhz or 2070.0
    peak = N_SMS * FP32_LANES_PER_SM * 2.0 * clock * 1e6 / 1e12
    ach = flops / (t_ms / 1000.0) / 1e12
    l0 = by_level_all.get("0", {}).get("patch_search", 0.0)
    f0 = 25.0 * ps * ps * iters * geo[0][2] * geo[0][3]
    return {"bound": "alu", "flop_per_frame": flops, "ms_per_frame": t_ms,
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "level0": {"flop": f0, "ms": l0,
                       "achieved": f0 / (l0 / 1000.0) / 1e12 if l0 > 0 else None},
            "peak_source": "derived: %d SMs x %d FP32 lanes x 2 flop (FMA) x %.0f MHz "
                           "(median SM clock of the timed region)"
                           % (N_SMS, FP32_LANES_PER_SM, clock),
            "l1_smem": profile_figure("patch_search_kernel_1280x720_level0.md",
                                      "l1tex__throughput")}


def profile_figure(name, metric):
    """A metric's value from a committed ncu summary under profiles/ (the
    table row whose metric name matches), or None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        for ln in open(path).read().splitlines():
            if ("`%s" % metric) in ln and ln.startswith("|"):
                cells = [c.strip() for c in ln.strip("|").split("|")]
                return {"metric": metric, "value": cells[-1], "source": "profiles/" + name}
    except OSError:
        pass
    return None


def geo_levels(p):
    out = []
    for l in range(p.levels):
        w, h = p.width >> l, p.height >> l
        if w < p.patch or h < p.patch:
            break
        npx = (w - p.patch + p.stride - 1) // p.stride + 1
        npy = (h - p.patch + p.stride - 1) // p.stride + 1
        out.append((w, h, npx, npy))
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def dram_traffic(stage, level):
    """DRAM bytes per launch of this stage at this level from the committed
    ncu summary (profiles/dram_traffic.txt), or None when the kernel's source
    file changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if not ln.strip() or ln.startswith("#"):
            continue
        f = ln.split()
        if len(f) < 6 or f[1] != stage or int(f[2]) != level:
            continue
        src = os.path.join(ROOT, f[4])
        try:
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        except OSError:
            return None
        return int(f[3]) if sha == f[5] else None
    return None


# ---------------------------------------------------------------- replicas
def replica_seed(rank):
    """Each rank runs its own camera stream (replicas, no data-path exchange)."""
    return 1 + rank


def combine_ranks(ms_local, frames_local, world, dist=None, device=None):
    """Whole-job timing: the slowest rank's time, and the frames of all ranks
    over it (weak scaling: every rank processes the same amount)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, frames_local * world / (ms / 1000.0)


# ---------------------------------------------------------------- multi-stream
def run_multistream(args, eb, torch, dev, rank):
    """16 concurrent camera streams in lockstep: 12 at 346x260 and 4 at
    1280x720, lognormal event counts in [5k, 500k] per window, rigid objects
    with random affine motion, FP16 storage.  One group per resolution, both
    stepped as one CUDA graph per step (ebof_multigroup: each group's step a
    branch of the graph); for comparison the same groups stepped separately
    on two CUDA streams.  The patch grid and the variational layouts of each
    resolution are picked by the autotuner."""
    from paper_2112_10591_gb300 import autotune, synth
    nw = max(3, args.ms_windows)
    specs = [(346, 260, 12, dict(n_objects=4, n_edges=60, radius=(15.0, 60.0),
                                 extra_length=(5.0, 40.0))),
             (1280, 720, 4, {})]
    groups = []
    for gi, (W, H, n, kw) in enumerate(specs):
        evs = [synth.rigid_objects(width=W, height=H, n_windows=nw, events=(5000, 500000),
                                   lognormal_counts=True, seed=1000 * (rank + 1) + 100 * gi + i,
                                   **kw) for i in range(n)]
        dev_ev = []
        for ev in evs:
            xs = torch.from_numpy(ev.x).to(dev)
            ys = torch.from_numpy(ev.y).to(dev)
            ts = torch.from_numpy(ev.t).to(dev)
            wins = []
            for k in range(nw):
                a, b = int(ev.offsets[k]), int(ev.offsets[k + 1])
                tb = int(ev.t_begin[k])
                wins.append((xs[a:b], ys[a:b], ts[a:b], tb, tb + ev.dt))
            dev_ev.append((wins, (xs, ys, ts)))
        calib = [(w[0][0], w[0][1]) for w in dev_ev]
        prm, table = autotune.tune(W, H, calib, storage=eb.EBOF_STORAGE_FP16,
                                   device=dev.index or 0)
        st, g = eb.ebof_group_create(prm, n, dev.index or 0)
        eb.check(st, "ebof_group_create")
        groups.append({"W": W, "H": H, "n": n, "g": g, "ev": dev_ev, "prm": prm,
                       "table": table, "cs": torch.cuda.Stream(device=dev),
                       "events": int(sum(int(ev.offsets[-1]) for ev in evs))})
    main = torch.cuda.current_stream(dev)
    st, mg = eb.ebof_multigroup_create([gr["g"] for gr in groups])
    eb.check(st, "ebof_multigroup_create")

    def step_graph(k):
        r = eb.ebof_multigroup_process(mg, [[w[0][k] for w in gr["ev"]] for gr in groups])
        if r < 0:
            raise eb.EbofError(r, "ebof_multigroup_process")

    def step_streams(k):
        for gr in groups:
            gr["cs"].wait_stream(main)
            with torch.cuda.stream(gr["cs"]):
                r = eb.ebof_group_process(gr["g"], [w[0][k] for w in gr["ev"]])
                if r < 0:
                    raise eb.EbofError(r, "ebof_group_process")
        for gr in groups:
            main.wait_stream(gr["cs"])

    def sweep(step, times=None):
        for gr in groups:
            eb.check(eb.ebof_group_reset(gr["g"]))
        step(0)
        for k in range(1, nw):
            if times is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(main)
                step(k)
                b.record(main)
                times.append((a, b))
            else:
                step(k)

    def timed(step):
        for _ in range(max(1, min(args.warmup, 2))):
            sweep(step)
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(args.steps):
            sweep(step, evs)
        torch.cuda.synchronize(dev)
        return np.asarray([a.elapsed_time(b) for a, b in evs])

    def kernels_per_step():
        lib = eb.load()
        before = lib.ebof_kernel_launches()
        step_graph(nw - 1)
        torch.cuda.synchronize(dev)
        return int(lib.ebof_kernel_launches() - before)

    two = timed(step_streams)
    step_ms = timed(step_graph)
    k_branches = kernels_per_step()
    # the same steps with every stage one launch for both resolutions
    fused = None
    def fused_mode(mode, launch):
        rf = eb.ebof_multigroup_set_fused(mg, mode)
        if rf != eb.EBOF_OK:
            return {"unavailable": eb.ebof_status_string(rf)}
        ms = timed(step_graph)
        res = {"value": sum(gr["n"] for gr in groups) * len(ms) / (ms.sum() / 1000.0),
               "p50_step_ms": float(np.percentile(ms, 50)),
               "p99_step_ms": float(np.percentile(ms, 99)),
               "kernels_per_step": kernels_per_step(), "launch": launch}
        eb.ebof_multigroup_set_fused(mg, 0)
        return res

    fused = fused_mode(1, "one CUDA graph per step, every stage ONE launch for the streams "
                          "of both resolutions (ebof_multigroup_set_fused 1): blocks map to "
                          "(group, frame, tile) through tables, the scatter walks a device "
                          "work list of 4096-event chunks")
    front_fused = fused_mode(2, "one CUDA graph per step, the front-end stages one launch for "
                                "both resolutions, the flow levels of each resolution a "
                                "concurrent branch (ebof_multigroup_set_fused 2)")
    nstreams = sum(gr["n"] for gr in groups)
    px = sum(gr["n"] * gr["W"] * gr["H"] for gr in groups)
    total_s = step_ms.sum() / 1000.0
    out = {"value": nstreams * len(step_ms) / total_s, "unit": UNIT,
           "mpx_per_s": px * len(step_ms) / total_s / 1e6,
           "streams": {"%dx%d" % (gr["W"], gr["H"]): gr["n"] for gr in groups},
           "storage": "fp16", "windows_per_stream": nw,
           "p50_step_ms": float(np.percentile(step_ms, 50)),
           "p99_step_ms": float(np.percentile(step_ms, 99)),
           "steps_timed": int(len(step_ms)),
           "launch": "one CUDA graph per step (ebof_multigroup): each resolution group's "
                     "step is one branch of the graph, every stage one launch per "
                     "resolution, the branches concurrent",
           "kernels_per_step": k_branches,
           "fused": fused,
           "front_end_fused": front_fused,
           "two_streams": {"value": nstreams * len(two) / (two.sum() / 1000.0),
                           "p99_step_ms": float(np.percentile(two, 99)),
                           "launch": "one graph replay per group and step, groups on two "
                                     "CUDA streams"},
           "autotune": {"%dx%d" % (gr["W"], gr["H"]): {
               "patch": gr["prm"].patch, "stride": gr["prm"].stride,
               "levels": gr["prm"].levels,
               "layouts": {k: getattr(gr["prm"], k) for k in autotune.LAYOUT_CANDIDATES},
               "table": gr["table"]} for gr in groups}}
    mg.close()
    for gr in groups:
        gr["g"].close()
    return out


def _gt_figures(eb, torch, dev, local, ev):
    """GPU flow of every window pair of ``ev`` against the generator's ground
    truth: mean AEE, median error, outlier share (error > 3 px and > 5 % of
    the motion) and the zero flow's AEE, over the flow frames."""
    prm = eb.ebof_default_params(ev.width, ev.height)
    st, s = eb.ebof_stream_create(prm, local)
    eb.check(st, "ebof_stream_create")
    W, H = ev.width, ev.height
    flows = []
    for k in range(ev.n_windows):
        x, y, t, _, tb, te = ev.window(k)
        fl = torch.empty((2, H, W), dtype=torch.float32, device=dev)
        eb.check(eb.ebof_process_window(s, torch.from_numpy(x).to(dev),
                                        torch.from_numpy(y).to(dev),
                                        torch.from_numpy(t).to(dev), None, tb, te, fl))
        flows.append(fl)
    torch.cuda.synchronize(dev)
    errs, med, outl, zero = [], [], [], []
    for k in range(1, ev.n_windows):
        U = flows[k].cpu().numpy().astype(np.float64)
        G, m = ev.true_flow(k)
        e = np.hypot(U[0] - G[0], U[1] - G[1])[m]
        mag = np.hypot(G[0], G[1])[m]
        errs.append(e.mean())
        med.append(np.median(e))
        outl.append(((e > 3.0) & (e > 0.05 * mag)).mean())
        zero.append(mag.mean())
    s.close()
    return {"aee_px": float(np.mean(errs)), "median_px": float(np.mean(med)),
            "outliers_pct": 100 * float(np.mean(outl)),
            "zero_flow_aee_px": float(np.mean(zero)),
            "aee_over_zero": float(np.mean(errs) / max(np.mean(zero), 1e-12)),
            "frames": ev.n_windows - 1}


def ground_truth_quality(eb, torch, dev, local):
    """§IV-C's AEE and outlier share (error > 3 px and > 5 % of the motion)
    of the GPU flow against the generator's ground truth at the previous
    window's event pixels: the 346x260 workload pair, and 20 flow frames of
    a 21-window copy of the 1280x720 workload (its own draws: the motion of
    a stream is drawn for its length).

    ``motion_sweep``: the 1280x720 scene with the largest translation per
    window set to 2.5, 5, 10 and 20 px (turns scaled alike, 2 degrees at
    20 px), 3 flow frames each, once with the workload's motion (every
    object's turn and translation drawn anew for every window) and once with
    constant velocity (drawn once).  It separates the size of the motion from
    its change between windows."""
    from paper_2112_10591_gb300 import synth
    out = {"346x260": _gt_figures(eb, torch, dev, local,
                                  synth.translating_segments(keep_truth=True)),
           "1280x720": _gt_figures(eb, torch, dev, local,
                                   synth.workload_1280x720(n_windows=21, keep_truth=True))}
    sweep = []
    for const in (False, True):
        for shift in (2.5, 5.0, 10.0, 20.0):
            ev = synth.rigid_objects(n_windows=4, max_shift=shift,
                                     max_rot_deg=2.0 * shift / 20.0, keep_truth=True,
                                     constant_velocity=const)
            row = {"motion": "constant velocity" if const else "redrawn every window",
                   "max_shift_px": shift}
            row.update(_gt_figures(eb, torch, dev, local, ev))
            sweep.append(row)
    out["motion_sweep"] = sweep
    return out


def run_serving(args, eb, torch, dev, rank):
    """64 camera streams served as their windows arrive: 32 at 346x260, 16 at
    640x480 and 16 at 1280x720 (4:2:2).  Each stream delivers windows as a
    Poisson process whose rate is drawn in [100, 250] Hz; window contents
    follow the lognormal [5k, 500k] event counts and per-object affine motion
    of the multi-stream workload, FP16 storage.  Every stream's state (its
    previous pyramid and buffers for its largest batch) is admitted
    under a 40 GB budget and stays resident.  The client submits each window
    at its arrival time through ebof_server_submit; the server's dispatcher
    batches each stream's backlog into list calls on the worker CUDA streams.
    Latency = completion seen by the dispatcher - arrival.  A run at a lower
    rate scale shows the latency when the offered load is below capacity."""
    import ctypes
    from paper_2112_10591_gb300 import synth
    lib = eb.load()
    rng = np.random.default_rng(4242 + rank)
    kinds = [(346, 260, 32, dict(n_objects=4, n_edges=60, radius=(15.0, 60.0),
                                 extra_length=(5.0, 40.0))),
             (640, 480, 16, dict(n_objects=8, n_edges=150, radius=(25.0, 110.0),
                                 extra_length=(8.0, 80.0))),
             (1280, 720, 16, {})]
    n_seq, L = 4, max(4, args.sv_windows)
    max_batch = args.sv_max_batch
    cfg = eb.ebof_server_default_config()
    cfg.device = dev.index or 0
    cfg.n_workers = args.sv_workers
    st, server = eb.ebof_server_create(cfg)
    eb.check(st, "ebof_server_create")
    streams = []
    keep = []
    for ki, (W, H, n, kw) in enumerate(kinds):
        pool = []
        for q in range(n_seq):
            ev = synth.rigid_objects(width=W, height=H, n_windows=L, events=(5000, 500000),
                                     lognormal_counts=True,
                                     seed=5000 * (rank + 1) + 100 * ki + q, **kw)
            xs = torch.from_numpy(ev.x).to(dev)
            ys = torch.from_numpy(ev.y).to(dev)
            ts = torch.from_numpy(ev.t).to(dev)
            keep.append((xs, ys, ts))
            descs = []
            for k in range(L):
                a, b = int(ev.offsets[k]), int(ev.offsets[k + 1])
                d = eb.ebof_window_desc()
                d.x = xs.data_ptr() + 2 * a
                d.y = ys.data_ptr() + 2 * a
                d.t = ts.data_ptr() + 8 * a
                d.n_events = b - a
                d.t_begin = int(ev.t_begin[k])
                d.t_end = int(ev.t_begin[k]) + ev.dt
                descs.append(d)
            pool.append(descs)
        prm = eb.ebof_default_params(W, H)
        prm.storage = eb.EBOF_STORAGE_FP16
        prm.max_batch = max_batch
        for i in range(n):
            r, sid = eb.ebof_server_open_stream(server, prm)
            eb.check(r, "ebof_server_open_stream")
            ring = 2 * max_batch + 1  # flows of one stream complete in order
            fl = torch.empty((ring, 2, H, W), dtype=torch.float32, device=dev)
            keep.append(fl)
            streams.append({"sid": sid, "W": W, "H": H, "seq": pool[i % n_seq],
                            "pos": (i // n_seq) * 3 % L, "rate": float(rng.uniform(100, 250)),
                            "flow": [fl[j].data_ptr() for j in range(ring)], "k": 0})
    info0 = eb.ebof_server_get_info(server)
    if info0.streams_waiting:
        server.close()
        raise RuntimeError("serving: %d of %d streams do not fit the %.0f GB budget with "
                           "batches of %d windows" % (info0.streams_waiting, len(streams),
                                                      cfg.memory_budget / 1e9, max_batch))
    buf = (eb.ebof_completion * 4096)()

    def run(seconds, scale):
        sched = []
        for si, sm in enumerate(streams):
            t, lam = 0.0, sm["rate"] * scale
            while True:
                t += rng.exponential(1.0 / lam)
                if t >= seconds:
                    break
                sched.append((t, si))
        sched.sort()
        t0 = int(lib.ebof_now_ns()) + 20_000_000
        comps = []
        for (toff, si) in sched:
            sm = streams[si]
            ta = t0 + int(toff * 1e9)
            while lib.ebof_now_ns() < ta:
                pass
            k = sm["k"]
            d = sm["seq"][(sm["pos"] + k) % L]
            r = lib.ebof_server_submit(server.handle, sm["sid"], ctypes.byref(d),
                                       sm["flow"][k % len(sm["flow"])], k, ta)
            if r < 0:
                raise eb.EbofError(r, "ebof_server_submit")
            sm["k"] = k + 1
        eb.check(lib.ebof_server_drain(server.handle, 120000), "ebof_server_drain")
        while True:
            n = lib.ebof_server_poll(server.handle, buf, 4096, 0)
            if n <= 0:
                break
            comps += [(buf[i].stream_id, buf[i].status, buf[i].arrival_ns, buf[i].launch_ns,
                       buf[i].done_ns, buf[i].batch) for i in range(n)]
        return sched, t0, comps

    # warm-up: first windows of every stream and the graphs of most batch sizes
    run(args.sv_warmup, 1.0)
    out = {"streams": {"%dx%d" % (W, H): n for (W, H, n, _) in kinds},
           "storage": "fp16", "max_batch": max_batch, "workers": cfg.n_workers,
           "memory_budget_gb": cfg.memory_budget / 1e9,
           "memory_in_use_gb": info0.memory_in_use / 1e9,
           "streams_admitted": info0.streams_admitted,
           "arrivals": "Poisson, per-stream rate U[100, 250] Hz x scale",
           "windows": "each stream cycles through %d generated windows of one of %d "
                      "sequences per resolution" % (L, n_seq),
           "runs": []}
    for scale in args.sv_scales:
        sched, t0, comps = run(args.sv_seconds, scale)
        sid_px = {sm["sid"]: (sm["W"], sm["H"]) for sm in streams}
        ok = [c for c in comps if c[1] >= 0]
        lat = np.asarray([(c[4] - c[2]) / 1e6 for c in ok])
        first = min(c[2] for c in comps)
        last = max(c[4] for c in comps)
        span = (last - first) / 1e9
        px = sum(sid_px[c[0]][0] * sid_px[c[0]][1] for c in ok)
        per_res = {}
        for key in {"%dx%d" % v for v in sid_px.values()}:
            lr = np.asarray([(c[4] - c[2]) / 1e6 for c in ok
                             if "%dx%d" % sid_px[c[0]] == key])
            per_res[key] = {"p50_ms": float(np.percentile(lr, 50)),
                            "p99_ms": float(np.percentile(lr, 99)), "windows": int(len(lr))}
        offered_px = sum(streams[si]["W"] * streams[si]["H"] for (_, si) in sched)
        out["runs"].append({
            "rate_scale": scale, "arrival_seconds": args.sv_seconds,
            "windows": len(comps), "errors": len(comps) - len(ok),
            "offered_windows_per_s": len(sched) / args.sv_seconds,
            "offered_mpx_per_s": offered_px / args.sv_seconds / 1e6,
            "frames_per_s": len(ok) / span, "mpx_per_s": px / span / 1e6,
            "span_s": span, "p50_latency_ms": float(np.percentile(lat, 50)),
            "p99_latency_ms": float(np.percentile(lat, 99)),
            "max_latency_ms": float(lat.max()),
            "mean_batch": float(np.mean([c[5] for c in comps])),
            "latency_by_resolution": per_res})
    bound = args.sv_p99_bound_ms
    ok_runs = [r for r in out["runs"] if r["p99_latency_ms"] <= bound and not r["errors"]]
    out["sustainable"] = {
        "p99_bound_ms": bound,
        "largest_rate_scale": max((r["rate_scale"] for r in ok_runs), default=None),
        "offered_mpx_per_s": max((r["offered_mpx_per_s"] for r in ok_runs), default=None),
        "scales_tried": [r["rate_scale"] for r in out["runs"]],
        "rule": "largest arrival-rate scale whose p99 latency stays within one 10 ms window"}
    server.close()
    del keep
    return out


def run_config0(args, eb, torch, dev, local):
    """The 346x260 single-window workload (seed 0: 40 segments translating at
    (3.0, -1.5) px per window, 20 000 events per window, 5 % noise), plain
    FP32: one ebof_process_window call per window, graph-replayed.  Its two
    windows are fed alternately, so every call after the first is one flow
    frame of the workload (0 -> 1, then 1 -> 0: the same work reversed)."""
    from paper_2112_10591_gb300 import synth
    ev = synth.workload_346x260(seed=0)
    W, H = ev.width, ev.height
    prm = eb.ebof_default_params(W, H)
    st, s = eb.ebof_stream_create(prm, local)
    eb.check(st, "ebof_stream_create 346x260")
    lib = eb.load()
    cs = torch.cuda.current_stream(dev)
    wins = []
    for k in range(2):
        x, y, t, _, tb, te = ev.window(k)
        wins.append((torch.from_numpy(np.ascontiguousarray(x)).to(dev),
                     torch.from_numpy(np.ascontiguousarray(y)).to(dev),
                     torch.from_numpy(np.ascontiguousarray(t)).to(dev), tb, te))
    flow = torch.empty((2, H, W), dtype=torch.float32, device=dev)
    n = max(8, args.c0_windows)

    def call(k):
        x, y, t, tb, te = wins[k & 1]
        r = lib.ebof_process_window(s.handle, x.data_ptr(), y.data_ptr(), t.data_ptr(), None,
                                    x.numel(), tb, te, flow.data_ptr(), None, None, None,
                                    cs.cuda_stream)
        if r < 0:
            raise eb.EbofError(r, "process_window 346x260")

    for k in range(max(3, args.warmup) + 1):
        call(k)
    torch.cuda.synchronize(dev)
    ea = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    eb_ = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(cs)
    for k in range(n):
        ea[k].record(cs)
        call(k)
        eb_[k].record(cs)
    t1.record(cs)
    torch.cuda.synchronize(dev)
    lat = np.asarray([a.elapsed_time(b) for a, b in zip(ea, eb_)])
    total = t0.elapsed_time(t1)
    # the same calls pipelined (each into its own flow buffer of a ring of 8)
    ring = [torch.empty((2, H, W), dtype=torch.float32, device=dev) for _ in range(8)]

    def acall(k):
        x, y, t, tb, te = wins[k & 1]
        r = lib.ebof_process_window_async(s.handle, x.data_ptr(), y.data_ptr(), t.data_ptr(),
                                          None, x.numel(), tb, te, ring[k % 8].data_ptr(),
                                          cs.cuda_stream)
        if r < 0:
            raise eb.EbofError(r, "process_window_async 346x260")

    for k in range(max(3, args.warmup) + 1):
        acall(k)
    eb.check(lib.ebof_stream_join(s.handle, cs.cuda_stream), "join")
    torch.cuda.synchronize(dev)
    t0.record(cs)
    for k in range(n):
        acall(k)
    eb.check(lib.ebof_stream_join(s.handle, cs.cuda_stream), "join")
    t1.record(cs)
    torch.cuda.synchronize(dev)
    ptotal = t0.elapsed_time(t1)
    s.close()
    return {"value": n / (total / 1000.0), "unit": UNIT, "mpx_per_s": n * W * H / total / 1e3,
            "pipelined": {"value": n / (ptotal / 1000.0), "unit": UNIT,
                          "call": "ebof_process_window_async, ebof_stream_join at the end"},
            "p50_latency_ms": float(np.percentile(lat, 50)),
            "p99_latency_ms": float(np.percentile(lat, 99)), "windows_timed": n,
            "levels": prm.levels, "patch": prm.patch, "stride": prm.stride,
            "workload": "346x260, 2 windows of 20 000 events (40 segments at (3.0, -1.5) "
                        "px/window, 5 % noise, seed 0) fed alternately; plain FP32, one "
                        "call per window, inputs resident (L2-resident: 0.5 MB of events)"}


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_2112_10591_gb300 as eb
    from paper_2112_10591_gb300 import synth

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    stream = synth.workload_1280x720(seed=replica_seed(rank), n_windows=args.windows)
    nwin = stream.n_windows
    frames_per_step = nwin - 1
    W, H = stream.width, stream.height
    P = W * H

    # oracle sample (rank 0, N = 1 only) before any GPU work: spawn-safe
    cpu = None
    oracle_flows = None
    prm = eb.ebof_default_params(W, H)
    if rank == 0 and world == 1 and not args.no_cpu:
        workers = cpu_workers()
        nfr = args.cpu_frames or workers
        oracle_flows, dt = oracle_sample(stream, _params_dict(prm), nfr, workers)
        cpu = {"value": nfr / dt, "unit": UNIT, "cores": workers, "kind": "oracle",
               "host_cores": os.cpu_count(),
               "sample": "%d frame pairs (windows 0..%d) of the 1280x720 stream, one per "
                         "process, FP64, %.1f s wall" % (nfr, nfr, dt),
               "single_thread": oracle_single_thread(stream, _params_dict(prm))}

    eb.load()
    xs = torch.from_numpy(stream.x).to(dev)
    ys = torch.from_numpy(stream.y).to(dev)
    ts = torch.from_numpy(stream.t).to(dev)
    ps = torch.from_numpy(stream.p).to(dev)
    off = [int(v) for v in stream.offsets]
    tb = [int(v) for v in stream.t_begin]
    flows = torch.empty((nwin, 2, H, W), dtype=torch.float32, device=dev)
    st, s = eb.ebof_stream_create(prm, local)
    eb.check(st, "ebof_stream_create")
    cs = torch.cuda.current_stream(dev)
    handle = cs.cuda_stream
    lib = eb.load()

    def step_plain(ev_a=None, ev_b=None):
        eb.check(lib.ebof_stream_reset(s.handle), "reset")
        for k in range(nwin):
            a, b = off[k], off[k + 1]
            if ev_a is not None:
                ev_a[k].record(cs)
            r = lib.ebof_process_window(
                s.handle, xs.data_ptr() + 2 * a, ys.data_ptr() + 2 * a, ts.data_ptr() + 8 * a,
                ps.data_ptr() + a, b - a, tb[k], tb[k] + stream.dt, flows[k].data_ptr(),
                None, None, None, handle)
            if r < 0:
                raise eb.EbofError(r, "process_window")
            if ev_b is not None:
                ev_b[k].record(cs)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step_plain()
    barrier()
    evs_a = [torch.cuda.Event(enable_timing=True) for _ in range(nwin)]
    evs_b = [torch.cuda.Event(enable_timing=True) for _ in range(nwin)]
    lat = []
    clk = ClockSampler(local)
    clk.start()
    launches0 = eb.ebof_kernel_launches()
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    t_start.record(cs)
    for i in range(args.steps):
        step_plain(evs_a, evs_b)
        if i + 1 < args.steps:  # keep the per-window events of this step
            torch.cuda.synchronize(dev)
            lat += [evs_a[k].elapsed_time(evs_b[k]) for k in range(1, nwin)]
    t_end.record(cs)
    barrier()
    wall = time.perf_counter() - w0
    lat += [evs_a[k].elapsed_time(evs_b[k]) for k in range(1, nwin)]
    launches_in_order = eb.ebof_kernel_launches() - launches0
    ms_in_order, value_in_order = combine_ranks(t_start.elapsed_time(t_end),
                                                frames_per_step * args.steps, world, dist, dev)

    # the same windows through the pipelined call: each window's front end
    # overlaps the previous window's flow levels; the timed region on the
    # caller's stream is closed by ebof_stream_join
    def step_pipelined():
        eb.check(lib.ebof_stream_reset(s.handle), "reset")
        for k in range(nwin):
            a, b = off[k], off[k + 1]
            r = lib.ebof_process_window_async(
                s.handle, xs.data_ptr() + 2 * a, ys.data_ptr() + 2 * a, ts.data_ptr() + 8 * a,
                ps.data_ptr() + a, b - a, tb[k], tb[k] + stream.dt, flows[k].data_ptr(), handle)
            if r < 0:
                raise eb.EbofError(r, "process_window_async")
        eb.check(lib.ebof_stream_join(s.handle, handle), "join")

    for _ in range(args.warmup):
        step_pipelined()
    barrier()
    p_start = torch.cuda.Event(enable_timing=True)
    p_end = torch.cuda.Event(enable_timing=True)
    launches0 = eb.ebof_kernel_launches()
    p_start.record(cs)
    for _ in range(args.steps):
        step_pipelined()
    p_end.record(cs)
    barrier()
    launches = eb.ebof_kernel_launches() - launches0
    clocks = clk.stop()
    # `value`: the pipelined calls; `in_order`: each window's stages in order
    # on the caller's stream (the latencies above)
    ms, value = combine_ranks(p_start.elapsed_time(p_end), frames_per_step * args.steps,
                              world, dist, dev)
    in_order = {"value": value_in_order, "unit": UNIT, "ms_per_step": ms_in_order / args.steps,
                "gpu_launches": int(launches_in_order),
                "call": "ebof_process_window per window: every stage of a window in order on "
                        "the caller's stream, one CUDA graph replay per window"}

    # stage profile over the same steps (events bracket each stage's launches)
    eb.check(eb.ebof_stream_set_profiling(s, True))
    nprof = max(1, min(args.steps, 2))
    for _ in range(nprof):
        step_plain()
    torch.cuda.synchronize(dev)
    pst, prof = eb.ebof_stream_get_profile(s)
    eb.check(pst)
    _, prof0 = eb.ebof_stream_get_profile_level(s, 0)
    _, profn = eb.ebof_stream_get_profile_level(s, -1)
    by_level = {}
    for lvl in [-1] + list(range(prm.levels)):
        _, pl = eb.ebof_stream_get_profile_level(s, lvl)
        by_level["all" if lvl < 0 else str(lvl)] = {
            k: round(v[0] / (nwin * nprof), 4) for k, v in pl.items() if v[1]}
    eb.ebof_stream_set_profiling(s, False)
    total_ms = sum(v[0] for v in prof.values()) or 1.0
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0]
    level = 0 if dom in PER_LEVEL else -1
    dom_ms, dom_launches = (prof0 if level == 0 else profn)[dom]
    gl = geo_levels(prm)
    n_ev_win = int(off[-1]) / nwin
    per_launch_bytes = algorithmic_bytes_per_launch(dom, level, gl, n_ev_win, P)
    per_launch_s = dom_ms / 1000.0 / max(dom_launches, 1)
    achieved = per_launch_bytes / per_launch_s / 1e9
    peak, peak_kind = load_peaks()
    kernel_io = {"kernel": dom, "level": level, "achieved": achieved, "unit": "GB/s",
                 "frac": achieved / peak, "traffic": dram_traffic(dom, level),
                 "bytes_per_launch": per_launch_bytes, "us_per_launch": per_launch_s * 1e6,
                 "launches_timed": int(dom_launches),
                 "bytes_rule": "the kernel's own inputs read once and outputs written once"}
    ms_frame = {k: v[0] / (nwin * nprof) for k, v in prof.items() if v[1]}
    roofline = a8_outer_iteration_roofline(by_level.get("0", {}), P, prm.var_outer, nwin * nprof,
                                           peak, dram_traffic("var_coeff", 0),
                                           dram_traffic("var_sor", 0)) or {}
    roofline.update({
        "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs; burst copy)",
        "kernel_io": kernel_io,
        "stage_roofline": stage_hbm_fractions(ms_frame, P, n_ev_win, len(gl), prm.var_outer,
                                              peak),
        "stage_share": {k: round(v[0] / total_ms, 4) for k, v in prof.items()},
        "stage_ms_per_frame": {k: round(v, 4) for k, v in ms_frame.items()},
        "stage_ms_per_frame_by_level": by_level,
        "stage_timing": "CUDA events around each stage's launches on the caller's stream "
                        "(eager launches, gaps included; the graph-replayed path times "
                        "the whole window only)"})
    # the whole path at the pipelined rate: every stage's algorithmic bytes
    # per frame times the frames per second of `value`
    allb = roofline["stage_roofline"].get("all stages", {}).get("bytes_per_frame")
    if allb:
        roofline["pipelined_all_stages"] = {
            "bytes_per_frame": allb, "frames_per_s": value,
            "achieved_gbs": round(allb * value / 1e9, 1),
            "frac": round(allb * value / 1e9 / peak, 4)}

    # batched path: the same stream through ebof_process_windows
    batched = None
    B = max(1, min(args.batch, nwin - 1))
    if B > 1:
        pb = eb.ebof_default_params(W, H)
        pb.max_batch = B
        stb, sb = eb.ebof_stream_create(pb, local)
        if stb >= 0:
            def step_batched():
                eb.check(lib.ebof_stream_reset(sb.handle), "reset")
                k = 0
                while k < nwin:
                    n = min(B, nwin - k)
                    a, b = off[k], off[k + n]
                    r = lib.ebof_process_windows(
                        sb.handle, n, xs.data_ptr() + 2 * a, ys.data_ptr() + 2 * a,
                        ts.data_ptr() + 8 * a, ps.data_ptr() + a, b - a, tb[k], stream.dt,
                        flows[k].data_ptr(), None, None, None, handle)
                    if r < 0:
                        raise eb.EbofError(r, "process_windows")
                    k += n
            for _ in range(args.warmup):
                step_batched()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cs)
            for _ in range(args.steps):
                step_batched()
            e1.record(cs)
            barrier()
            bms, bval = combine_ranks(e0.elapsed_time(e1), frames_per_step * args.steps, world,
                                      dist, dev)
            eb.check(eb.ebof_stream_set_profiling(sb, True))
            step_batched()
            torch.cuda.synchronize(dev)
            _, bprof = eb.ebof_stream_get_profile(sb)
            eb.ebof_stream_set_profiling(sb, False)
            btot = sum(v[0] for v in bprof.values()) or 1.0
            batched = {"value": bval,
                       "unit": UNIT, "windows_per_call": B,
                       "ms_per_step": bms / args.steps,
                       "stage_ms_per_frame": {k: round(v[0] / frames_per_step, 4)
                                              for k, v in bprof.items() if v[1]},
                       "stage_share": {k: round(v[0] / btot, 4) for k, v in bprof.items()
                                       if v[1]}}
            batched["stage_roofline"] = stage_hbm_fractions(
                {k: v[0] / frames_per_step for k, v in bprof.items() if v[1]}, P, n_ev_win,
                len(gl), prm.var_outer, peak)
            sb.close()
            # the same batches with FP16 storage of surfaces, pyramids and gradients
            pb.storage = eb.EBOF_STORAGE_FP16
            st16b, sb = eb.ebof_stream_create(pb, local)
            if st16b >= 0:
                for _ in range(args.warmup):
                    step_batched()
                barrier()
                e0.record(cs)
                for _ in range(args.steps):
                    step_batched()
                e1.record(cs)
                barrier()
                hms, hval = combine_ranks(e0.elapsed_time(e1), frames_per_step * args.steps,
                                          world, dist, dev)
                batched["fp16_storage"] = {"value": hval, "unit": UNIT,
                                           "ms_per_step": hms / args.steps}
                sb.close()
        else:
            batched = {"unavailable": eb.ebof_status_string(stb)}

    # EPE of the GPU flow against the oracle sample (same windows)
    epe = None
    nchk = min(len(oracle_flows) if oracle_flows is not None else 8, nwin - 1)
    step_plain()
    torch.cuda.synchronize(dev)
    flows32 = [flows[k + 1].cpu().numpy() for k in range(nchk)]
    if oracle_flows is not None:
        e = np.stack([np.hypot(g[0] - U[0], g[1] - U[1])
                      for g, U in zip(flows32, oracle_flows[:nchk])])
        epe = {"mean_px": float(e.mean()), "p99_px": float(np.percentile(e, 99)),
               "frames": len(flows32)}

    # flow quality without ground truth: the Flow Warping Loss (§IV-C) of
    # every flow frame of the stream, on the events of its window
    scr = torch.empty(eb.ebof_fwl_scratch_bytes(W, H), dtype=torch.uint8, device=dev)
    fwl_out = torch.zeros((nwin, 3), dtype=torch.float64, device=dev)
    for k in range(1, nwin):
        a, b = off[k], off[k + 1]
        eb.check(lib.ebof_fwl(xs.data_ptr() + 2 * a, ys.data_ptr() + 2 * a,
                              ts.data_ptr() + 8 * a, ps.data_ptr() + a, b - a, tb[k],
                              tb[k] + stream.dt, flows[k].data_ptr(), W, H, scr.data_ptr(),
                              fwl_out[k].data_ptr(), handle), "ebof_fwl")
    torch.cuda.synchronize(dev)
    fw = fwl_out[1:, 0].cpu().numpy()
    quality = {"fwl_mean": float(fw.mean()), "fwl_min": float(fw.min()),
               "fwl_max": float(fw.max()), "frames_fwl_above_1": float((fw > 1.0).mean()),
               "frames": int(len(fw)),
               "note": "FWL = var(events moved back along the flow) / var(events unmoved), "
                       "with polarity; > 1 beats the zero flow"}
    del scr
    quality["vs_ground_truth"] = ground_truth_quality(eb, torch, dev, local)

    # FP16 storage of surfaces, pyramid levels and gradients (same stream)
    fp16 = None
    p16 = eb.ebof_default_params(W, H)
    p16.storage = eb.EBOF_STORAGE_FP16
    st16, s16 = eb.ebof_stream_create(p16, local)
    if st16 >= 0:
        def step_plain16():
            eb.check(lib.ebof_stream_reset(s16.handle), "reset")
            for k in range(nwin):
                a, b = off[k], off[k + 1]
                r = lib.ebof_process_window(
                    s16.handle, xs.data_ptr() + 2 * a, ys.data_ptr() + 2 * a,
                    ts.data_ptr() + 8 * a, ps.data_ptr() + a, b - a, tb[k], tb[k] + stream.dt,
                    flows[k].data_ptr(), None, None, None, handle)
                if r < 0:
                    raise eb.EbofError(r, "process_window fp16")
        for _ in range(args.warmup):
            step_plain16()
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(cs)
        for _ in range(args.steps):
            step_plain16()
        f1.record(cs)
        barrier()
        fms, fval = combine_ranks(f0.elapsed_time(f1), frames_per_step * args.steps, world,
                                  dist, dev)
        flows16 = [flows[k + 1].cpu().numpy() for k in range(nchk)]
        e16 = np.stack([np.hypot(a[0] - b[0], a[1] - b[1]) for a, b in zip(flows16, flows32)])
        fp16 = {"value": fval, "unit": UNIT, "ms_per_step": fms / args.steps,
                "epe_vs_fp32_gpu": {"mean_px": float(e16.mean()),
                                    "p99_px": float(np.percentile(e16, 99)), "frames": nchk}}
        if oracle_flows is not None:
            eo = np.stack([np.hypot(a[0] - U[0], a[1] - U[1])
                           for a, U in zip(flows16, oracle_flows[:nchk])])
            fp16["epe_vs_oracle"] = {"mean_px": float(eo.mean()),
                                     "p99_px": float(np.percentile(eo, 99)), "frames": nchk}
        s16.close()

    # end-to-end through the host-buffer call
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(stream.x).pin_memory().numpy()
        hy = torch.from_numpy(stream.y).pin_memory().numpy()
        ht = torch.from_numpy(stream.t).pin_memory().numpy()
        hflow = torch.empty((2, H, W), dtype=torch.float32).pin_memory().numpy()

        def step_host():
            eb.check(lib.ebof_stream_reset(s.handle), "reset")
            for k in range(nwin):
                a, b = off[k], off[k + 1]
                r = lib.ebof_process_window_host(
                    s.handle, hx.ctypes.data + 2 * a, hy.ctypes.data + 2 * a,
                    ht.ctypes.data + 8 * a, b - a, tb[k], tb[k] + stream.dt, hflow.ctypes.data,
                    handle)
                if r < 0:
                    raise eb.EbofError(r, "process_window_host")

        # streaming: every window enqueued without waiting (its kernels read
        # the pinned events and write the flow into a ring of 8 pinned host
        # buffers in place), one synchronisation per step
        hring = [torch.empty((2, H, W), dtype=torch.float32).pin_memory().numpy()
                 for _ in range(8)]

        def step_host_async():
            eb.check(lib.ebof_stream_reset(s.handle), "reset")
            for k in range(nwin):
                a, b = off[k], off[k + 1]
                r = lib.ebof_process_window_host_async(
                    s.handle, hx.ctypes.data + 2 * a, hy.ctypes.data + 2 * a,
                    ht.ctypes.data + 8 * a, b - a, tb[k], tb[k] + stream.dt,
                    hring[k % 8].ctypes.data, handle)
                if r < 0:
                    raise eb.EbofError(r, "process_window_host_async")
            eb.check(lib.ebof_stream_sync(s.handle, None, 0), "sync")

        def timed_host(step):
            for _ in range(min(args.warmup, 1)):
                step()
            barrier()
            h0 = time.perf_counter()
            for _ in range(args.steps):
                step()
            barrier()
            return combine_ranks(1000.0 * (time.perf_counter() - h0),
                                 frames_per_step * args.steps, world, dist, dev)

        _, hval_sync = timed_host(step_host)
        hms, hval = timed_host(step_host_async)
        e2e = {"value": hval, "unit": UNIT,
               "h2d_bytes_per_step": int(off[-1]) * 12,
               "d2h_bytes_per_step": nwin * 2 * P * 4,
               "call": "ebof_process_window_host_async per window (pinned events read and "
                       "flows written in place by the kernels), one ebof_stream_sync per step",
               "synchronous_per_window": {
                   "value": hval_sync, "unit": UNIT,
                   "call": "ebof_process_window_host per window (returns after its "
                           "stream synchronises)"}}

    roofline["a6_patch_search"] = a6_flop_roof(by_level, gl, prm.patch, prm.gn_iters,
                                               clocks.get("sm_mhz"))
    config0 = None if args.no_config0 else run_config0(args, eb, torch, dev, local)

    multistream = None if args.no_multistream else run_multistream(args, eb, torch, dev, rank)
    serving = None if args.no_serving else run_serving(args, eb, torch, dev, rank)

    if rank == 0:
        lat = np.asarray(lat)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(_params_dict(prm), nwin, world),
            "path": "one window per call, pipelined (ebof_process_window_async: a window's "
                    "front end on one internal stream, its flow on one of four flow "
                    "streams in turn, so that front ends and the flows of four "
                    "consecutive windows overlap; graph replays; ebof_stream_join closes "
                    "the step); latencies from in-order ebof_process_window calls",
            "events_mb_per_step": int(off[-1]) * 13 / 1e6,
            "p50_latency_ms": float(np.percentile(lat, 50)),
            "p99_latency_ms": float(np.percentile(lat, 99)),
            "mpx_per_s": value * P / 1e6,
            "wall_s": wall,
            "in_order": in_order,
            "batched": batched,
            "config0_346x260": config0,
            "epe_vs_oracle": epe,
            "flow_quality": quality,
            "fp16_storage": fp16,
            "multistream": multistream,
            "serving": serving,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
