#!/usr/bin/env python3
"""SAFR per-frame reconstruction benchmark (GB300, sm_103a).

Workload: the MORFEO-like frame: 39 m aperture, 80x80 pupil samples
zero-padded to a 256x256 grid, 6 LGS (90 km, 2 arcmin ring) + 3 NGS
(1.3 arcmin), 9 layers 0-16 km, FP32, batch 1, synthetic von Karman
wavefronts (seeded).  One step = one frame through safr_reconstruct (pad +
row FFT, column FFT + apply + inverse column FFT, inverse row FFT + resample
+ store).

  value         frames/s of --steps frames submitted back to back (no host
                synchronisation between frames) over a pool of --pool plans of
                the workload, whose B (21 MB each) together exceed the L2: every
                frame reads its B from HBM.  CUDA events bracket the run.
  latency_10k   per-frame latency of --latency-frames frames (default 10 000,
                as many as the paper's loop simulation runs), CUDA events around
                each frame, the L2 (129 MB) flushed before every frame by writing
                a 256 MB buffer and then reading another one.
  warm_L2       the same back-to-back frames on one plan (B stays in the L2),
                against the L2/HBM roofline bytes_B / BW_L2 + bytes_io / BW_HBM,
                BW_L2 measured here from a plain L2-resident copy.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl safr|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs its own replica
(frame-parallel, no collective on the data path) and rank 0 prints the line.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SAFR frames/s & p99 latency (MORFEO-like, FP32) vs FP64 oracle, % roofline"
UNIT = "frames/s"
WORKLOAD = "morfeo-256"
FLUSH_BYTES = 256 << 20
REF_BUDGET_S = 120.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="safr", choices=["safr", "reference"])
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--pool", type=int, default=8, help="plans cycled by the back-to-back frames (B from HBM)")
    ap.add_argument("--latency-frames", type=int, default=10000, help="frames of the flushed latency run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", default="auto", choices=["auto", "fused", "passes"])
    ap.add_argument("--no-workloads", action="store_true", help="skip the secondary workloads (32-grid, 512-grid, batched, learned filter, loop step, refresh)")
    ap.add_argument("--workloads", default="all",
                    help="comma-separated secondary workloads to run (tiny, fp16-512, batch, learned, loop, refresh), "
                         "or 'all'")
    return ap.parse_args()


# the sources the persistent frame kernel is compiled from (its counters go stale when one changes)
FRAME_KERNEL_SOURCES = ("common.cuh", "frame.cu", "frame_dispatch.cuh", "frame_f16.cu", "frame_f32.cu",
                        "frame_f64.cu", "frame_impl.cuh", "freqorder.h", "plan.h", "warpfft.cuh")


def csrc_sha256() -> str:
    """sha256 over the frame kernel's sources (file name and bytes, sorted by name)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2510_19542_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(FRAME_KERNEL_SOURCES):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def config_block(g, pool=1):
    return {"workload": WORKLOAD, "grid": g["M"], "pupil": g["P"], "lgs": int(np.sum(g["kind"] == 1)),
            "ngs": int(np.sum(g["kind"] == 0)), "layers": len(g["h"]), "batch": 1,
            "precision": "fp32",
            "l2": (f"value: inputs larger than the L2 (frames back to back over {pool} plans, {pool} x 21 MB "
                   "of B); latency: flushed before every frame (256 MB written, then 256 MB read)")}


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# oracle (CPU) timing
# ----------------------------------------------------------------------------
def oracle_frames(geom, frames, budget_s, max_frames):
    import oracle
    oracle.build()
    pl = oracle.OraclePlan(geom)
    t0 = time.perf_counter()
    n = 0
    outs = {}
    while n < max_frames:
        outs[n % len(frames)] = pl.reconstruct(frames[n % len(frames)])
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n, dt, oracle.threads(), outs


def run_reference(args):
    from paper_2510_19542_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g = synth.config(2)
    frames = [synth.frame(g, seed=100 + i) for i in range(2)]
    import oracle
    oracle.build()
    pl = oracle.OraclePlan(g)
    for i in range(min(args.warmup, 1)):
        pl.reconstruct(frames[i % 2])
    t0 = time.perf_counter()
    done = 0
    for i in range(args.steps):
        pl.reconstruct(frames[i % 2])
        done += 1
        if time.perf_counter() - t0 > REF_BUDGET_S:
            break
    dt = time.perf_counter() - t0
    val = done / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": done, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / done, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic von Karman frames (seeded)", "config": config_block(g, args.pool),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{done} full frames of the workload (FP64 oracle: naive DFT2, "
                                       "Jacobi-SVD B precomputed once, untimed); warm-up "
                                       f"{min(args.warmup, 1)} frame; steps stop after {REF_BUDGET_S:.0f} s"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def layer_errors(got, ref):
    """(overall relative L2 error, [error of each layer relative to its own RMS])."""
    diff = got - ref
    overall = float(np.linalg.norm(diff) / np.linalg.norm(ref))
    own = np.sqrt(np.mean(diff ** 2, axis=(1, 2))) / np.maximum(np.sqrt(np.mean(ref ** 2, axis=(1, 2))), 1e-300)
    return overall, [float(v) for v in own]


# ----------------------------------------------------------------------------
# secondary workloads (same protocol, reported inside the main line)
# ----------------------------------------------------------------------------
def measure_workload(safr, synth, torch, dev, stream, k, steps, warmup, flush_l2, hbm):
    """frames/s, p50/p99 latency and error against the FP64 oracle for workload k:
    1 = 32 grid, 3 NGS, 3 layers, FP64; 3 = 512 grid, 3 NGS, 35 layers, FP16
    storage.  Every output is compared with the full oracle, overall and per
    layer (each layer's error relative to its own RMS)."""
    import oracle
    g = synth.config(k)
    prec = g["precision"]
    x = synth.frame(g, seed=200 + k)
    plan = safr.Plan(g, device=dev.index)
    info = plan.info
    if prec == "fp16":
        h, sc = synth.to_fp16_storage(x)
        xin = torch.from_numpy(h).to(dev)
        isc = torch.from_numpy(sc).to(dev)
        osc = torch.empty(info["L"], dtype=torch.float32, device=dev)
        x_or = synth.from_fp16_storage(h, sc)
    else:
        xin = torch.from_numpy(x.astype(np.float64 if prec == "fp64" else np.float32)).to(dev)
        isc, osc, x_or = None, None, x
    layers = plan.empty_layers()

    def one(i):
        flush_l2(i)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        safr.safr_reconstruct(plan.handle, xin, layers, in_scales=isc, out_scales=osc, stream=stream)
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e)

    for i in range(warmup):
        one(i)
    lat = sorted(one(i) for i in range(steps))
    got = layers.double().cpu().numpy()
    if osc is not None:
        got = got * osc.double().cpu().numpy()[:, None, None]
    ref = oracle.OraclePlan(g).reconstruct(x_or)
    err, own = layer_errors(got, ref)
    what = "all outputs (full FP64 oracle)"
    es = {"fp64": 8, "fp32": 4, "fp16": 2}[prec]
    M = info["M"]
    fbytes = (M * (M // 2) * info["L"] * info["G"] * (16 if prec == "fp64" else 8)
              + info["G"] * info["P"] ** 2 * es + info["L"] * M * M * es)
    mean_ms = float(np.mean(lat))
    out = {"grid": M, "pupil": info["P"], "stars": info["G"], "layers": info["L"], "precision": prec,
           "frames_per_s": 1e3 / mean_ms, "latency_ms": {"p50": lat[len(lat) // 2],
                                                         "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
           "path": {safr.SAFR_PATH_FUSED: "fused", safr.SAFR_PATH_PASSES: "passes",
                    safr.SAFR_PATH_CLUSTER: "cluster"}[safr.safr_get_path(plan.handle)],
           "algorithmic_bytes": fbytes, "frac_of_hbm": fbytes / (mean_ms * 1e-3) / 1e9 / hbm,
           "rel_l2_vs_oracle": err, "rel_l2_per_layer_own": own, "rel_l2_per_layer_own_max": max(own),
           "compared": what, "steps": steps}
    plan.close()
    return g["name"], out


def measure_batch(safr, synth, torch, dev, stream, steps, warmup, flush_l2, hbm, n=64):
    """The batched workload: n frames of uneven geometry (seeded), one plan per
    frame, autotuned, reconstructed by one safr_batch_reconstruct per step (one
    CUDA graph launch of the frames' own launches).  Beside it, the same frames
    submitted one by one through safr_reconstruct."""
    geoms = synth.batch_configs(n=n, seed=4)
    plans = [safr.Plan(g, device=dev.index) for g in geoms]
    for p in plans:
        safr.safr_autotune(p.handle, stream)
    xs = [torch.from_numpy(synth.random_frame(g, 4000 + f).astype(np.float32)).to(dev) for f, g in enumerate(geoms)]
    outs = [p.empty_layers() for p in plans]
    batch = safr.safr_batch_create([p.handle for p in plans])

    def timed(fn, i):
        flush_l2(i)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e)

    run_batch = lambda: safr.safr_batch_reconstruct(batch, xs, outs, stream=stream)  # noqa: E731

    def run_seq():
        for p, x, o in zip(plans, xs, outs):
            safr.safr_reconstruct(p.handle, x, o, stream=stream)

    for i in range(warmup):
        timed(run_batch, i)
        timed(run_seq, i)
    tb = [timed(run_batch, i) for i in range(steps)]
    ts = [timed(run_seq, i) for i in range(steps)]
    # every frame of the batch equals its frame-by-frame result
    run_batch()
    torch.cuda.synchronize(dev)
    got = [o.clone() for o in outs]
    run_seq()
    torch.cuda.synchronize(dev)
    same = all(torch.equal(a, b) for a, b in zip(got, outs))
    status = safr.safr_batch_get_status(batch)
    # reconstruction error of the batched form: per distinct grid size, the batch frame with the
    # fewest layers (the oracle's cost grows with L) against the full FP64 oracle
    import oracle
    run_batch()
    torch.cuda.synchronize(dev)
    err_by_grid = {}
    for M in sorted({g["M"] for g in geoms}):
        f = min((i for i, g in enumerate(geoms) if g["M"] == M), key=lambda i: (len(geoms[i]["h"]), i))
        ref = oracle.OraclePlan(geoms[f]).reconstruct(synth.random_frame(geoms[f], 4000 + f).astype(np.float32))
        overall, own = layer_errors(outs[f].double().cpu().numpy(), ref)
        err_by_grid[str(M)] = {"frame": f, "stars": len(geoms[f]["dir_x"]), "layers": len(geoms[f]["h"]),
                               "rel_l2_vs_oracle": overall, "rel_l2_per_layer_own_max": max(own)}
    nbytes = 0
    for p in plans:
        i = p.info
        M = i["M"]
        nbytes += M * (M // 2) * i["L"] * i["G"] * 8 + i["G"] * i["P"] ** 2 * 4 + i["L"] * M * M * 4
    paths = [safr.safr_get_plan_info(p.handle)["path"] for p in plans]
    mb, ms = float(np.mean(tb)), float(np.mean(ts))
    out = {"frames": n, "grids": sorted({g["M"] for g in geoms}), "stars": [3, 9], "layers": [3, 35],
           "precision": "fp32", "frames_per_s": n / (mb * 1e-3), "ms_per_batch": mb,
           "launches_per_batch": safr.safr_batch_launches(batch), "graph": safr.safr_batch_graph(batch),
           "concurrent_chains": safr.safr_batch_chains(batch),
           "autotuned_paths": {
               "fused": paths.count(safr.SAFR_PATH_FUSED), "passes": paths.count(safr.SAFR_PATH_PASSES)},
           "algorithmic_bytes_per_batch": nbytes, "frac_of_hbm": nbytes / (mb * 1e-3) / 1e9 / hbm,
           "one_by_one": {"frames_per_s": n / (ms * 1e-3), "ms_per_batch": ms},
           "equals_frame_by_frame": bool(same), "rel_l2_vs_oracle_by_grid": err_by_grid,
           "autotuned": "per plan: schedule (persistent kernel or three passes) and phase-3 tile height; "
                        "per batch: concurrent chains K in {1, 2, 4, 8}.  The FFT radix is not tuned: it is "
                        "fixed by the warp structure (32 lanes x M/32 values per lane, radix-2 lane stages)",
           "device_status": status, "steps": steps,
           "l2": "flushed before every timed batch"}
    safr.safr_batch_destroy(batch)
    for p in plans:
        p.close()
    return "batched-64-uneven", out


def measure_loop(safr, synth, torch, dev, stream, steps, warmup, flush_l2, hbm):
    """One AO-loop iteration of Algorithm 3 around SAFR on the MORFEO-like
    geometry: POLC of the wavefronts with the mirror/layer state, the SAFR frame
    (LGS tip/tilt removal included), and the integrator (gain 0.5), through
    safr_loop_step; beside it each step alone.  L2 flushed before every call."""
    g = synth.config(2)
    plan = safr.Plan(g, device=dev.index)
    info = plan.info
    L, M, G, P = info["L"], info["M"], info["G"], info["P"]
    x = torch.from_numpy(synth.frame(g, seed=700).astype(np.float32)).to(dev)
    a = torch.zeros((L, M, M), dtype=torch.float32, device=dev)
    tmp = torch.empty((G, P, P), dtype=torch.float32, device=dev)
    phi = plan.empty_layers().zero_()

    def timed(fn, i):
        flush_l2(i)
        s0 = torch.cuda.Event(enable_timing=True)
        e0 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        fn()
        e0.record(stream)
        e0.synchronize()
        return s0.elapsed_time(e0)

    step = lambda: safr.safr_loop_step(plan.handle, x, a, 0.5, stream=stream)  # noqa: E731
    polc = lambda: safr.safr_polc(plan.handle, x, a, tmp, stream=stream)  # noqa: E731
    integ = lambda: safr.safr_integrate(plan.handle, phi, a, 0.5, stream=stream)  # noqa: E731
    for i in range(warmup):
        timed(step, i)
    lat = sorted(timed(step, i) for i in range(steps))
    t_polc = float(np.median([timed(polc, i) for i in range(20)]))
    t_int = float(np.median([timed(integ, i) for i in range(20)]))
    status = safr.safr_get_status(plan.handle)
    nbytes = M * (M // 2) * L * G * 8 + G * P * P * 4 + 2 * L * M * M * 4  # B, wavefronts, state read + write
    mean_ms = float(np.mean(lat))
    out = {"grid": M, "pupil": P, "stars": G, "layers": L, "precision": "fp32", "gain": 0.5,
           "frames_per_s": 1e3 / mean_ms,
           "latency_ms": {"p50": lat[len(lat) // 2],
                          "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
           "launches_per_step": 1 if safr.safr_get_path(plan.handle) == safr.SAFR_PATH_FUSED else
           2 + safr.safr_launches_per_frame(plan.handle),
           "fusion": "POLC as phase 0 and the integrator in the store of the frame kernel"
           if safr.safr_get_path(plan.handle) == safr.SAFR_PATH_FUSED else "separate kernels",
           "polc_ms": t_polc, "integrate_ms": t_int,
           "algorithmic_bytes": nbytes, "frac_of_hbm": nbytes / (mean_ms * 1e-3) / 1e9 / hbm,
           "device_status": status, "steps": steps}
    plan.close()
    return "loop-step-morfeo-256", out


def measure_refresh(safr, synth, torch, dev, stream, steps):
    """Soft real-time refresh of B on the MORFEO-like plan: safr_refresh with a
    new alpha, and with a rotated asterism and a new Cn2 profile (tables copied,
    Algorithm 2 rerun in place), timed with CUDA events on the stream; the
    plan file round trip timed on the host."""
    import tempfile
    import time
    g = synth.config(2)
    plan = safr.Plan(g, device=dev.index)
    rng = np.random.default_rng(12)

    def timed(fn):
        s0 = torch.cuda.Event(enable_timing=True)
        e0 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        fn()
        e0.record(stream)
        e0.synchronize()
        return s0.elapsed_time(e0)

    def new_asterism():
        rot = rng.uniform(-0.05, 0.05)
        dx, dy = np.asarray(g["dir_x"]), np.asarray(g["dir_y"])
        return dict(cn2=np.asarray(g["cn2"]) * rng.uniform(0.8, 1.2, len(g["h"])),
                    dir_x=np.cos(rot) * dx - np.sin(rot) * dy, dir_y=np.sin(rot) * dx + np.cos(rot) * dy)

    for _ in range(3):
        timed(lambda: safr.safr_refresh(plan.handle, alpha=g["alpha"], stream=stream))
    t_alpha = sorted(timed(lambda: safr.safr_refresh(plan.handle, alpha=g["alpha"] * rng.uniform(0.5, 2), stream=stream))
                     for _ in range(steps))
    t_geo = sorted(timed(lambda: safr.safr_refresh(plan.handle, stream=stream, **new_asterism()))
                   for _ in range(steps))
    t_pre = sorted(timed(lambda: safr.safr_precompute(plan.handle, stream)) for _ in range(steps))
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "morfeo.safr")
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        safr.safr_plan_save(plan.handle, path)
        t_save = time.perf_counter() - t0
        size = os.path.getsize(path)
        t0 = time.perf_counter()
        q = safr.Plan.load(path, dev.index)
        torch.cuda.synchronize(dev)
        t_load = time.perf_counter() - t0
        same = bool(np.array_equal(safr.safr_copy_B(q.handle, 0), safr.safr_copy_B(plan.handle, 0)))
        q.close()
    plan.close()
    med = lambda v: float(v[len(v) // 2])  # noqa: E731
    return "refresh-morfeo-256", {
        "refresh_alpha_ms": {"p50": med(t_alpha), "max": float(t_alpha[-1])},
        "refresh_asterism_and_profile_ms": {"p50": med(t_geo), "max": float(t_geo[-1])},
        "precompute_only_ms": {"p50": med(t_pre)},
        "plan_file": {"bytes": size, "save_ms": t_save * 1e3, "load_ms": t_load * 1e3, "B_identical": same},
        "steps": steps}


def measure_learned(safr, synth, torch, dev, stream, steps, warmup, flush_l2):
    """The learned spectral filter on the 32-grid geometry with 35 layers: GPU
    training on 100k forward-model frames (2 epochs), the held-out comparison
    with plain SAFR, the time to rebuild B from the weights, frames with the
    learned B (the same frame kernel), the learned B against the FP64 oracle,
    and the layer error against the true screens of 8 synthetic frames for both
    filters."""
    import time

    import oracle
    g = synth.config(5)
    plan = safr.Plan(g, device=dev.index)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    w, res = safr.safr_filter_train(plan.handle, g["r0"], g["L0"], g["noise"], 100000, 4096, 2, lr=1e-3, seed=5,
                                    stream=stream)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    used = res["used_learned"]
    ta = []
    for _ in range(5):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        safr.safr_filter_apply(plan.handle, w, g["noise"], stream=stream)
        ta.append((time.perf_counter() - t0) * 1e3)
    # the learned B against the oracle's, from the same BF16 parameters
    M = g["M"]
    cn2 = np.asarray(g["cn2"], np.float64)
    Bo = oracle.group_B_learned(M, M * g["pitch"] / 2.0, np.asarray(g["h"], np.float64), np.ones(len(g["h"])),
                                cn2 / cn2.sum(), np.asarray(g["dir_x"], np.float64),
                                np.asarray(g["dir_y"], np.float64), g["beta"], w.astype(np.float64), g["noise"])
    Bo = np.transpose(Bo[:, :M // 2], (1, 2, 3, 0))
    Bg = safr.safr_copy_B(plan.handle, 0)
    b_err = float(np.abs(Bg - Bo).max() / np.abs(Bo).max())
    # frames with the learned B
    xin = torch.from_numpy(synth.frame(g, seed=600).astype(np.float32)).to(dev)
    layers = plan.empty_layers()

    def one(i):
        flush_l2(i)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        safr.safr_reconstruct(plan.handle, xin, layers, stream=stream)
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e)

    for i in range(warmup):
        one(i)
    lat = sorted(one(i) for i in range(steps))

    def truth_error():
        num = den = 0.0
        for sd in range(500, 508):
            x, coeffs = synth.frame(g, seed=sd, return_truth=True)
            out = plan.reconstruct(torch.from_numpy(x.astype(np.float32)).to(dev), stream=stream)
            torch.cuda.synchronize(dev)
            t = synth.truth_layers(g, coeffs)
            num += float(np.sum((out.double().cpu().numpy() - t) ** 2))
            den += float(np.sum(t ** 2))
        return num / den

    e_learned = truth_error()
    safr.safr_filter_reset(plan.handle, stream=stream)
    e_plain = truth_error()
    lat_plain = sorted(one(i) for i in range(steps))  # the same frame kernel with plain SAFR's B
    if not used:  # the plan kept plain SAFR
        e_learned = e_plain
    mean_ms = float(np.mean(lat))
    out = {"grid": M, "stars": len(g["dir_x"]), "layers": len(g["h"]), "precision": "fp32 (MLP: bf16 weights)",
           "train": {"frames": 100000, "epochs": 2, "steps": res["steps"], "s": train_s,
                     "frames_per_s": res["steps"] * 256 / train_s,
                     "loss_first": res["train_loss_first"], "loss_last": res["train_loss_last"]},
           "heldout_rel_sq_error": {"learned": res["valid_loss_learned"], "plain_safr": res["valid_loss_plain"],
                                    "frames": 4096},
           "used_learned": used, "nonfinite": res["nonfinite"],
           "rebuild_B_ms": float(np.median(ta)), "B_max_rel_err_vs_oracle": b_err,
           "synthetic_frames_rel_sq_error_vs_truth": {"learned": e_learned, "plain_safr": e_plain, "frames": 8},
           "frames_per_s": 1e3 / mean_ms,
           "latency_ms": {"p50": lat[len(lat) // 2],
                          "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]},
           "plain_safr": {"frames_per_s": 1e3 / float(np.mean(lat_plain)),
                          "latency_ms": {"p50": lat_plain[len(lat_plain) // 2],
                                         "p99": lat_plain[min(len(lat_plain) - 1,
                                                              int(math.ceil(0.99 * len(lat_plain))) - 1)]}},
           "inference": "the MLP's inputs (|n|, h_l, sigma_r, noise level) do not change per frame, so its "
                        "factors are folded into B when B is rebuilt; the frame kernel is plain SAFR's, and the "
                        "noise level is a plan parameter",
           "steps": steps}
    plan.close()
    return g["name"], out


# ----------------------------------------------------------------------------
# ranks (one process per GPU, replicas: no collective on the data path)
# ----------------------------------------------------------------------------
def rank_max(value: float, device) -> float:
    """The largest of the ranks' values (a timed region's wall, max over ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, total_ms_max: float) -> float:
    """Whole-job frames/s: every rank reconstructs `steps` frames of its own; the
    job takes the slowest rank's time."""
    return world * steps / (total_ms_max * 1e-3)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def measure_l2_bandwidth(torch, dev, stream):
    """L2 bandwidth from a plain device copy whose source and destination stay in
    the L2 (sizes well below its 126 MB): 40 copies captured in one CUDA graph
    (so that launch gaps do not count), read + write bytes over the CUDA-event
    time of a replay; the best over a few sizes."""
    best, rows = 0.0, []
    for mb in (8, 16, 24, 32):
        n = (mb << 20) // 4
        a = torch.ones(n, dtype=torch.float32, device=dev)
        b = torch.empty_like(a)
        reps = 40
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                b.copy_(a)
        stream.wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                b.copy_(a)
        times = []
        for _ in range(5):
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            g.replay()
            e.record(stream)
            e.synchronize()
            times.append(s.elapsed_time(e))
        gbs = 2.0 * n * 4 * reps / (min(times) * 1e-3) / 1e9
        rows.append({"mb_each": mb, "gbs": gbs})
        best = max(best, gbs)
        del g, a, b
    return best, rows


def back_to_back(safr, torch, stream, plans, xs, outs, n, host_us=30.0):
    """n frames submitted back to back (no host synchronisation between them),
    cycling over the given plans and frames; CUDA events bracket the whole run.
    A bounded GPU sleep queued first, 1.5 x the expected host submission time
    (host_us per frame), lets the host queue the frames before the GPU reaches
    them, so the GPU does not wait for submissions.  Returns (ms on the device,
    host seconds spent submitting, seconds of sleep queued)."""
    torch.cuda.synchronize()
    sleep_s = min(0.5, 1.5 * n * host_us * 1e-6)
    torch.cuda._sleep(int(sleep_s * 2.07e9))  # GPU clock cycles (2070 MHz maximum SM clock)
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(stream)
    t0 = time.perf_counter()
    np_ = len(plans)
    for i in range(n):
        j = i % np_
        safr.safr_reconstruct(plans[j].handle, xs[i % len(xs)] if np_ == 1 else xs[j], outs[j], stream=stream)
    host_s = time.perf_counter() - t0
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e), host_s, sleep_s


def latency_run(safr, torch, stream, plan, xs, out, n, flush_l2, chunk=500):
    """Per-frame latency of n frames, the L2 flushed before each: flush, event,
    frame, event, submitted in chunks without host synchronisation inside a
    chunk.  Returns the sorted latencies in ms."""
    lat = []
    for c0 in range(0, n, chunk):
        ev = []
        for i in range(c0, min(n, c0 + chunk)):
            flush_l2(i)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            safr.safr_reconstruct(plan.handle, xs[i % len(xs)], out, stream=stream)
            b.record(stream)
            ev.append((a, b))
        ev[-1][1].synchronize()
        lat.extend(a.elapsed_time(b) for a, b in ev)
    return sorted(lat)


def pct(v, q):
    """The q-quantile of the sorted list v (nearest rank)."""
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]


def run_safr(args):
    import torch
    import torch.distributed as dist

    from paper_2510_19542_gb300 import safr, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    g = synth.config(2)
    frames_np = [synth.frame(g, seed=100 + i) for i in range(8)]

    # CPU baseline first (rank 0, N = 1): the oracle as it stands on the host cores
    cpu, ref_layers = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, dt, cores, ref_layers = oracle_frames(g, frames_np, args.cpu_sample_s, 64)
        cpu = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} full frames of the workload in {dt:.1f} s (FP64 oracle, naive DFT2; its "
                         "Jacobi-SVD B precompute untimed)"}

    path = {"auto": 0, "fused": 1, "passes": 2}[args.path]
    # a pool of plans of the workload: their B (21 MB each) and buffers together exceed the L2, so
    # frames submitted back to back over the pool read every B from HBM
    pool = [safr.Plan(g, device=local, path=path) for _ in range(args.pool)]
    plan = pool[0]
    stream = torch.cuda.current_stream(dev)
    frames = [torch.from_numpy(f.astype(np.float32)).to(dev) for f in frames_np]
    outs = [p.empty_layers() for p in pool]
    layers = outs[0]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_rd = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush_l2(i):
        # write 256 MB (evicts every line of the frame's data from the 129 MB L2),
        # then read another 256 MB so that the lines left behind are clean and the
        # timed frame pays no write-backs of the flush buffer
        flush.fill_(float(i & 7))
        flush_rd.sum()
    launches = safr.safr_launches_per_frame(plan.handle)
    info = plan.info
    stamps = []

    def one(i, trace):
        flush_l2(i)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        safr.safr_reconstruct(plan.handle, frames[i % len(frames)], layers, stream=stream)
        e.record(stream)
        e.synchronize()
        ph = safr.safr_trace_read(plan.handle) if trace else None
        if trace and launches == 1:
            stamps.append(safr.safr_trace_phases(plan.handle))
        return s.elapsed_time(e), ph

    # warm-up: every plan of the pool, back to back and flushed
    for i in range(args.warmup):
        one(i, False)
    _, h_s, _ = back_to_back(safr, torch, stream, pool, frames, outs, max(args.warmup, 4) * len(pool))
    host_us = 1e6 * h_s / (max(args.warmup, 4) * len(pool))  # host time per submitted frame
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    # (1) the value: frames submitted back to back over the pool (every B from HBM)
    cold_ms, cold_host_s, cold_sleep_s = back_to_back(safr, torch, stream, pool, frames, outs, args.steps, host_us)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    # (2) the same frames back to back on one plan: B stays in the L2 (warm)
    warm_ms, warm_host_s, warm_sleep_s = back_to_back(safr, torch, stream, [plan], frames, [layers], args.steps,
                                                      host_us)
    # (3) the pool's frames as one batch graph per call (safr_batch_reconstruct): frames run
    # concurrently on K chains of the graph, each on 1/K of the SMs (K timed at the first capture)
    batch = safr.safr_batch_create([p.handle for p in pool])
    xs_b = [frames[j % len(frames)] for j in range(len(pool))]
    safr.safr_batch_reconstruct(batch, xs_b, outs, stream=stream)  # capture (times K)
    torch.cuda.synchronize(dev)
    n_calls = max(1, args.steps // len(pool))
    for _ in range(3):
        safr.safr_batch_reconstruct(batch, xs_b, outs, stream=stream)
    torch.cuda.synchronize(dev)
    bs, be = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bs.record(stream)
    for _ in range(n_calls):
        safr.safr_batch_reconstruct(batch, xs_b, outs, stream=stream)
    be.record(stream)
    be.synchronize()
    conc_ms = bs.elapsed_time(be)
    conc_chains = safr.safr_batch_chains(batch)
    conc_status = safr.safr_batch_get_status(batch)
    safr.safr_batch_destroy(batch)
    # (4) many frames of one plan in one launch (safr_reconstruct_frames): no launch and no prologue
    # wait between frames; B stays in the L2
    nmf = 256
    xs_mf = torch.stack([frames[j % len(frames)] for j in range(nmf)])
    out_mf = torch.empty((nmf,) + tuple(layers.shape), dtype=layers.dtype, device=dev)
    safr.safr_reconstruct_frames(plan.handle, nmf, xs_mf, out_mf, stream=stream)
    torch.cuda.synchronize(dev)
    mf_calls = max(1, args.steps // nmf)
    ms_, me_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms_.record(stream)
    for _ in range(mf_calls):
        safr.safr_reconstruct_frames(plan.handle, nmf, xs_mf, out_mf, stream=stream)
    me_.record(stream)
    me_.synchronize()
    mf_ms = ms_.elapsed_time(me_)
    mf_same = bool(torch.equal(out_mf[nmf - 1], out_mf[(nmf - 1) % len(frames)]))
    del xs_mf, out_mf
    # (5) per-frame latency, L2 flushed before every frame
    lat = latency_run(safr, torch, stream, plan, frames, layers, args.latency_frames, flush_l2)
    clk = clocks.stop()
    # per-kernel durations and in-kernel phase marks from separate traced frames
    safr.safr_trace(plan.handle, True)
    phases = []
    for i in range(min(args.steps, 50)):
        _, ph = one(i, True)
        phases.append(ph)
    safr.safr_trace(plan.handle, False)
    total_ms = rank_max(cold_ms, dev)
    status = max(safr.safr_get_status(p.handle) for p in pool)
    bw_l2, l2_rows = measure_l2_bandwidth(torch, dev, stream)

    # end to end through the public host-buffer entry point (pinned memory)
    hin = [torch.from_numpy(f.astype(np.float32)).pin_memory() for f in frames_np]
    hout = torch.empty((info["L"], info["M"], info["M"]), dtype=torch.float32).pin_memory()
    for i in range(min(args.warmup, 5)):
        safr.safr_reconstruct_host(plan.handle, hin[i % 8], hout, stream=stream)
    e2e_ms = 0.0
    e2e_n = min(args.steps, 500)
    for i in range(e2e_n):
        flush_l2(i)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        safr.safr_reconstruct_host(plan.handle, hin[i % 8], hout, stream=stream)
        e2e_ms += 1e3 * (time.perf_counter() - t0)
    e2e_ms = rank_max(e2e_ms, dev)

    # a frame of the workload against the FP64 oracle, overall and per layer
    rel_l2, rel_own = None, None
    if ref_layers:
        fi = min(ref_layers)
        safr.safr_reconstruct(plan.handle, frames[fi], layers, stream=stream)
        torch.cuda.synchronize(dev)
        rel_l2, rel_own = layer_errors(layers.double().cpu().numpy(), ref_layers[fi])

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    workloads = {}
    if rank == 0 and world == 1 and not args.no_workloads:
        want = set(args.workloads.split(",")) if args.workloads != "all" else \
            {"tiny", "fp16-512", "batch", "learned", "loop", "refresh"}
        for kk, key in ((1, "tiny"), (3, "fp16-512")):
            if key in want:
                name, res = measure_workload(safr, synth, torch, dev, stream, kk, min(args.steps, 100), 5, flush_l2,
                                             hbm)
                workloads[name] = res
        if "batch" in want:
            name, res = measure_batch(safr, synth, torch, dev, stream, min(args.steps, 20), 3, flush_l2, hbm)
            workloads[name] = res
        if "learned" in want:
            name, res = measure_learned(safr, synth, torch, dev, stream, min(args.steps, 100), 5, flush_l2)
            workloads[name] = res
        if "loop" in want:
            name, res = measure_loop(safr, synth, torch, dev, stream, min(args.steps, 100), 5, flush_l2, hbm)
            workloads[name] = res
        if "refresh" in want:
            name, res = measure_refresh(safr, synth, torch, dev, stream, 10)
            workloads[name] = res

    if rank == 0:
        ph = np.array(phases)  # [frames][launches]
        ph_mean = ph.mean(axis=0).tolist()
        M, Mh = info["M"], info["M"] // 2
        sumLG = info["L"] * info["G"]
        b_bytes = M * Mh * sumLG * 8                  # algorithmic B: half spectrum, no Nyquist column
        in_bytes = info["G"] * info["P"] ** 2 * 4
        out_bytes = info["L"] * M * M * 4
        frame_bytes = b_bytes + in_bytes + out_bytes
        cold_s = total_ms / args.steps * 1e-3       # per frame, back to back, B from HBM
        warm_s = warm_ms / args.steps * 1e-3        # per frame, back to back, B in the L2
        if launches == 1:
            # one library kernel per frame: the events bracket exactly the frames' launches
            kname, k_bytes, k_s = "k_frame", frame_bytes, cold_s
            phase_names = ["frame"]
        else:
            kname, k_bytes, k_s = "k_cols_apply", b_bytes, ph_mean[1] * 1e-3
            phase_names = ["rows_forward", "cols_apply", "rows_inverse"]
        achieved = k_bytes / k_s / 1e9
        traffic = None
        try:
            with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
                rec = json.load(f).get(WORKLOAD, {}).get(kname)
            # counters taken on other kernel sources say nothing about this build
            if rec and rec.get("csrc_sha256") == csrc_sha256():
                traffic = rec["traffic_bytes"]
        except (OSError, ValueError, KeyError):
            traffic = None
        t_roof_l2 = b_bytes / (bw_l2 * 1e9) + (in_bytes + out_bytes) / (hbm * 1e9)
        value = job_throughput(world, args.steps, total_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic von Karman frames (seeded), FP32", "config": config_block(g, args.pool),
            "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "mean": float(np.mean(lat)),
                           "frames": len(lat), "l2": "flushed before every frame"},
            "latency_10k": {"frames": len(lat), "p50_us": 1e3 * pct(lat, 0.5), "p90_us": 1e3 * pct(lat, 0.9),
                            "p99_us": 1e3 * pct(lat, 0.99), "p999_us": 1e3 * pct(lat, 0.999),
                            "max_us": 1e3 * lat[-1], "mean_us": 1e3 * float(np.mean(lat)),
                            "how": "CUDA events around each safr_reconstruct, L2 flushed (256 MB written, "
                                   "256 MB read) before every frame, frames submitted in chunks of 500"},
            "throughput_back_to_back": {
                "cold_B": {"frames_per_s": args.steps / (total_ms * 1e-3), "us_per_frame": 1e6 * cold_s,
                           "host_submit_us_per_frame": 1e6 * cold_host_s / args.steps,
                           "all_queued_before_gpu_start": cold_host_s < cold_sleep_s,
                           "how": f"{args.steps} frames back to back over {args.pool} plans of the workload "
                                  f"({args.pool} x 21 MB of B: every frame's B comes from HBM)"},
                "concurrent_chains": {"frames_per_s": n_calls * len(pool) / (conc_ms * 1e-3),
                                      "us_per_frame": 1e3 * conc_ms / (n_calls * len(pool)), "chains": conc_chains,
                                      "device_status": conc_status,
                                      "how": f"the {len(pool)} plans' frames as one safr_batch_reconstruct graph "
                                             f"launch per call, {n_calls} calls back to back: the frames run "
                                             f"{conc_chains} at a time, each on 1/{conc_chains} of the SMs"},
                "multi_frame_launch": {"frames_per_s": mf_calls * nmf / (mf_ms * 1e-3),
                                       "us_per_frame": 1e3 * mf_ms / (mf_calls * nmf),
                                       "repeated_frames_identical": mf_same,
                                       "how": f"safr_reconstruct_frames: {nmf} frames of one plan per launch, "
                                              f"{mf_calls} launches back to back (B stays in the L2)"},
                "warm_L2": {"frames_per_s": args.steps / (warm_ms * 1e-3), "us_per_frame": 1e6 * warm_s,
                            "host_submit_us_per_frame": 1e6 * warm_host_s / args.steps,
                            "all_queued_before_gpu_start": warm_host_s < warm_sleep_s,
                            "how": f"{args.steps} frames back to back on one plan (B stays in the L2)"}},
            "kernels_ms": dict(zip(phase_names, ph_mean)), "path": "fused" if launches == 1 else "passes",
            "fused_phases_us": ({k: float(np.median([st[k] for st in stamps])) for k in stamps[0]}
                                if stamps else None),
            "frame_roofline": {"bytes": frame_bytes, "achieved_gbs": frame_bytes / cold_s / 1e9,
                               "peak_gbs": hbm, "frac": frame_bytes / cold_s / 1e9 / hbm},
            "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                         "algorithmic_bytes": k_bytes,
                         "duration": "mean launch time of the back-to-back frames over the plan pool"},
            "roofline_l2": {"bound": "l2+hbm", "bw_l2_gbs": bw_l2, "bw_hbm_gbs": hbm,
                            "bw_l2_how": "plain device copy (torch copy_, 40 copies in one CUDA graph) with source "
                                         "and destination resident in the L2, read + write bytes / CUDA-event "
                                         "time; best of "
                                         + ", ".join(f"{r['mb_each']} MB ({r['gbs']:.0f} GB/s)" for r in l2_rows),
                            "t_roof_us": 1e6 * t_roof_l2, "achieved_us": 1e6 * warm_s,
                            "frac": t_roof_l2 / warm_s,
                            "formula": "bytes_B / BW_L2 + (bytes_in + bytes_out) / BW_HBM, against the warm "
                                       "back-to-back frame"},
            "clocks": clk, "gpu_launches": launches * args.steps, "device_status": status,
            "rel_l2_vs_oracle": rel_l2, "rel_l2_per_layer_own": rel_own,
            "e2e": {"value": job_throughput(world, e2e_n, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
                    "ms_per_step": e2e_ms / e2e_n, "steps": e2e_n},
            "wall_s_timed_region": wall,
        }
        if workloads:
            line["workloads"] = workloads
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    for p in pool:
        p.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_safr(args)


if __name__ == "__main__":
    sys.exit(main())
