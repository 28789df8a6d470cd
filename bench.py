#!/usr/bin/env python3
"""Benchmark of the 3-D segmentation stage on the time-lapse workload.

Workload: 512x512x64 uint16 volumes, 60 frames x 2 channels (nuclei random
walk with divisions + static vessels, noise N(200,25)), 2.01 G voxels per
step.  A step segments every volume-channel once: smoothing, histogram, Otsu,
threshold, 26-connected labelling, minimum-volume filter, numbering, features.

value:  Gvoxels/s with the inputs already resident in HBM (device-timed with
        CUDA events on the ordering stream around all steps).
e2e:    the same metric through the C ABI from pinned host buffers: every step
        copies the inputs host->device inside seg_submit_volume and reads the
        segmentation back to host memory (each cell's voxels as label runs,
        and the cell table); one thread submits while another reads, so both
        directions of the host link overlap.  e2e_dense_labels: the same with
        the dense uint32 label images read instead of the runs.
roofline: the kernel with the largest share of device time in the timed
        region, its algorithmic bytes per launch over its mean CUDA-event
        duration, against the measured copy bandwidth.
cpu_baseline: the CPU oracle (single-threaded C) on a bounded sample.

--impl reference times the CPU oracle instead (one process per host core,
independent volume-channels), on the same metric and workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Gvoxels/s segmented (fraction of HBM roofline); served p50/p99 latency per volume")
WORKLOAD = "time-lapse 512x512x64 x 60 frames x 2 channels uint16"
DIMS = (512, 512, 64)
FRAMES = 60
CHANNELS = 2
ALGO_BYTES_PER_VOXEL = 8.0  # 2 B raw read + 2 B re-read after Otsu + 4 B label write
# Algorithmic bytes per voxel of each kernel (the units one launch processes
# are all voxels of the batch).
KERNEL_BYTES_PER_VOXEL = {
    "smooth_rows": 2.0,            # raw uint16 read once (row-aligned volumes)
    "smooth_hist": 2.0,            # raw uint16 read once (other volumes)
    "threshold_runs": 1 / 8.0,     # 1-bit mask write (the smoothed re-read is the 2 B
                                   # counted in the 8 B/voxel path total)
    "label_features": 4.0,         # uint32 label write (run tables are O(runs))
    "row_count": 1 / 8.0,
    "row_runs": 1 / 8.0,
    "init": 0.0,
}
# DRAM bytes (read + write) per voxel measured by ncu on the same kernel build
# (8 volume-channels of the 512x512x64 time-lapse, 134 M voxels, inputs larger
# than L2); the per-launch figure scales with the voxels a launch processes
# since every 512x512x64 volume is tiled the same way.
KERNEL_TRAFFIC_BYTES_PER_VOXEL = {
    "smooth_rows": 4.04,           # 2.28 read (halo rows partly from L2) + 1.76 smoothed
                                   # and word-maximum writes
    "smooth_hist": 7.69,           # 5.88 read (halo lines re-read) + 1.81 smoothed write
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank):
    """Each rank segments its own time-lapse (weak scaling, independent
    volumes, no data exchanged between ranks)."""
    return 2 + 1000 * rank


def max_over_ranks(ms, device, ws):
    """Largest per-rank time: the whole job ends when the slowest rank does."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gvox_per_s(voxels_per_rank, ms, ws):
    """Whole-job throughput: voxels of all ranks over the slowest rank's time."""
    return voxels_per_rank * ws / (ms / 1e3) / 1e9


def make_workload(rank, frames=FRAMES):
    import synth
    tl = synth.TimeLapse(seed=rank_seed(rank), frames=frames)
    X, Y, Z = DIMS
    host = np.empty((frames, CHANNELS, Z, Y, X), dtype=np.uint16)
    for t in range(frames):
        for c in range(CHANNELS):
            host[t, c] = tl.frame(t, c)
    return host


def cpu_baseline(host, budget_s=12.0):
    """Single-threaded oracle on the first volume-channels until ~budget_s."""
    import oracle
    n, t0, done = 0, time.perf_counter(), 0
    vox = 0
    for t in range(host.shape[0]):
        for c in range(host.shape[1]):
            oracle.segment(host[t, c], min_volume=30)
            vox += host[t, c].size
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": vox / dt / 1e9, "unit": "Gvoxels/s", "cores": 1, "kind": "oracle",
            "sample": "%d of %d volume-channels of the workload, single-threaded C oracle, %.1f s"
                      % (done, host.shape[0] * host.shape[1], dt)}


_CACHE = {}


def _oracle_config_job(args):
    """Segments one volume-channel of another workload with the oracle:
    ("uneven", i) is volume i of the batched-uneven workload, ("serving", i, c)
    channel c of request i of the serving stream.  Volumes are generated in
    the worker before the clock starts; returns (voxels, seconds, pid)."""
    import oracle
    import synth
    key = args
    if key not in _CACHE:
        if args[0] == "uneven":
            d = synth.batched_uneven_dims()[args[1]]
            _CACHE[key] = synth.density_volume(d, synth.mix_seed(3, 3, args[1]))
        else:
            d = synth.serving_requests(seed=5, n=args[1] + 1)[args[1]][1]
            _CACHE[key] = synth.serving_volume(d, 5, args[1], args[2])
    vol = _CACHE.pop(key)
    t0 = time.perf_counter()
    oracle.segment(vol, min_volume=30)
    return vol.size, time.perf_counter() - t0, os.getpid()


def cpu_other_configs(n_serving=32):
    """The CPU oracle on the other workloads, in the same run: the single
    128x128x32 frame on one core (repeated for about 2 s), and with one
    process per host core all 48 batched-uneven volumes and the first
    n_serving requests (both channels) of the serving stream.  A multi-core
    figure divides the voxels by the makespan (the largest per-process sum
    of oracle time; generation is excluded)."""
    import multiprocessing as mp
    import oracle
    import synth
    cores = os.cpu_count() or 1
    out = {}
    v1 = synth.single_frame()
    oracle.segment(v1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 2.0:
        oracle.segment(v1, min_volume=30)
        n += 1
    dt = time.perf_counter() - t0
    out["single_frame"] = {"value": n * v1.size / dt / 1e9, "unit": "Gvoxels/s", "cores": 1, "kind": "oracle",
                           "latency_ms": dt / n * 1e3,
                           "sample": "the 128x128x32 frame segmented %d times, single-threaded" % n}
    jobs = {"uneven": [("uneven", i) for i in range(48)],
            "serving": [("serving", i, c) for i in range(n_serving) for c in range(2)]}
    samples = {"uneven": "all 48 volumes (0.73 G voxels)",
               "serving": "requests 0-%d of the Poisson stream, both channels" % (n_serving - 1)}
    with mp.get_context("spawn").Pool(cores) as pool:
        for name, jl in jobs.items():
            res = pool.map(_oracle_config_job, jl, chunksize=1)
            per, vox = {}, 0
            for v, d, pid in res:
                per[pid] = per.get(pid, 0.0) + d
                vox += v
            span = max(per.values())
            out[name] = {"value": vox / span / 1e9, "unit": "Gvoxels/s", "cores": cores, "kind": "oracle",
                         "sample": samples[name] + ", one oracle process per core; makespan %.1f s" % span}
    return out


def _oracle_job(args):
    """Segments one volume-channel with the oracle; returns (voxels, oracle
    seconds, pid).  Volumes are generated once per worker and cached, so the
    timing covers the oracle only."""
    seed, t, c = args
    import oracle
    key = (seed, t, c)
    if key not in _CACHE:
        import synth
        tl = synth.TimeLapse(seed=seed, frames=FRAMES)
        _CACHE[key] = tl.frame(t, c)
    vol = _CACHE[key]
    t0 = time.perf_counter()
    oracle.segment(vol, min_volume=30)
    return vol.size, time.perf_counter() - t0, os.getpid()


def run_reference(args):
    """CPU oracle arm: each step segments a bounded sample of the workload's
    volume-channels, one process per host core.  A step's time is its
    makespan: the largest per-process sum of oracle time in that step."""
    import multiprocessing as mp
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    per_step = max(cores, 1)
    ctxp = mp.get_context("spawn")
    jobs = [(2, (i // CHANNELS) % FRAMES, i % CHANNELS) for i in range(per_step)]
    with ctxp.Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_job, jobs, chunksize=1)
        total, vox = 0.0, 0
        for _ in range(args.steps):
            res = pool.map(_oracle_job, jobs, chunksize=1)
            per = {}
            for v, dt, pid in res:
                per[pid] = per.get(pid, 0.0) + dt
                vox += v
            total += max(per.values())
    dt = total
    value = vox / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gvoxels/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16/u32 (Otsu f64)",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": "%d volume-channels" % per_step},
        "cpu_baseline": {"value": value, "unit": "Gvoxels/s", "cores": cores, "kind": "oracle",
                         "sample": "%d volume-channels per step (each 512x512x64), one oracle process per core; "
                                   "step time = largest per-process oracle time (generation excluded)" % per_step},
        "e2e": {"value": value, "unit": "Gvoxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1407_2089_gb300 as seg

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host = make_workload(rank, args.frames)
    T, C, Z, Y, X = host.shape
    vox_step = host.size
    cpu = cpu_baseline(host) if (rank == 0 and not args.no_cpu) else None
    cpu_other = cpu_other_configs() if (rank == 0 and not args.no_cpu) else None

    d_in = torch.from_numpy(host.view(np.int16)).to(dev)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)  # ordering stream (a non-null handle)
    flags = seg.SEG_PROFILE
    tile = {}
    if args.tile:
        ty, tz = (int(v) for v in args.tile.split(","))
        flags |= seg.SEG_FORCE_TILE
        tile = {"tile_y": ty, "tile_z": tz}
    ctx = seg.seg_create(device=local, flags=flags, batch_window_us=2_000_000, order_stream=stream.cuda_stream,
                         max_inflight=args.inflight, **tile)

    def step(ctx, in_ptr_fn):
        reqs = []
        for t in range(T):
            reqs.append(in_ptr_fn(t))
        seg.seg_flush(ctx)
        for r in reqs:
            seg.seg_enqueue_wait(ctx, r, stream.cuda_stream)
        return reqs

    vol_elems = C * Z * Y * X

    def submit_dev(t):
        return seg.seg_submit_volume(ctx, d_in[t], dims=(X, Y, Z), channels=C)

    def finish(reqs):
        for r in reqs:
            if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            seg.seg_release(ctx, r)

    # warm-up, in the same pipelined pattern as the timed steps (one step in
    # flight while the previous one is read), so that the memory pool and the
    # captured graphs of every slot are in their steady state before timing
    pend = []
    for _ in range(args.warmup):
        pend.append(step(ctx, submit_dev))
        if len(pend) > 1:
            finish(pend.pop(0))
    for p in pend:
        finish(p)
    torch.cuda.synchronize()
    seg.seg_reset_stats(ctx)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        pend = []
        for _ in range(args.steps):
            pend.append(step(ctx, submit_dev))
            if len(pend) > 1:
                finish(pend.pop(0))
        ev1.record(stream)
        for p in pend:
            finish(p)
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev, ws)
    if ws > 1:
        dist.barrier()
    stats = seg.seg_get_stats(ctx)
    value = job_gvox_per_s(vox_step * args.steps, ms, ws)
    launches = sum(k["launches"] for k in stats["kernels"].values())

    # dominant kernel and its roofline
    peak, peak_kind = peaks()
    kern = stats["kernels"]
    dom = max((n for n in kern if n in KERNEL_BYTES_PER_VOXEL and KERNEL_BYTES_PER_VOXEL[n] > 0),
              key=lambda n: kern[n]["ms"])
    mean_ms = kern[dom]["ms"] / max(kern[dom]["launches"], 1)
    vox_launch = stats["voxels"] / max(kern[dom]["launches"], 1)
    achieved = KERNEL_BYTES_PER_VOXEL[dom] * vox_launch / (mean_ms / 1e3) / 1e9
    total_kernel_ms = sum(k["ms"] for k in kern.values())
    shares = {n: round(k["ms"] / total_kernel_ms, 4) for n, k in kern.items()} if total_kernel_ms else {}
    seg.seg_destroy(ctx)
    denoise = closing = distmap = mrfd = reg = None
    if args.denoise_radius:
        denoise = denoise_run(seg, torch, d_in, (X, Y, Z), local, max(1, min(args.steps, 5)), args.denoise_radius)
    if args.closing_radius:
        closing = closing_run(seg, torch, d_in, (X, Y, Z), local, max(1, min(args.steps, 5)), args.closing_radius)
    if args.register:
        reg = registration_run(seg, torch, local)
    if args.mrf_iterations:
        mrfd = mrf_run(seg, torch, d_in, (X, Y, Z), local, max(1, min(args.steps, 3)), args.mrf_iterations)
    if args.distance_weights != "0":
        distmap = distance_run(seg, torch, d_in, (X, Y, Z), local, max(1, min(args.steps, 5)),
                               [int(a) for a in args.distance_weights.split(",")])
    forms = None
    if not args.no_forms:
        forms = {"batched": value / ws, "plain": plain_form(seg, torch, d_in, (X, Y, Z), local,
                                                            max(1, min(args.steps, 3)))}
    del d_in
    torch.cuda.empty_cache()
    uneven = None
    if not args.no_uneven and rank == 0:
        uneven = uneven_forms(seg, torch, local, max(1, min(args.steps, 5)))
        torch.cuda.empty_cache()
    mont = None
    if args.montage and rank == 0:
        mont = montage_run(seg, torch, local, max(1, min(args.steps, 3)))
        torch.cuda.empty_cache()
    serve = None
    if args.serving_requests and rank == 0:
        queued = args.serving_copies == "queued"
        serve = {"batched": serving(seg, torch, local, args.serving_requests, 200.0, 0, 2, queued),
                 "plain": serving(seg, torch, local, args.serving_requests, 200.0, seg.SEG_PLAIN, 1, queued),
                 "input_copies": args.serving_copies}

    # end to end through the C ABI with pinned host buffers
    e2e = e2e_dense = None
    if not args.no_e2e:
        h_in = torch.from_numpy(host.view(np.int16)).pin_memory()
        group = max(1, args.e2e_group)
        queued = args.e2e_copies == "queued"
        e2e = e2e_run(seg, torch, dist, args, local, dev, ws, stream, h_in, (X, Y, Z), T, C, group, "runs", queued,
                      args.e2e_ahead)
        e2e_dense = e2e_run(seg, torch, dist, args, local, dev, ws, stream, h_in, (X, Y, Z), T, C, group,
                            "labels", queued, args.e2e_ahead)
        e2e["value"] = job_gvox_per_s(vox_step * e2e.pop("steps_timed"), e2e.pop("ms"), ws)
        e2e_dense["value"] = job_gvox_per_s(vox_step * e2e_dense.pop("steps_timed"), e2e_dense.pop("ms"), ws)
        # the boundary's own result call (seg_read_labels: dense uint32 label
        # images) beside the run-encoded read of the headline figure
        e2e["dense_labels"] = {k: e2e_dense[k] for k in ("value", "d2h_bytes_per_step", "step_ms_max")
                               if k in e2e_dense}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gvoxels/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16/u32 (Otsu f64)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("x 60 frames", "x %d frames" % T), "voxels_per_step": vox_step, "min_volume": 30,
                       "tile": [int(stats["tile_y"]), int(stats["tile_z"])],
                       "batches_per_step": stats["batches"] / args.steps,
                       "l2": "inputs %.2f GB per step > 129 MB L2; no flush" % (vox_step * 2 / 1e9),
                       "form": "batched (one graph-captured launch sequence per step)"},
            "hbm_fraction": value * ALGO_BYTES_PER_VOXEL / peak,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (KERNEL_TRAFFIC_BYTES_PER_VOXEL[dom] * vox_launch
                                     if dom in KERNEL_TRAFFIC_BYTES_PER_VOXEL else None),
                         "peak_source": peak_kind,
                         "algo_bytes_per_voxel": KERNEL_BYTES_PER_VOXEL[dom]},
            "kernel_share": shares,
            "cpu_baseline": cpu,
            "cpu_baseline_other_configs": cpu_other,
            "e2e": e2e,
            "e2e_dense_labels": e2e_dense,
            "forms_gvox_s_per_gpu": forms,
            "uneven_batch": uneven,
            "montage": mont,
            "denoise_front_end": denoise,
            "closing": closing,
            "distance_map": distmap,
            "mrf_denoise": mrfd,
            "registration": reg,
            "serving": serve,
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def option_run(seg, torch, d_in, dims, local, steps, denoise, closing, distance_weights=None, mrf_iterations=0):
    """The same workload, batched as in the main measurement, with per-channel
    options (denoise radii, closing radii, distance-map weights).  Returns
    Gvoxels/s of the whole stage, ms per step and the mean per-step
    CUDA-event time of every kernel."""
    T, C = d_in.shape[0], d_in.shape[1]
    X, Y, Z = dims
    stream = torch.cuda.Stream()
    ctx = seg.seg_create(device=local, flags=seg.SEG_PROFILE, batch_window_us=2_000_000,
                         order_stream=stream.cuda_stream, max_inflight=1)

    def one_pass():
        reqs = [seg.seg_submit_volume(ctx, d_in[t], dims=(X, Y, Z), channels=C, denoise_radius=denoise,
                                      closing_radius=closing, distance_weights=distance_weights,
                                      mrf_iterations=mrf_iterations)
                for t in range(T)]
        seg.seg_flush(ctx)
        for r in reqs:
            seg.seg_enqueue_wait(ctx, r, stream.cuda_stream)
        return reqs

    def finish(reqs):
        for r in reqs:
            if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            seg.seg_release(ctx, r)

    for _ in range(2):
        finish(one_pass())
    torch.cuda.synchronize()
    seg.seg_reset_stats(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pend = []
    for _ in range(steps):
        pend.append(one_pass())
        if len(pend) > 1:
            finish(pend.pop(0))
    e1.record(stream)
    for p in pend:
        finish(p)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kern = seg.seg_get_stats(ctx)["kernels"]
    seg.seg_destroy(ctx)
    per = {n: k["ms"] / steps for n, k in kern.items()}
    return d_in.numel() / (ms / 1e3) / 1e9, ms, per


def denoise_run(seg, torch, d_in, dims, local, steps, radius):
    """The denoise front end of Eq. 1 on the stem-cell channel (channel 0)."""
    T, C = d_in.shape[0], d_in.shape[1]
    X, Y, Z = dims
    gv, ms, per = option_run(seg, torch, d_in, dims, local, steps, [radius] + [0] * (C - 1), 0)
    vox_dn = T * X * Y * Z  # voxels through the front end per step (channel 0)
    front_ms = per["denoise_box"] + per["denoise_median"]
    return {"radius": radius, "channels_denoised": 1, "gvox_s": gv,
            "ms_per_step": ms, "front_end_ms_per_step": front_ms,
            "front_end_gvox_s": vox_dn / (front_ms / 1e3) / 1e9 if front_ms else None,
            "kernel_ms_per_step": {n: per[n] for n in ("denoise_box", "denoise_median")},
            # algorithmic bytes of the front end: read the observed image,
            # write the denoised one (4 B/voxel); the box passes move 12 B
            "front_end_hbm_frac": (vox_dn * 4.0 / (front_ms / 1e3) / 1e9) / peaks()[0] if front_ms else None}


def closing_run(seg, torch, d_in, dims, local, steps, radius):
    """The closing of the foreground with a ball of `radius` on every channel."""
    gv, ms, per = option_run(seg, torch, d_in, dims, local, steps, 0, radius)
    close_ms = per["dilate"] + per["erode"]
    return {"radius": radius, "gvox_s": gv, "ms_per_step": ms, "closing_ms_per_step": close_ms,
            "kernel_ms_per_step": {n: per[n] for n in ("dilate", "erode")}}


def distance_run(seg, torch, d_in, dims, local, steps, weights):
    """The distance map of the vessel channel (the last one) with the given
    weights; every channel otherwise as in the main measurement."""
    T, C = d_in.shape[0], d_in.shape[1]
    X, Y, Z = dims
    gv, ms, per = option_run(seg, torch, d_in, dims, local, steps, 0, 0,
                             [None] * (C - 1) + [tuple(weights)])
    vox = T * X * Y * Z  # voxels with a distance map per step
    names = ("dist_xy", "dist_xy_1024", "dist_x", "dist_y", "dist_z", "dist_z_long")
    dist_ms = sum(per[n] for n in names)
    # algorithmic bytes per voxel: the x (or fused x+y) pass reads the mask bit
    # and writes a uint32; each line pass reads and writes one uint32 (stack
    # traffic is not counted); mask to map at least 4.125 B
    algo = {"dist_xy": 4.125, "dist_xy_1024": 4.125, "dist_x": 4.125, "dist_y": 8.0, "dist_z": 8.0,
            "dist_z_long": 8.0}
    peak = peaks()[0]
    return {"weights": list(weights), "channels": 1, "gvox_s": gv, "ms_per_step": ms,
            "distance_ms_per_step": dist_ms,
            "distance_gvox_s": vox / (dist_ms / 1e3) / 1e9 if dist_ms else None,
            "kernel_ms_per_step": {n: per[n] for n in names},
            # kernels that took this workload (the others only launch and exit)
            "kernel_hbm_frac": {n: (vox * algo[n] / (per[n] / 1e3) / 1e9) / peak
                                for n in names if per[n] > 0.05 * dist_ms},
            "stage_hbm_frac": (vox * 4.125 / (dist_ms / 1e3) / 1e9) / peak if dist_ms else None}


def mrf_run(seg, torch, d_in, dims, local, steps, iters):
    """The MRF vessel denoise (Eqs. 2-3) on the vessel channel (the last one),
    at most `iters` steps; every channel otherwise as in the main measurement."""
    T, C = d_in.shape[0], d_in.shape[1]
    X, Y, Z = dims
    gv, ms, per = option_run(seg, torch, d_in, dims, local, steps, 0, 0, None, [0] * (C - 1) + [iters])
    vox = T * X * Y * Z  # voxels through the MRF denoise per step
    mrf_ms = per["mrf_stats"] + per["mrf_iterate"]
    # algorithmic bytes: the statistics pass reads the input once (2 B); each
    # step reads the current image and the input and writes the next (6 B)
    return {"max_steps": iters, "channels": 1, "gvox_s": gv, "ms_per_step": ms,
            "mrf_ms_per_step": mrf_ms,
            "kernel_ms_per_step": {n: per[n] for n in ("mrf_stats", "mrf_iterate")},
            "ms_per_mrf_step": per["mrf_iterate"] / iters if iters else None,
            "step_hbm_frac": ((vox * 6.0 * iters / (per["mrf_iterate"] / 1e3) / 1e9) / peaks()[0]
                              if per["mrf_iterate"] else None)}


def registration_run(seg, torch, local, grid=(3, 3), dims=(1024, 1024, 64), overlap=0.1, radius=(4, 4, 1),
                     reps=3):
    """Montage registration (Eq. 4 + maximum spanning tree): tiles cut on the
    GPU from one seeded noise volume at planted positions, stage positions
    off by up to half the window; the whole call is timed (wall clock,
    synchronous)."""
    import synth
    rng = np.random.default_rng(synth.mix_seed(4, 7))
    X, Y, Z = dims
    ov = (int(round(X * overlap)), int(round(Y * overlap)))
    true, stage = [], []
    for j in range(grid[1]):
        for i in range(grid[0]):
            st = np.array([i * (X - ov[0]) + radius[0], j * (Y - ov[1]) + radius[1], 0])
            t = st + np.array([rng.integers(-(radius[0] // 2), radius[0] // 2 + 1),
                               rng.integers(-(radius[1] // 2), radius[1] // 2 + 1), rng.integers(0, radius[2] + 1)])
            true.append(t)
            stage.append(st)
    true, stage = np.array(true), np.array(stage)
    ext = true.max(axis=0) + np.array(dims) + 1
    g = torch.Generator(device="cuda:%d" % local)
    g.manual_seed(int(synth.mix_seed(4, 8)) & 0x7FFFFFFF)
    G = torch.randint(0, 3000, (int(ext[2]), int(ext[1]), int(ext[0])), generator=g, device="cuda:%d" % local,
                      dtype=torch.int32)
    tiles = [G[t[2]:t[2] + Z, t[1]:t[1] + Y, t[0]:t[0] + X].to(torch.int16).contiguous() for t in true]
    del G
    torch.cuda.synchronize()
    seg.seg_register_montage(tiles, stage, radius)  # warm-up
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        delta, edges = seg.seg_register_montage(tiles, stage, radius)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.median(ts))
    # products of the correlation: every shift's shared box, summed
    prod = 0
    for e in edges:
        d0 = stage[e["b"]] - stage[e["a"]]
        for sz in range(-radius[2], radius[2] + 1):
            for sy in range(-radius[1], radius[1] + 1):
                for sx in range(-radius[0], radius[0] + 1):
                    n = 1
                    for k, (d, D) in enumerate(zip(d0 + np.array([sx, sy, sz]), dims)):
                        n *= max(0, min(D, d + D) - max(0, d))
                    prod += n
    ok = bool(np.array_equal(delta, (true - stage) - (true - stage)[0]))
    del tiles
    torch.cuda.empty_cache()
    return {"tiles": int(np.prod(grid)), "tile_dims": list(dims), "overlap": overlap, "radius": list(radius),
            "edges": int(len(edges)), "ms_per_registration": ms, "products": int(prod),
            "gproducts_s": prod / (ms / 1e3) / 1e9, "planted_offsets_recovered": ok}


def plain_form(seg, torch, d_in, dims, local, steps):
    """Same workload through the plain per-frame form: one request (both
    channels of a frame) per launch sequence, one stream, no graphs."""
    T, C = d_in.shape[0], d_in.shape[1]
    X, Y, Z = dims
    stream = torch.cuda.Stream()
    ctx = seg.seg_create(device=local, flags=seg.SEG_PLAIN, order_stream=stream.cuda_stream)
    vox = 0

    def one_pass():
        reqs = [seg.seg_submit_volume(ctx, d_in[t], dims=(X, Y, Z), channels=C) for t in range(T)]
        for r in reqs:
            seg.seg_enqueue_wait(ctx, r, stream.cuda_stream)
        return reqs

    def finish(reqs):
        for r in reqs:
            if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            seg.seg_release(ctx, r)

    finish(one_pass())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pend = []
    for _ in range(steps):
        pend.append(one_pass())
        vox += d_in.numel()
        if len(pend) > 1:
            finish(pend.pop(0))
    e1.record(stream)
    for p in pend:
        finish(p)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    seg.seg_destroy(ctx)
    return vox / (ms / 1e3) / 1e9


def uneven_forms(seg, torch, local, steps):
    """The batched-uneven workload (48 uint16 volumes, 64^3 ... 1024x1024x96,
    nuclei 1 per 40^3 voxels), resident on the device: all of them in one
    graph-captured launch sequence (batched) against one plain launch
    sequence per volume, timed on an ordering stream like the main line.
    Also the single 128x128x32 frame through the plain form: median latency
    of sequential requests, submit to done."""
    import synth
    vols = synth.batched_uneven()
    dvols = [torch.from_numpy(v.view(np.int16)).to("cuda:%d" % local) for v in vols]
    vox = int(sum(v.size for v in vols))
    out = {"volumes": len(vols), "voxels": vox}
    for name, flags in (("batched", 0), ("plain", seg.SEG_PLAIN)):
        stream = torch.cuda.Stream()
        # a long batch window: the flush after the last submit starts one batch
        ctx = seg.seg_create(device=local, flags=flags, order_stream=stream.cuda_stream,
                             batch_window_us=0 if flags else 10_000_000)

        def one_pass():
            reqs = [seg.seg_submit_volume(ctx, dv, dims=(v.shape[2], v.shape[1], v.shape[0]), channels=1)
                    for dv, v in zip(dvols, vols)]
            seg.seg_flush(ctx)
            for r in reqs:
                seg.seg_enqueue_wait(ctx, r, stream.cuda_stream)
            return reqs

        def finish(reqs):
            for r in reqs:
                if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                    raise RuntimeError("request failed")
                seg.seg_release(ctx, r)

        for _ in range(2):
            finish(one_pass())
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            finish(one_pass())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if name == "batched":
            out["batches_per_pass"] = seg.seg_get_stats(ctx)["batches"] / (steps + 2)
        seg.seg_destroy(ctx)
        out[name] = {"ms_per_pass": ms, "gvox_s": vox / (ms / 1e3) / 1e9}
    del dvols
    # the single frame, submit -> done, sequential requests: the plain form,
    # and the same with every kernel launched on its own (no graph)
    v1 = synth.single_frame()
    d1 = torch.from_numpy(v1.view(np.int16)).to("cuda:%d" % local)
    for name, flags in (("single_frame_plain", seg.SEG_PLAIN),
                        ("single_frame_plain_no_graph", seg.SEG_PLAIN | seg.SEG_NO_GRAPH)):
        ctx = seg.seg_create(device=local, flags=flags)
        lat = []
        for i in range(53):
            t0 = time.perf_counter()
            r = seg.seg_submit_volume(ctx, d1, dims=(v1.shape[2], v1.shape[1], v1.shape[0]), channels=1)
            if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            if i >= 3:
                lat.append((time.perf_counter() - t0) * 1e3)
            seg.seg_release(ctx, r)
        seg.seg_destroy(ctx)
        out[name] = {"dims": [int(v1.shape[2]), int(v1.shape[1]), int(v1.shape[0])],
                     "latency_ms_median": statistics.median(lat),
                     "latency_ms_p99": float(np.percentile(lat, 99)),
                     "gvox_s": v1.size / (statistics.median(lat) / 1e3) / 1e9}
    return out


def montage_run(seg, torch, local, steps):
    """The montage workload, 5530 x 5530 x 80 x 2 channels (4.9 G voxels),
    segmented whole as one request: resident on the device (CUDA events on an
    ordering stream around submit -> done) and end to end through the C ABI
    from pinned host memory (input copied inside seg_submit_volume, both
    label images and cell tables read back to host memory)."""
    import synth
    dims = (5530, 5530, 80)
    t0 = time.perf_counter()
    host = np.empty((2, dims[2], dims[1], dims[0]), dtype=np.uint16)
    for c in range(2):
        host[c] = synth.montage(channel=c)
    gen_s = time.perf_counter() - t0
    vox = host.size
    stream = torch.cuda.Stream()
    ctx = seg.seg_create(device=local, flags=seg.SEG_PROFILE, order_stream=stream.cuda_stream)
    out = {"dims": list(dims), "channels": 2, "voxels": int(vox), "generation_s": gen_s}
    try:
        d_in = torch.from_numpy(host.view(np.int16)).to("cuda:%d" % local)

        def dev_step():
            r = seg.seg_submit_volume(ctx, d_in, dims=dims, channels=2)
            seg.seg_flush(ctx)
            seg.seg_enqueue_wait(ctx, r, stream.cuda_stream)
            return r

        def finish(r):
            if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            seg.seg_release(ctx, r)

        finish(dev_step())
        torch.cuda.synchronize()
        seg.seg_reset_stats(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            finish(dev_step())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = seg.seg_get_stats(ctx)
        kernel_ms = {n: round(v["ms"] / steps, 3) for n, v in st["kernels"].items() if v["ms"] / steps > 0.05}
        del d_in
        torch.cuda.empty_cache()
        peak, _ = peaks()
        out["device"] = {"ms": ms, "gvox_s": vox / (ms / 1e3) / 1e9,
                         "hbm_fraction": vox * ALGO_BYTES_PER_VOXEL / (ms / 1e3) / 1e9 / peak,
                         "kernel_ms": kernel_ms}
        pin = torch.from_numpy(host.view(np.int16)).pin_memory()
        labs = [torch.empty(host[0].size, dtype=torch.int32).pin_memory() for _ in range(2)]
        walls = []
        for i in range(steps + 1):
            t0 = time.perf_counter()
            r = seg.seg_submit_volume(ctx, pin, dims=dims, channels=2)
            seg.seg_flush(ctx)
            if seg.seg_wait(ctx, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            for c in range(2):
                seg.seg_read_labels(ctx, r, c, labs[c])
                seg.seg_read_features(ctx, r, c)
            seg.seg_release(ctx, r)
            if i:
                walls.append(time.perf_counter() - t0)
        w = statistics.median(walls)
        out["e2e"] = {"ms": w * 1e3, "gvox_s": vox / w / 1e9, "h2d_bytes": int(host.nbytes),
                      "d2h_bytes": int(4 * vox), "read": "dense labels + cells, both channels"}
    finally:
        seg.seg_destroy(ctx)
    return out


def serving(seg, torch, local, n_requests, rate, flags, max_inflight, queued=False):
    """Open-loop Poisson request stream (2-channel volumes, sizes log-uniform
    from 128^3 to 2048x2048x64) through the C ABI from pinned host memory.
    Latency = completion observed by the runtime - arrival time."""
    import synth
    reqs = synth.serving_requests(seed=5, n=n_requests, rate=rate)
    maxn = max(d[0] * d[1] * d[2] for _, d in reqs)
    # one pinned pool [channel 0 | channel 1] of the largest size; a request
    # of n voxels per channel uses its first 2n voxels as [2][Z][Y][X]
    base = np.empty(2 * maxn, dtype=np.uint16)
    base[:maxn] = synth.density_volume((2048, 2048, 64), synth.mix_seed(5, 1)).reshape(-1)[:maxn]
    base[maxn:] = synth.density_volume((2048, 2048, 64), synth.mix_seed(5, 2)).reshape(-1)[:maxn]
    pool = torch.from_numpy(base.view(np.int16)).pin_memory()
    ctx = seg.seg_create(device=local, flags=flags, hbm_budget_bytes=120 * 10 ** 9, max_inflight=max_inflight)
    lat = []
    phases = []
    vox = 0
    done_at = []
    lock = threading.Lock()
    pending = []
    finished = threading.Event()

    def waiter():
        while True:
            with lock:
                item = pending.pop(0) if pending else None
            if item is None:
                if finished.is_set():
                    return
                time.sleep(0.0002)
                continue
            rid, arrival, submit_wall, nvox = item
            st = seg.seg_wait(ctx, rid)
            sub_ms, adm_ms, lau_ms, done_ms = seg.seg_request_times(ctx, rid)
            if st != seg.SEG_DONE:
                raise RuntimeError("request failed")
            lat.append((done_ms - sub_ms) + (submit_wall - arrival) * 1e3)
            # where the time went: arrival -> submit returned (host wait and
            # copy), -> launch (waiting for a slot), -> done (on the GPU)
            phases.append(((submit_wall - arrival) * 1e3, lau_ms - sub_ms, done_ms - lau_ms))
            done_at.append(submit_wall + (done_ms - sub_ms) / 1e3)
            seg.seg_release(ctx, rid)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for arrival, (X, Y, Z) in reqs:
        n = X * Y * Z
        host = pool[:2 * n]
        while True:
            left = arrival - (time.perf_counter() - t0)
            if left <= 0:
                break
            if left > 0.001:
                time.sleep(left - 0.0005)
        a_wall = t0 + arrival
        # queued: the call only queues the copy (the pool never changes, so
        # it stays valid until the request is done)
        rid = seg.seg_submit_volume(ctx, host, dims=(X, Y, Z), channels=2, keep_host_input=queued)
        s_wall = time.perf_counter()
        vox += 2 * n
        with lock:
            pending.append((rid, a_wall, s_wall, 2 * n))
    finished.set()
    th.join()
    seg.seg_destroy(ctx)
    span = max(done_at) - t0
    lat = np.sort(np.array(lat))
    ph = np.array(phases)
    parts = {name: {"p50_ms": float(np.percentile(ph[:, i], 50)), "p99_ms": float(np.percentile(ph[:, i], 99))}
             for i, name in enumerate(("submit", "wait_slot", "gpu"))}
    return {"requests": len(reqs), "rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "phases": parts,
            "achieved_gvox_s": vox / span / 1e9,
            "offered_gvox_s": vox / reqs[-1][0] / 1e9}


def e2e_run(seg, torch, dist, args, local, dev, ws, stream, h_in, dims, T, C, group, read, queued=True, ahead=12):
    """Steps through the C ABI from pinned host buffers.  One thread submits
    (each submit copies its frame host->device) and flushes every `group`
    frames; this thread waits for the frames in order, reads each channel's
    result back and releases the frame, so the two directions of the host
    link and the kernels overlap.  read = "runs": the label runs and cells
    (the complete segmentation: each cell's voxels as x-runs, and its
    features); read = "labels": the dense uint32 label images and cells.
    queued: the submits only queue their copies (the pinned inputs stay
    unchanged until each frame is done), at most `ahead` frames beyond the
    last frame read back, so the copies run back to back while reads that
    share the host link never wait behind a long queue of them."""
    X, Y, Z = dims
    # with queued copies every submit returns at once, so a batch is capped
    # at one flush group (else the first batch would wait for every copy)
    ctx2 = seg.seg_create(device=local, max_inflight=3, max_batch_volumes=group * C if queued else 0)
    dense = torch.empty((T, C, Z, Y, X), dtype=torch.int32).pin_memory() if read == "labels" else None
    run_buf = None
    d2h = [0]
    phases = {"inputs_sent_ms": [], "step_ms": []}

    def step():
        q, err = [], []
        done, stop = [0], [False]
        cv = threading.Condition()
        t_start = time.perf_counter()

        def submitter():
            try:
                for t in range(T):
                    if queued:
                        # at most `ahead` frames queued beyond the last one read back
                        with cv:
                            cv.wait_for(lambda: done[0] >= t - ahead or stop[0])
                    if stop[0]:
                        return
                    r = seg.seg_submit_volume(ctx2, h_in[t], dims=(X, Y, Z), channels=C, keep_host_input=queued)
                    if (t + 1) % group == 0 or t + 1 == T:
                        seg.seg_flush(ctx2)
                    with cv:
                        q.append(r)
                        cv.notify()
                phases["inputs_sent_ms"].append((time.perf_counter() - t_start) * 1e3)
            except BaseException as e:  # surfaced by the reader below
                err.append(e)
                with cv:
                    cv.notify()

        th = threading.Thread(target=submitter)
        th.start()
        nb = 0
        try:
            for t in range(T):
                with cv:
                    cv.wait_for(lambda: len(q) > t or err)
                    if len(q) <= t:
                        break
                    r = q[t]
                if seg.seg_wait(ctx2, r) != seg.SEG_DONE:
                    raise RuntimeError("request failed")
                for c in range(C):
                    if dense is not None:
                        seg.seg_read_labels(ctx2, r, c, dense[t, c])
                        nb += dense[t, c].numel() * 4
                    else:
                        nb += seg.seg_read_label_runs(ctx2, r, c, run_buf[t][c]).numel()
                    cells, _ = seg.seg_read_features(ctx2, r, c)
                    nb += cells.nbytes
                seg.seg_release(ctx2, r)
                with cv:
                    done[0] = t + 1
                    cv.notify_all()
        finally:
            with cv:  # a reader that stops early releases a waiting submitter
                stop[0] = True
                cv.notify_all()
            th.join()
        if err:
            raise err[0]
        d2h[0] = nb
        phases["step_ms"].append((time.perf_counter() - t_start) * 1e3)

    if read == "runs":
        # size one pinned buffer per volume-channel from a first pass
        counts = []
        for t in range(T):
            r = seg.seg_submit_volume(ctx2, h_in[t], dims=(X, Y, Z), channels=C)
            seg.seg_flush(ctx2)
            if seg.seg_wait(ctx2, r) != seg.SEG_DONE:
                raise RuntimeError("request failed")
            counts.append([len(seg.seg_read_label_runs(ctx2, r, c)) for c in range(C)])
            seg.seg_release(ctx2, r)
        run_buf = [[torch.empty(12 * (n + n // 4 + 1024), dtype=torch.uint8).pin_memory() for n in row]
                   for row in counts]
    for _ in range(max(1, min(args.warmup, 2))):
        step()
    for v in phases.values():
        v.clear()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n2 = max(1, min(args.steps, args.e2e_steps))
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(n2):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ems = max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3), dev, ws)
    seg.seg_destroy(ctx2)
    return {"value": None, "unit": "Gvoxels/s", "h2d_bytes_per_step": int(h_in.numel() * 2),
            "d2h_bytes_per_step": int(d2h[0]), "steps": n2, "read": read,
            "pipeline": "submit thread (%s) + read thread, flush every %d frames" % (
                "copies queued, %d frames ahead" % ahead if queued else "copies awaited", group),
            "phases_ms": {k: round(statistics.median(v), 2) for k, v in phases.items() if v},
            "step_ms_max": round(max(phases["step_ms"]), 2) if phases["step_ms"] else None,
            "steps_timed": n2, "ms": ems}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-group", type=int, default=6, help="frames per flush in the e2e pipeline")
    ap.add_argument("--e2e-copies", choices=("queued", "awaited"), default="awaited",
                    help="e2e submits queue their input copies, or wait for each")
    ap.add_argument("--e2e-ahead", type=int, default=12, help="queued copies: frames submitted beyond the last read")
    ap.add_argument("--inflight", type=int, default=1,
                    help="batches in flight; 1 keeps per-kernel CUDA-event times free of overlap")
    ap.add_argument("--frames", type=int, default=FRAMES,
                    help="time-lapse frames per step (fewer frames: a small case for profiling)")
    ap.add_argument("--tile", default="", help="force the tile height and z-chunk, e.g. 32,64")
    ap.add_argument("--denoise-radius", type=int, default=8,
                    help="also time the stage with the denoise front end on channel 0 (0 skips)")
    ap.add_argument("--closing-radius", type=int, default=1,
                    help="also time the stage with the foreground closed by this ball (0 skips)")
    ap.add_argument("--register", type=int, default=1,
                    help="also time the montage registration of a 3x3 montage of 1024x1024x64 tiles (0 skips)")
    ap.add_argument("--mrf-iterations", type=int, default=20,
                    help="also time the stage with the MRF vessel denoise, at most this many steps (0 skips)")
    ap.add_argument("--distance-weights", default="16,16,25",
                    help="also time the vessel-channel distance map with these weights of dx^2, dy^2, "
                         "dz^2 (0.8 x 0.8 x 1.0 um in 0.2 um units; 0 skips)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-uneven", action="store_true", help="skip the 48 uneven volumes and the single frame")
    ap.add_argument("--no-forms", action="store_true", help="skip the plain per-frame comparison")
    ap.add_argument("--montage", type=int, default=1, help="1: segment the 5530x5530x80x2 montage as well")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="Poisson requests (200/s) for the served latency; 0 skips serving")
    ap.add_argument("--serving-copies", choices=("queued", "awaited"), default="awaited",
                    help="serving: queue each request's input copy, or await it in the submit call")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
