#!/usr/bin/env python3
"""Throughput benchmark of the RGB-D Gaussian-mixture background subtraction
and fusion tick on GB300.

One step = one tick of the whole path (colour mixture, depth mixture, List-1
fusion, bit-packed mask) over one frame of every camera of the workload. The
default workload is c2: 64 cameras at mixed resolutions advanced by one
pooled launch per tick (CUDA graph, online-tuned launch shape), FP32 state.
The metric is Mpixel-frames/s; the JSON line also carries the HBM roofline
fraction of the pooled kernel, per-tick latency percentiles, an end-to-end
figure with host frames and masks, the same cameras one launch per camera
(`plain`), the same cameras with FP16/BF16 state (`fp16_state`), a short run
of the serving engine with frame-latency percentiles (`serving`), and the
FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2]
  python bench.py --impl reference ...   # the oracle arm, on host cores

Frames are synthetic (seeded generator standing in for Kinect captures) and
resident in device memory before the timed region. Under torchrun every rank
runs its own cameras (weak scaling, no data-path collective); the timed
region is bracketed by a barrier and a device synchronisation and the
slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PARAMS = dict(alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05)
WORKLOADS = {
    "c0": dict(name="single camera 640x480, M=3, FP32 state, 100-frame sequence",
               H=480, W=640, M=3, kind=0, frames=100, prec=0),
    "c1": dict(name="single camera 1920x1080, M=5, FP32 state, 300-frame sequence",
               H=1080, W=1920, M=5, kind=1, frames=300, prec=0),
    "c2": dict(name="64 cameras (16 each at 320x240, 640x480, 1280x720, 1920x1080), M from "
                    "{3,5} by seed, FP32 state, 300-frame sequences, one persistent launch per "
                    "tick (CUDA graph, autotuned launch shape)",
               pool=True, cams_per_res=16, frames=300, prec=0, M=5),
    "c3": dict(name="the 64-camera mix of c2 with FP16 means/variances and BF16 weights (FP32 "
                    "arithmetic), 1000 ticks over 300 resident frames per camera",
               pool=True, cams_per_res=16, frames=300, prec=1, M=5),
}
WORKLOADS["c4"] = dict(
    name="serving: 256 cameras (64 each at 320x240, 640x480, 1280x720, 1920x1080), M from {3,5} "
         "by seed, FP16/BF16 state, sessions joining and leaving on a seeded Poisson schedule "
         "(mean session 600 frames, 75% of cameras live on average), 30 fps per camera with "
         "+-2 ms jitter, 80 GB memory budget, continuous batching",
    serve=True, cams_per_res=64, prec=1, M=5, fps=30.0, session_frames=600, live_fraction=0.75,
    budget_gb=80.0, duration_s=20.0, tight_budget_gb=8.0, tight_duration_s=8.0, frames=8)
CAMERA_RESOLUTIONS = [(240, 320), (480, 640), (720, 1280), (1080, 1920)]
KERNELS = {"staged": 0, "direct": 1}
METRIC = "Mpixel-frames/s (RGB+depth GMM+fusion)"
UNIT = "Mpixel-frames/s"
FALLBACK_HBM_GBS = 6800.0
# end-to-end passes take at least this many steps (fewer would mostly time the
# pipeline filling and draining)
E2E_MIN_STEPS = 200
L2_BYTES = 129 * 1024 * 1024
CSRC = os.path.join(ROOT, "paper_2110_14934_gb300", "csrc")
# Committed ncu captures whose DRAM traffic the roofline quotes, keyed by
# (kernel, state precision): the profile, the kernel sources the capture was
# taken on (a capture of other sources is not quoted) and the suffix of its
# keys. The pooled capture is a smaller camera mix than the bench's; its
# traffic is scaled to the bench's launch by the algorithmic bytes (both
# grow with the pixels, since state, frames and masks are each read or
# written once per pixel).
TRAFFIC_RECORDS = {
    ("tick", 0): ("gmm_tick_f32_m5_1920x1080.md", ("gmm_device.cuh", "gmm_kernels.cu"), ""),
    ("tick", 1): ("gmm_tick_f16_m5_1920x1080.md", ("gmm_device.cuh", "gmm_kernels.cu"), ""),
    ("pool", 0): ("gmm_pool_tick_mixed_cameras.md", ("gmm_device.cuh", "gmm_pool_kernel.cu"), "_f32"),
    ("pool", 1): ("gmm_pool_tick_mixed_cameras.md", ("gmm_device.cuh", "gmm_pool_kernel.cu"), "_f16"),
    ("pool_flat", 0): ("gmm_pool_tick_mixed_cameras.md", ("gmm_device.cuh", "gmm_pool_kernel.cu"),
                       "_flat_f32"),
    ("pool_flat", 1): ("gmm_pool_tick_mixed_cameras.md", ("gmm_device.cuh", "gmm_pool_kernel.cu"),
                       "_flat_f16"),
    # one-pass captures of the full 64-camera launch (quoted only for that launch)
    ("pool_full", 0): ("gmm_pool_tick_mixed_cameras.md", ("gmm_device.cuh", "gmm_pool_kernel.cu"),
                       "_full_f32"),
    ("pool_full", 1): ("gmm_pool_tick_mixed_cameras.md", ("gmm_device.cuh", "gmm_pool_kernel.cu"),
                       "_full_f16"),
}
KERNEL_SOURCES = [os.path.join(CSRC, f) for f in TRAFFIC_RECORDS[("tick", 0)][1]]


def bytes_per_pixel(M: int, prec: int) -> float:
    """Algorithmic bytes per pixel and tick: state read + written (8 values
    per component: 4 bytes each in FP32, 2 in FP16/BF16), RGB (3) + depth (2)
    read, the List-1 byte read and written (2), one mask bit (1/8)."""
    per_comp = 64 if prec == 0 else 32
    return per_comp * M + 3 + 2 + 2 + 0.125


def kernel_source_hash(sources=None) -> str:
    """Hash of the kernel sources' code: comments removed and whitespace
    collapsed, so only a change of the code itself voids a recorded capture."""
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kind: str, prec: int, launch_bytes: float, exact: bool = False):
    """DRAM bytes per launch (read + write) from the committed ncu summary of
    this kernel, if it was taken on the current kernel sources; scaled to
    launch_bytes when the capture was a smaller case. exact: only a capture
    of a launch with these very algorithmic bytes. Else None."""
    rec = TRAFFIC_RECORDS.get((kind, prec))
    if rec is None:
        return None
    path = os.path.join(ROOT, "profiles", rec[0])
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(rf"traffic_bytes_per_launch{rec[2]}\s*=\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256_16\s*=\s*([0-9a-f]+)", text)
    a = re.search(rf"algorithmic_bytes_per_launch{rec[2]}\s*=\s*([0-9.eE+]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash([os.path.join(CSRC, f) for f in rec[1]]):
        return None
    if exact and (not a or abs(float(a.group(1)) - launch_bytes) > 1e-9 * launch_bytes):
        return None
    return float(m.group(1)) * (launch_bytes / float(a.group(1)) if a else 1.0)


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- distributed
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(base: int, rank: int) -> int:
    """Each rank owns its own camera: an independent seeded sequence."""
    return base + 7919 * rank


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a float over ranks (the slowest rank's time); identity at N=1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mpx_per_s(world: int, steps: int, pixels_per_step: int, max_ms: float) -> float:
    """Whole-job throughput: every rank processed `steps` frames of
    `pixels_per_step` pixels; the job took the slowest rank's time."""
    return world * steps * pixels_per_step / (max_ms / 1e3) / 1e6


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a window."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.samples = []
        self.t0 = self.t1 = None
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", str(period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def wait_first(self, timeout=10.0):
        t = time.time()
        while self.proc and not self.samples and time.time() - t < timeout:
            time.sleep(0.05)

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()
        time.sleep(0.12)  # let the sample straddling the end arrive

    def close(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or self.t0 is None:
            return None
        win = [s for (t, s) in self.samples if self.t0 <= t <= self.t1]
        window = "timed"
        if not win:  # region shorter than the sampling period: nearest sample
            near = sorted(self.samples, key=lambda ts: abs(ts[0] - self.t1))[:1]
            win = [s for (_, s) in near]
            window = "nearest"
        sm, mx, reasons = [], [], set()
        for s in win:
            try:
                sm.append(float(s[1]))
                mx.append(float(s[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(self.REASONS, s[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window": window}


# ---------------------------------------------------------------- oracle arm
def oracle_rate(wl: dict, frames: int, rows: int, seed: int):
    """Time the FP64 oracle on `rows` rows (a horizontal band through the
    middle) of the first `frames` frames of the workload. Returns
    (Mpixel-frames/s, seconds, sample description). Single thread."""
    import oracle as O
    import synth
    H, W, M = wl["H"], wl["W"], wl["M"]
    rows = max(1, min(rows, H))
    y0 = (H - rows) // 2
    s = synth.scene(seed, H, W, wl["kind"])
    rgb, dep, _ = synth.rows_host(s, 0, frames, y0, rows)
    g = O.OracleGMM(rows, W, M, **{k: PARAMS[k] for k in ("alpha", "match_k", "bg_T", "init_var", "init_w")})
    g.tick(rgb[0], dep[0])  # first frame initialises; not timed
    t = time.perf_counter()
    for f in range(1, frames):
        g.tick(rgb[f], dep[f])
    dt = time.perf_counter() - t
    px = (frames - 1) * rows * W
    return px / dt / 1e6, dt, f"frames 1-{frames - 1} of the sequence, rows {y0}-{y0 + rows - 1} " \
                              f"({rows}x{W} px per frame), FP64, 1 thread"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_band_worker(bands, warmup, steps, barrier, out):
    """One oracle process: bands = [(H, W, M, seed, kind, y0, rows, nf)]. Ticks
    each band `warmup` times (the first tick initialises), waits for the other
    processes, then times `steps` ticks of every band. Puts (pixels, seconds)."""
    import oracle as O
    import synth
    work = []
    for (H, W, M, seed, kind, y0, rows, nf) in bands:
        rgb, dep, _ = synth.rows_host(synth.scene(seed, H, W, kind), 0, nf, y0, rows)
        g = O.OracleGMM(rows, W, M, **PARAMS)
        work.append((g, rgb, dep, nf, rows * W))
    for k in range(warmup):
        for g, rgb, dep, nf, _ in work:
            g.tick(rgb[k % nf], dep[k % nf])
    barrier.wait()
    t = time.perf_counter()
    for k in range(steps):
        for g, rgb, dep, nf, _ in work:
            f = (warmup + k) % nf
            g.tick(rgb[f], dep[f])
    dt = time.perf_counter() - t
    out.put((steps * sum(w[4] for w in work), dt))


def oracle_parallel(bands, warmup, steps, procs):
    """The oracle, unchanged, in `procs` spawned processes at once, each over
    its own row bands (pixels are independent, so the split is exact).
    Returns (Mpixel-frames/s over the slowest process's time, seconds)."""
    import multiprocessing as mp
    import oracle as O
    import synth
    O.lib()              # built here, before the processes load them
    synth.host_lib()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    out = ctx.Queue()
    per = [[] for _ in range(procs)]
    for i, b in enumerate(bands):
        per[i % procs].append(b)
    ps = [ctx.Process(target=_oracle_band_worker, args=(per[i], warmup, steps, barrier, out))
          for i in range(procs)]
    for p_ in ps:
        p_.start()
    res = [out.get(timeout=600) for _ in ps]
    for p_ in ps:
        p_.join(timeout=60)
    px = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return px / dt / 1e6, dt


def split_rows(H, W, M, seed, kind, y0, rows, nf, parts):
    """Row band [y0, y0 + rows) cut into at most `parts` contiguous bands."""
    parts = max(1, min(parts, rows))
    cuts = [y0 + (rows * i) // parts for i in range(parts + 1)]
    return [(H, W, M, seed, kind, cuts[i], cuts[i + 1] - cuts[i], nf)
            for i in range(parts) if cuts[i + 1] > cuts[i]]


def oracle_all_cores(wl, frames, seed):
    """The oracle over every row of `frames` frames of the workload's camera,
    one band of rows per host core. Returns (Mpixel-frames/s, seconds, cores,
    sample description)."""
    H, W, M = wl["H"], wl["W"], wl["M"]
    n = host_cores()
    bands = split_rows(H, W, M, seed, wl["kind"], 0, H, frames, n)
    v, dt = oracle_parallel(bands, 1, frames - 1, len(bands))
    return v, dt, len(bands), (f"frames 1-{frames - 1} of the sequence, all {H}x{W} px, "
                               f"{len(bands)} processes over row bands, FP64")


def oracle_many_cameras(wl, seconds: float):
    """The oracle on all host cores over a band of rows of one camera per
    resolution of a many-camera workload, each band ticking through
    consecutive frames; sized for about `seconds` of wall time. Returns the
    cpu_baseline dict."""
    cams = reference_cameras(wl)
    procs = host_cores()
    H0, W0, M0, s0, k0 = max(cams, key=lambda c: c[0] * c[1])
    probe_rate, _, _ = oracle_rate(dict(H=H0, W=W0, M=M0, kind=k0), 3, 16, s0)
    steps = 8
    px_per_cam = seconds * probe_rate * procs * 1e6 / (steps + 1) / len(cams)
    bands, descr = [], []
    for (H, W, M, seed, kind) in cams:
        rows = int(max(1, min(H, px_per_cam / W)))
        y0 = (H - rows) // 2
        bands += split_rows(H, W, M, seed, kind, y0, rows, steps + 1, procs)
        descr.append(f"rows {y0}-{y0 + rows - 1} of a {W}x{H} M={M} camera")
    procs = min(procs, len(bands))
    value, dt = oracle_parallel(bands, 1, steps, procs)
    return {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"frames 1-{steps}: " + "; ".join(descr) + f", FP64, {procs} processes "
                      "over row bands", "seconds": dt}


def reference_cameras(wl):
    """(H, W, M, seed, scene kind) the reference arm samples: the workload's
    camera, or one camera per resolution of a many-camera mix."""
    if wl.get("pool") or wl.get("serve"):
        mix = camera_mix(wl["cams_per_res"], 0)
        return [(H, W, M, seed, 1) for (H, W, M, seed) in mix[::wl["cams_per_res"]]]
    return [(wl["H"], wl["W"], wl["M"], 1, wl["kind"])]


def run_reference(args, wl):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    cams = reference_cameras(wl)
    steps = args.steps + args.warmup
    procs = host_cores()
    # size each step's sample so that warmup + steps take about a minute on
    # all host cores (one process per core, each over its own rows)
    H0, W0, M0, s0, k0 = max(cams, key=lambda c: c[0] * c[1])
    probe_rate, _, _ = oracle_rate(dict(H=H0, W=W0, M=M0, kind=k0), 3, 16, s0)
    target_s = float(os.environ.get("GMM_REFERENCE_SECONDS", "60"))
    px_per_cam = target_s * probe_rate * procs * 1e6 / max(steps, 1) / len(cams)
    bands, descr = [], []
    for (H, W, M, seed, kind) in cams:
        rows = int(max(1, min(H, px_per_cam / W)))
        y0 = (H - rows) // 2
        nf = min(wl["frames"], steps + 1)
        bands += split_rows(H, W, M, seed, kind, y0, rows, nf, procs)
        descr.append(f"rows {y0}-{y0 + rows - 1} of a {W}x{H} M={M} camera")
    procs = min(procs, len(bands))
    value, dt = oracle_parallel(bands, args.warmup, args.steps, procs)
    sample = ("each step: " + "; ".join(descr) + f" (one frame each), FP64, {procs} processes "
              "over row bands")
    cfg = (pool_config(args.workload, wl, world, camera_mix(wl["cams_per_res"], 0), None, None)
           if (wl.get("pool") or wl.get("serve")) else config_dict(args.workload, wl, world))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def model_flags(args, G) -> int:
    """Model flags the options ask for (storage options only; the method's
    readings stay the default)."""
    return G.FLAG_STOCHASTIC_WEIGHTS if getattr(args, "stochastic_weights", False) else 0


def config_dict(key, wl, world):
    state_mb = wl["H"] * wl["W"] * wl["M"] * (32 if wl["prec"] == 0 else 16) / 1e6
    return {"workload": f"{key}: {wl['name']}", "H": wl["H"], "W": wl["W"], "M": wl["M"],
            "state": "f32" if wl["prec"] == 0 else "f16/bf16",
            "alpha": PARAMS["alpha"], "k": PARAMS["match_k"], "T": PARAMS["bg_T"],
            "cameras_per_gpu": 1, "parallelism": f"camera-sharded x{world}",
            "l2": f"state {state_mb:.0f} MB per camera vs L2 129 MB: "
                  + ("inputs larger than L2 between iterations" if state_mb * 1e6 > L2_BYTES
                     else "state may stay L2-resident")}


# ---------------------------------------------------------------- our arm
def run_gmm(args, wl):
    import torch
    import paper_2110_14934_gb300 as G
    import synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    H, W, M, prec = wl["H"], wl["W"], wl["M"], wl["prec"]
    nf = min(wl["frames"], args.frames) if args.frames > 0 else wl["frames"]
    scene = synth.scene(rank_seed(1, rank), H, W, wl["kind"])
    rgb_d, dep_d, _ = synth.frames_device(scene, 0, nf, device=dev, with_gt=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    # --morph: the handle runs the tick and the 3x3 opening of the fused mask
    # back to back in every step (gmm_apply with morph_open = 1).
    g = G.GMM(H, W, M, precision=prec, device=dev, flags=model_flags(args, G),
              morph_open=args.morph, **PARAMS)
    g.set_kernel(KERNELS[args.kernel], args.variant, args.ctas)
    mask = g.new_mask()
    K, Wm = args.steps, args.warmup

    def step(f):
        g.apply(rgb_d[f], dep_d[f], mask, stream=stream)

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.wait_first()
    for k in range(Wm):
        step(k % nf)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier(world, dev)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t_start.record(stream)
    for k in range(K):
        step((Wm + k) % nf)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world, dev)
    clk = None
    if clocks:  # the sampler stops with the timed region: nothing polls the GPU after it
        clocks.stop()
        clk = clocks.summary()
        clocks.close()
    local_ms = t_start.elapsed_time(t_end)
    total_ms = reduce_max(local_ms, world, dev)
    value = aggregate_mpx_per_s(world, K, H * W, total_ms)

    # Roofline of the tick kernel. Without --morph it is the only work in the
    # timed region (one launch per step, back to back on one stream), so its
    # average launch duration is the region's event time over K. With --morph
    # a separate pass times a handle without the opening back to back (the
    # tick's duration), then steps of tick + gmm_morph_open3 with events
    # around the opening (its own duration; the events add a little to it).
    bpp = bytes_per_pixel(M, prec)
    morph_info = None
    if args.morph:
        n_att = min(K, 2000)
        solo = G.GMM(H, W, M, precision=prec, device=dev, flags=model_flags(args, G), **PARAMS)
        solo.set_kernel(KERNELS[args.kernel], args.variant, args.ctas)
        scratch = solo.new_mask()
        for k in range(Wm):
            solo.apply(rgb_d[k % nf], dep_d[k % nf], scratch, stream=stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for k in range(n_att):
            f = (Wm + k) % nf
            solo.apply(rgb_d[f], dep_d[f], scratch, stream=stream)
        a1.record(stream)
        marks = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_att)]
        for k in range(n_att):
            f = (Wm + k) % nf
            solo.apply(rgb_d[f], dep_d[f], scratch, stream=stream)
            marks[k][0].record(stream)
            G.morph_open3(scratch, mask, H, W, stream=stream)
            marks[k][1].record(stream)
        torch.cuda.synchronize()
        tick_s = a0.elapsed_time(a1) / n_att / 1e3
        morph_s = sum(b.elapsed_time(c) for b, c in marks) / n_att / 1e3
        solo.close()
        avg_kernel_s = tick_s
        morph_bytes = 2 * H * G.mask_words_per_row(W) * 4
        morph_info = {"kernel": "k_morph_open3", "avg_us": morph_s * 1e6,
                      "algorithmic_bytes_per_launch": morph_bytes,
                      "achieved_gbs": morph_bytes / morph_s / 1e9,
                      "step_us_with_opening": local_ms / K * 1e3,
                      "tick_alone_us": tick_s * 1e6,
                      "opening_cost_us_per_step": local_ms / K * 1e3 - tick_s * 1e6,
                      "attribution": f"{n_att} ticks alone back to back; {n_att} openings "
                                     "between two events"}
    else:
        avg_kernel_s = local_ms / K / 1e3
    achieved = H * W * bpp / avg_kernel_s / 1e9

    # Per-tick device latency: a separate pass with an event pair per tick.
    n_lat = min(K, 2000)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n_lat)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n_lat)]
    for k in range(n_lat):
        f = (Wm + K + k) % nf
        starts[k].record(stream)
        step(f)
        ends[k].record(stream)
    torch.cuda.synchronize()
    tick_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    peak, peak_src = measured_hbm_peak()
    # the captures are of the default kernel instance on the 1920x1080 M=5 workload
    traffic = (recorded_traffic("tick", prec, H * W * bpp)
               if args.workload == "c1" and not args.frame_size and args.kernel == "direct"
               and args.variant == 0 and not model_flags(args, G) else None)

    # end to end through the host-memory C-ABI path (pipelined, Fig. 4(a))
    e2e = run_e2e(G, torch, g_args=(H, W, M, prec), frames=(rgb_d, dep_d), dev=dev,
                  steps=args.e2e_steps or max(K, E2E_MIN_STEPS), warmup=Wm, world=world,
                  kernel=(KERNELS[args.kernel], args.variant, args.ctas), morph=args.morph)
    del rgb_d, dep_d
    cpu = None
    if rank == 0 and world == 1 and args.cpu_frames > 0:
        v1, secs1, sample1 = oracle_rate(wl, args.cpu_frames, args.cpu_rows or H, rank_seed(1, 0))
        if args.cpu_all_frames > 1:
            v, secs, cores, sample = oracle_all_cores(wl, args.cpu_all_frames, rank_seed(1, 0))
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                   "seconds": secs, "single_thread": {"value": v1, "cores": 1,
                                                      "sample": sample1, "seconds": secs1}}
        else:
            cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample1,
                   "seconds": secs1}
    if rank == 0:
        tick_sorted = sorted(tick_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(args.workload, wl, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src, "algorithmic_bytes_per_px": bpp,
                         "kernel": (f"k_tick_staged<M={M},{'f32' if prec == 0 else 'f16'}>"
                                    f" variant {args.variant}" if args.kernel == "staged" else
                                    f"k_tick_{'f32' if prec == 0 else 'f16'}<M={M}>")},
            "latency_ms": {"tick_p50": pct(tick_sorted, 50), "tick_p99": pct(tick_sorted, 99),
                           "e2e_p50": e2e["lat_p50"], "e2e_p99": e2e["lat_p99"]},
            "e2e": {"value": e2e["value"], "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                    "d2h_bytes_per_step": e2e["d2h"], "path": "gmm_pipe_submit/gmm_pipe_wait, "
                    "pinned host frames, 3 frames in flight"},
            "e2e_zero_copy": {"value": e2e["zero_copy"], "unit": UNIT,
                              "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                              "path": "gmm_apply on the same page-locked host frames and masks: "
                                      "the kernel reads the frame and writes the mask over the "
                                      "host link, timed to the last mask in host memory"},
            "cpu_baseline": cpu,
            "gpu_launches": K * (2 if args.morph else 1),
            "clocks": clk,
        }
        if morph_info:
            line["config"]["morph_open"] = True
            line["morph"] = morph_info
        if model_flags(args, G):
            line["config"]["weights_rounding"] = "stochastic"
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- many cameras
def camera_mix(cams_per_res: int, rank: int):
    """(H, W, M, seed) of every camera of a rank: cams_per_res cameras at each
    resolution, each with its own seed; M drawn from {3, 5} by the seed."""
    import random
    out = []
    for ri, (H, W) in enumerate(CAMERA_RESOLUTIONS):
        for i in range(cams_per_res):
            seed = rank_seed(1000 + 100 * ri + i, rank)
            out.append((H, W, random.Random(seed).choice((3, 5)), seed))
    return out


def pool_config(key, wl, world, cams, shape, graph):
    px = sum(H * W for (H, W, _, _) in cams)
    state = sum(H * W * M * (32 if wl["prec"] == 0 else 16) for (H, W, M, _) in cams)
    return {"workload": f"{key}: {wl['name']}", "cameras_per_gpu": len(cams),
            "pixels_per_tick": px, "M3_cameras": sum(1 for c in cams if c[2] == 3),
            "M5_cameras": sum(1 for c in cams if c[2] == 5),
            "state": "f32" if wl["prec"] == 0 else "f16/bf16",
            "alpha": PARAMS["alpha"], "k": PARAMS["match_k"], "T": PARAMS["bg_T"],
            "launch": shape, "cuda_graph": graph, "parallelism": f"camera-sharded x{world}",
            "l2": f"state {state / 1e9:.1f} GB per GPU vs L2 129 MB: inputs larger than L2 "
                  "between iterations"}


def run_pool(args, wl):
    import torch
    import paper_2110_14934_gb300 as G
    import synth

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prec = wl["prec"]
    cams = camera_mix(wl["cams_per_res"], rank)
    nf = min(wl["frames"], args.frames) if args.frames > 0 else wl["frames"]
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.current_stream(dev)
    frames = []
    for (H, W, M, seed) in cams:
        r, d, _ = synth.frames_device(synth.scene(seed, H, W, 1), 0, nf, device=dev, with_gt=False)
        frames.append((r, d))
    masks = [torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device=dev)
             for (H, W, _, _) in cams]
    torch.cuda.synchronize()
    rgb_base = [f[0].data_ptr() for f in frames]
    dep_base = [f[1].data_ptr() for f in frames]
    rgb_step = [H * W * 3 for (H, W, _, _) in cams]
    dep_step = [H * W * 2 for (H, W, _, _) in cams]
    mask_ptr = [m.data_ptr() for m in masks]

    pool = G.Pool(precision=prec, max_cams=len(cams), device=dev)
    ids = [pool.admit(H, W, M, flags=model_flags(args, G), **PARAMS) for (H, W, M, _) in cams]
    pool.set_stream(stream)
    graph = not args.no_graph
    pool.use_graph(graph)

    def submit(f):
        pool.submit_many(ids, [b + f * s for b, s in zip(rgb_base, rgb_step)],
                         [b + f * s for b, s in zip(dep_base, dep_step)], mask_ptr)

    submit(0)
    pool.tick(stream)  # frame 0 initialises every model
    k = 1
    if args.pool_launch:
        pool.set_launch(*[int(v) for v in args.pool_launch.split(",")])
        shape = pool.tuning()[1]
    elif not args.no_autotune:
        # online tuning: the first warm-up ticks of the sequence try each
        # candidate launch shape (3 ticks each) and the pool keeps the best
        pool.autotune_online(3)
        while pool.tuning()[0] and k < 2000:
            submit(k % nf)
            pool.tick(stream)
            k += 1
        torch.cuda.synchronize()
        tuning, shape = pool.tuning()
        assert not tuning, "online tuning did not finish"
        shape["tuning_ticks"] = k - 1
    else:
        shape = None
    for j in range(Wm):
        submit((k + j) % nf)
        pool.tick(stream)
    F0 = k + Wm  # frames consumed before the timed region
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.wait_first()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world, dev)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t0.record(stream)
    for k in range(K):
        submit((F0 + k) % nf)
        pool.tick(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world, dev)
    clk = None
    if clocks:  # the sampler stops with the timed region: nothing polls the GPU after it
        clocks.stop()
        clk = clocks.summary()
        clocks.close()
    local_ms = t0.elapsed_time(t1)
    total_ms = reduce_max(local_ms, world, dev)
    px = sum(H * W for (H, W, _, _) in cams)
    value = aggregate_mpx_per_s(world, K, px, total_ms)
    tick_bytes = sum(H * W * bytes_per_pixel(M, prec) for (H, W, M, _) in cams)
    achieved = tick_bytes / (local_ms / K / 1e3) / 1e9
    # one launch per tick up to 128 cameras (more: a launch per 128)
    flat = bool(shape) and shape.get("ctas_per_sm", 0) < 0
    traffic = recorded_traffic("pool_full", prec, tick_bytes, exact=True) if not flat else None
    traffic_note = "one-pass ncu capture of this 64-camera launch"
    if traffic is None:
        traffic = (recorded_traffic("pool_flat" if flat else "pool", prec, tick_bytes)
                   if len(cams) <= 128 else None)
        traffic_note = "scaled from an 8-camera capture by algorithmic bytes"
    peak, peak_src = measured_hbm_peak()

    # per-tick device latency
    n_lat = min(K, 500)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n_lat)]
    for k in range(n_lat):
        submit((F0 + K + k) % nf)
        ev[k][0].record(stream)
        pool.tick(stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    tick_ms = sorted(a.elapsed_time(b) for a, b in ev)

    # The plain path: one FP32 handle per camera, one launch per camera per tick.
    L = G.load_library()
    plain = [G.GMM(H, W, M, precision=G.PREC_F32, device=dev, **PARAMS) for (H, W, M, _) in cams]
    for g in plain:
        g.set_stream(stream)
    hs = [g._h for g in plain]
    n_plain = min(max(K, 100), 300)  # at least 100 ticks: a steady comparison
    for k in range(Wm):
        for i, h in enumerate(hs):
            L.gmm_apply(h, rgb_base[i] + (k % nf) * rgb_step[i], dep_base[i] + (k % nf) * dep_step[i],
                        mask_ptr[i])
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for k in range(n_plain):
        f = (Wm + k) % nf
        for i, h in enumerate(hs):
            L.gmm_apply(h, rgb_base[i] + f * rgb_step[i], dep_base[i] + f * dep_step[i], mask_ptr[i])
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = reduce_max(p0.elapsed_time(p1), world, dev)
    plain_value = aggregate_mpx_per_s(world, n_plain, px, plain_ms)
    for g in plain:
        g.close()

    e2e = run_pool_e2e(G, torch, pool, ids, cams, frames, dev, stream,
                       args.e2e_steps or min(max(K, E2E_MIN_STEPS), 600),
                       Wm, world, retune=not args.pool_launch and not args.no_autotune)
    # c2 at N = 1: the same cameras and frames with FP16/BF16 state (the
    # precision configuration) and a short run of the serving engine
    extras = args.workload == "c2" and world == 1 and not args.no_extras
    fp16 = (pool_precision_extra(G, torch, args, cams, rgb_base, dep_base, rgb_step, dep_step,
                                 mask_ptr, nf, stream, max(K, 100), Wm) if extras else None)
    serving = serving_extra(G, torch, args, dev) if extras else None
    cpu = (oracle_many_cameras(wl, args.cpu_seconds)
           if rank == 0 and world == 1 and args.cpu_seconds > 0 else None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": pool_config(args.workload, wl, world, cams, shape, graph),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "traffic_note": traffic_note,
                         "algorithmic_bytes_per_tick": tick_bytes,
                         "kernel": f"k_pool_{'flat' if flat else 'tick'}<{'f32' if prec == 0 else 'f16'}>"},
            "plain": {"value": plain_value, "unit": UNIT, "steps": n_plain,
                      "pooled_over_plain": value / plain_value,
                      "path": "the same cameras and frames, one FP32 handle per camera, one "
                              "gmm_apply launch per camera per tick"},
            "latency_ms": {"tick_p50": pct(tick_ms, 50), "tick_p99": pct(tick_ms, 99)},
            "e2e": {"value": e2e["value"], "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                    "d2h_bytes_per_step": e2e["d2h"], "launch": e2e["launch"],
                    "path": "pinned packed tick-sets -> device staging (copy stream) -> "
                            "gmm_pool_submit_many + gmm_pool_tick -> masks to pinned host "
                            "(FP16/BF16 next-tile prefetch off; the launch shape tuned in "
                            "this pipeline unless fixed)"},
            "e2e_zero_copy": {"value": e2e["zero_copy"], "unit": UNIT,
                              "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                              "launch": e2e["launch_zero_copy"],
                              "path": "gmm_pool_submit_many on the same page-locked tick-sets and "
                                      "masks: the pooled kernel reads frames and writes masks "
                                      "over the host link"},
            "cpu_baseline": cpu,
            "gpu_launches": K * pool_launches(cams, shape),
            "clocks": clk,
        }
        if fp16 is not None:
            line["fp16_state"] = fp16
        if serving is not None:
            line["serving"] = serving
        if model_flags(args, G):
            line["config"]["weights_rounding"] = "stochastic"
        print(json.dumps(line), flush=True)
    pool.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def pool_precision_extra(G, torch, args, cams, rgb_base, dep_base, rgb_step, dep_step, mask_ptr,
                         nf, stream, steps, warmup):
    """The c2 cameras and frames in a pool with FP16 means/variances and
    BF16 weights (workload c3's storage), tuned online the same way; K
    device-timed ticks. Returns the value, the pooled kernel's roofline and
    the launch shape."""
    prec = 1
    pool = G.Pool(precision=prec, max_cams=len(cams), device=stream.device)
    ids = [pool.admit(H, W, M, **PARAMS) for (H, W, M, _) in cams]
    pool.set_stream(stream)
    pool.use_graph(True)

    def submit(f):
        pool.submit_many(ids, [b + f * s for b, s in zip(rgb_base, rgb_step)],
                         [b + f * s for b, s in zip(dep_base, dep_step)], mask_ptr)

    submit(0)
    pool.tick(stream)
    pool.autotune_online(3)
    k = 1
    while pool.tuning()[0] and k < 2000:
        submit(k % nf)
        pool.tick(stream)
        k += 1
    for j in range(warmup):
        submit((k + j) % nf)
        pool.tick(stream)
    f0 = k + warmup
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for j in range(steps):
        submit((f0 + j) % nf)
        pool.tick(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    shape = pool.tuning()[1]
    pool.close()
    px = sum(H * W for (H, W, _, _) in cams)
    tick_bytes = sum(H * W * bytes_per_pixel(M, prec) for (H, W, M, _) in cams)
    achieved = tick_bytes / (ms / steps / 1e3) / 1e9
    peak, peak_src = measured_hbm_peak()
    flat = shape.get("ctas_per_sm", 0) < 0
    return {"workload": "the c2 cameras and frames with FP16 means/variances and BF16 weights "
                        "(FP32 arithmetic), as in c3",
            "value": steps * px / ms / 1e3, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
            "launch": shape,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": (recorded_traffic("pool_full", prec, tick_bytes, exact=True)
                                     if not flat else None)
                                    or (recorded_traffic("pool_flat" if flat else "pool", prec,
                                                         tick_bytes) if len(cams) <= 128 else None),
                         "algorithmic_bytes_per_tick": tick_bytes,
                         "kernel": f"k_pool_{'flat' if flat else 'tick'}<f16>"}}


def serving_setup(G, torch, wl, rank, dev):
    """Cameras of the serving workload and a small ring of page-locked host
    frames per resolution (the frames the simulated cameras deliver)."""
    import synth
    cams = camera_mix(wl["cams_per_res"], rank)
    ring = []
    for ri, (H, W) in enumerate(CAMERA_RESOLUTIONS):
        r, d, _ = synth.frames_device(synth.scene(rank_seed(5000 + ri, rank), H, W, 1), 0,
                                      wl["frames"], device=dev, with_gt=False)
        ring.append((r.cpu().pin_memory(), d.cpu().pin_memory()))
    return cams, ring


def serving_extra(G, torch, args, dev):
    """A short run of workload c4 (256 cameras, Poisson sessions, 30 fps each,
    80 GB budget, FP16/BF16 state) on the serving engine in its default
    zero-copy mode: frame latency (arrival to fused mask in host memory),
    drops and rejections; the same cameras as a genlocked rig (every camera's
    frames arrive together, so each period opens with a burst that continuous
    batching packs into few ticks); a tight 8 GB budget, to exercise
    admission control; and both schedules again in the engine's copy mode."""
    wl = WORKLOADS["c4"]
    cams, ring = serving_setup(G, torch, wl, 0, dev)
    dur = args.extra_serve_seconds
    out = {"workload": f"c4: {wl['name']}", "duration_s": dur, "unit": "ms",
           "transfer": "zero-copy: the pooled kernel reads the page-locked frames and writes "
                       "the masks in host memory"}
    st, lat, wall, _, rel_err, _, parts = serve_run(G, torch, cams, ring, wl,
                                                    int(wl["budget_gb"] * 1e9), dur, 2021)
    lat = list(lat)
    out.update({"p50": fnum(pct(lat, 50)), "p99": fnum(pct(lat, 99)), "p999": fnum(pct(lat, 99.9)),
                "max": fnum(lat[-1]) if lat else None,
                "what": "frame arrival to fused mask in host memory",
                "frames_completed": st["completed"], "frames_dropped": st["dropped"],
                "sessions_admitted": st["admitted"], "admissions_rejected": st["rejected"],
                "budget_gb": wl["budget_gb"], "ticks": st["ticks"],
                "mean_frames_per_tick": st["completed"] / max(st["ticks"], 1),
                "mpx_frames_per_s": st["pixels"] / wall / 1e6, "release_errors": len(rel_err),
                "device_ms_p99": parts["device_ms"]["p99"] if parts else None})
    st3, lat3, _, _, _, _, _ = serve_run(G, torch, cams, ring, wl, int(wl["budget_gb"] * 1e9),
                                         dur, 2021, genlocked=True)
    lat3 = list(lat3)
    out["genlocked"] = {"p50": fnum(pct(lat3, 50)), "p99": fnum(pct(lat3, 99)),
                        "p999": fnum(pct(lat3, 99.9)), "frames_completed": st3["completed"],
                        "frames_dropped": st3["dropped"], "ticks": st3["ticks"],
                        "mean_frames_per_tick": st3["completed"] / max(st3["ticks"], 1)}
    short = min(dur, 6.0)
    st2, lat2, _, _, _, _, _ = serve_run(G, torch, cams, ring, wl,
                                         int(wl["tight_budget_gb"] * 1e9), short, 77)
    out["tight_budget"] = {"budget_gb": wl["tight_budget_gb"], "duration_s": short,
                           "sessions_admitted": st2["admitted"],
                           "admissions_rejected": st2["rejected"],
                           "p99": fnum(pct(list(lat2), 99))}
    # the same two schedules with the engine's copy mode (uploads, downloads)
    cm = {}
    for key, gl in (("independent", False), ("genlocked", True)):
        stc, latc, _, _, _, _, _ = serve_run(G, torch, cams, ring, wl, int(wl["budget_gb"] * 1e9),
                                             short, 2021, genlocked=gl, transfer=G.SERVE_COPY)
        latc = list(latc)
        cm[key] = {"p50": fnum(pct(latc, 50)), "p99": fnum(pct(latc, 99)),
                   "p999": fnum(pct(latc, 99.9)), "frames_completed": stc["completed"],
                   "mean_frames_per_tick": stc["completed"] / max(stc["ticks"], 1)}
    cm["duration_s"] = short
    out["copy_mode"] = cm
    return out


def pool_launches(cams, shape):
    """Kernels per pooled tick: one per 128 cameras; the flat form launches
    each M group separately."""
    if shape and shape.get("ctas_per_sm", 0) < 0:
        ms = [M for (_, _, M, _) in cams]
        return sum((ms.count(m) + 127) // 128 for m in set(ms))
    return (len(cams) + 127) // 128


def run_pool_e2e(G, torch, pool, ids, cams, frames, dev, stream, steps, warmup, world,
                 retune=False):
    """Frames from pinned host memory each tick: every camera's frame of a
    tick is packed into one pinned buffer, uploaded with one copy into one of
    two device staging buffers on a copy stream (overlapping the previous
    tick's compute), the pool ticks from there, and the packed masks come back
    with one copy on a third stream, with the pool's FP16/BF16 next-tile
    prefetch turned off (the library documents that uploads beside each tick
    slow down under it). Then the zero-copy form, prefetch on. retune: the
    pool's online tuner runs again inside each of the two pipelines before
    its warm-up (a shape's tick period then includes what its kernel delays
    in the uploads beside it, or in its own reads over the host link)."""
    def al(x):
        return (x + 255) // 256 * 256
    off, o = [], 0
    for (H, W, _, _) in cams:
        off.append((o, o + al(H * W * 3)))
        o += al(H * W * 3) + al(H * W * 2)
    set_bytes = o
    moff, mo = [], 0
    for (H, W, _, _) in cams:
        moff.append(mo)
        mo += al(H * G.mask_words_per_row(W) * 4)
    mask_bytes = mo
    ring = 3
    host = torch.empty((ring, set_bytes), dtype=torch.uint8).pin_memory()
    for r in range(ring):
        for (a, b), (rg, dp), (H, W, _, _) in zip(off, frames, cams):
            host[r, a:a + H * W * 3].copy_(rg[r].reshape(-1))
            host[r, b:b + H * W * 2].copy_(dp[r].reshape(-1).view(torch.uint8))
    stage = torch.empty((2, set_bytes), dtype=torch.uint8, device=dev)
    dmask = torch.empty((2, mask_bytes), dtype=torch.uint8, device=dev)
    hmask = torch.empty((ring, mask_bytes), dtype=torch.uint8).pin_memory()
    up_s, down_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    up = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    down = [torch.cuda.Event() for _ in range(2)]

    def tick(k):
        b, r = k % 2, k % ring
        with torch.cuda.stream(up_s):
            up_s.wait_event(done[b])        # tick k-2 has finished reading stage b
            stage[b].copy_(host[r], non_blocking=True)
            up[b].record(up_s)
        stream.wait_event(up[b])
        stream.wait_event(down[b])          # tick k-2's masks have left dmask b
        sb, mb = stage[b].data_ptr(), dmask[b].data_ptr()
        pool.submit_many(ids, [sb + a for a, _ in off], [sb + c for _, c in off],
                         [mb + m for m in moff])
        pool.tick(stream)
        done[b].record(stream)
        with torch.cuda.stream(down_s):
            down_s.wait_event(done[b])
            hmask[k % ring].copy_(dmask[b], non_blocking=True)
            down[b].record(down_s)

    def tune(step):
        n = 0
        if retune:
            pool.autotune_online(3)
            while pool.tuning()[0] and n < 2000:
                step(n)
                n += 1
            torch.cuda.synchronize()
            assert not pool.tuning()[0], "online tuning did not finish"
        shape = dict(pool.tuning()[1])
        if retune:
            shape["tuning_ticks"] = n
        return n, shape

    pool.set_prefetch(False)
    k0, shape = tune(tick)
    for k in range(warmup):
        tick(k0 + k)
    torch.cuda.synchronize()
    barrier(world, dev)
    t = time.perf_counter()
    for k in range(steps):
        tick(k0 + warmup + k)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    barrier(world, dev)
    dt = reduce_max(dt, world, dev)
    # zero-copy: the pool reads the packed page-locked frames and writes the
    # page-locked masks directly over the host link
    hb, mb_h = host.data_ptr(), hmask.data_ptr()

    def tick_zc(k):
        r = k % ring
        pool.submit_many(ids, [hb + r * set_bytes + a for a, _ in off],
                         [hb + r * set_bytes + c for _, c in off],
                         [mb_h + r * mask_bytes + m for m in moff])
        pool.tick(stream)

    pool.set_prefetch(True)
    z0, shape_zc = tune(tick_zc)
    for k in range(warmup):
        tick_zc(z0 + k)
    torch.cuda.synchronize()
    barrier(world, dev)
    t = time.perf_counter()
    for k in range(steps):
        tick_zc(z0 + warmup + k)
    torch.cuda.synchronize()
    dz = time.perf_counter() - t
    barrier(world, dev)
    dz = reduce_max(dz, world, dev)
    px = sum(H * W for (H, W, _, _) in cams)
    return {"value": world * steps * px / dt / 1e6, "launch": shape,
            "zero_copy": world * steps * px / dz / 1e6, "launch_zero_copy": shape_zc,
            "h2d": sum(H * W * 5 for (H, W, _, _) in cams),
            "d2h": sum(H * G.mask_words_per_row(W) * 4 for (H, W, _, _) in cams)}


# ---------------------------------------------------------------- serving
def serving_schedule(n_cams, duration, fps, session_s, live_fraction, seed, genlocked=False):
    """Seeded session and frame schedule: every camera alternates idle gaps
    and sessions, both exponential (Poisson joins and leaves), with mean
    session session_s and mean gap chosen for the given live fraction; a
    live camera offers frames every 1/fps s with +-2 ms uniform jitter.
    The cameras already live when the window opens joined at unrelated
    earlier times, so each runs at its own phase (uniform in one frame
    period); genlocked: they all run at phase 0 (a synchronised rig: their
    frames arrive together, every period). Returns time-sorted events
    (t, kind, cam, k) with kind 0 = join, 1 = frame k of the session,
    2 = leave."""
    import numpy as np
    rng = np.random.default_rng(seed)                # sessions
    rng_t = np.random.default_rng([seed, 1])         # phases and jitter
    gap_s = session_s * (1.0 - live_fraction) / live_fraction
    ev = []
    for c in range(n_cams):
        live = rng.random() < live_fraction
        phase = 0.0 if genlocked or not live else rng_t.uniform(0.0, 1.0 / fps)
        t = 0.0
        while t < duration:
            if live:
                end = min(duration, t + rng.exponential(session_s))
                ev.append((t, 0, c, 0))
                k = 0
                while True:
                    tf = t + phase + k / fps + rng_t.uniform(-0.002, 0.002)
                    if tf >= end:
                        break
                    ev.append((max(t, tf), 1, c, k))
                    k += 1
                ev.append((end, 2, c, 0))
                t = end
                phase = 0.0
            else:
                t += rng.exponential(gap_s)
            live = not live
    ev.sort(key=lambda e: (e[0], e[1]))
    return ev


def serve_run(G, torch, cams, ring, wl, budget_bytes, duration, seed, queue_depth=4,
              genlocked=False, transfer=None):
    """Drive a Server through a seeded schedule in real time; returns stats.
    transfer: the engine's transfer mode (None: its default, zero-copy)."""
    import queue as pyqueue

    import numpy as np
    srv = G.Server(budget_bytes=budget_bytes, precision=wl["prec"], max_cams=len(cams),
                   queue_depth=queue_depth, transfer=transfer)
    copy_mode = transfer == G.SERVE_COPY
    # device memory for every camera's state and staging mapped before the
    # clock starts (up to the budget), so no admission maps new memory

    def al(x):
        return (x + 255) // 256 * 256
    state_all = sum(G.state_bytes(H, W, M, wl["prec"]) for (H, W, M, _) in cams)
    stage_all = sum(al(H * W * 3) + al(H * W * 2) + al(H * G.mask_words_per_row(W) * 4)
                    for (H, W, _, _) in cams) if copy_mode else 0
    cap = budget_bytes if budget_bytes else state_all + stage_all
    srv.reserve(min(state_all, cap), min(stage_all, max(cap - min(state_all, cap), 0)))
    events = serving_schedule(len(cams), duration, wl["fps"], wl["session_frames"] / wl["fps"],
                              wl["live_fraction"], seed, genlocked)
    n_slot = queue_depth + 4
    # every camera's mask buffers, carved from one page-locked allocation made
    # before the clock starts (allocating page-locked memory in the loop
    # stalls the client)
    words = [H * G.mask_words_per_row(W) for (H, W, _, _) in cams]
    pinned = torch.empty(sum(words) * n_slot, dtype=torch.int32).pin_memory()
    masks, off = {}, 0
    for c, (H, W, _, _) in enumerate(cams):
        for slot in range(n_slot):
            masks[(c, slot)] = pinned[off:off + words[c]].view(H, G.mask_words_per_row(W))
            off += words[c]
    live = {}          # camera -> server id of its current session
    slot_ticket = {}   # (camera, slot) -> ticket using that mask buffer
    rel_q = pyqueue.Queue()
    rel_err = []

    def releaser():
        while True:
            sid = rel_q.get()
            if sid is None:
                return
            try:
                srv.release(sid, 60000)
            except Exception as e:  # reported, not fatal to the run
                rel_err.append(str(e))

    import threading as th
    rt = th.Thread(target=releaser, daemon=True)
    rt.start()
    tickets, lag, admit_ms = [], [], []
    # camera of each ticket (tickets count up from 0), allocated up front: a
    # dict that grows in the real-time loop stalls it for tens of ms when it
    # resizes
    ticket_cam = np.full(sum(1 for e in events if e[1] == 1) + 1, -1, dtype=np.int32)
    # The cameras live when the window opens are admitted before the clock
    # starts (a server is up before it is measured); later joins are timed.
    n_initial = 0
    while n_initial < len(events) and events[n_initial][0] == 0.0 and events[n_initial][1] == 0:
        H, W, M, _ = cams[events[n_initial][2]]
        try:
            live[events[n_initial][2]] = srv.admit(H, W, M, **PARAMS)
        except G.GMMError as e:
            if e.code != G.EBUDGET:
                raise
        n_initial += 1
    import gc
    gc.disable()  # no collector pauses in the client's real-time loop
    t0 = srv.now() + 0.5
    stalls = []  # events the client reached > 2 ms late, with the event before
    slow_iters, waited = [], 0
    prev = (None, 0.0)
    for (t, kind, c, k) in events[n_initial:]:
        due = t0 + t
        while True:
            d = due - srv.now()
            if d <= 0:
                break
            time.sleep(d - 0.0005) if d > 0.001 else None
        ti = srv.now()
        if ti - due > 0.002 and len(stalls) < 20:
            stalls.append({"t_s": round(t, 4), "kind": kind, "late_ms": round((ti - due) * 1e3, 3),
                           "prev_kind": prev[0], "prev_call_ms": round(prev[1] * 1e3, 3)})
        H, W, M, _ = cams[c]
        if kind == 0:
            ta = time.perf_counter()
            try:
                live[c] = srv.admit(H, W, M, **PARAMS)
            except G.GMMError as e:
                if e.code != G.EBUDGET:
                    raise
            admit_ms.append((time.perf_counter() - ta) * 1e3)
        elif kind == 2:
            sid = live.pop(c, None)
            if sid is not None:
                rel_q.put(sid)
        elif c in live:
            ri = CAMERA_RESOLUTIONS.index((H, W))
            rgb_h, dep_h = ring[ri]
            slot = k % n_slot
            old = slot_ticket.get((c, slot))
            if old is not None and not srv.done(old):
                srv.wait(old, 60000)
                waited += 1
            ts1 = srv.now()
            f = (k + c) % rgb_h.shape[0]
            lag.append((srv.now() - due) * 1e3)
            try:
                ts2 = srv.now()
                tk = srv.push(live[c], rgb_h[f], dep_h[f], masks[(c, slot)], t_arrival=due)
                ts3 = srv.now()
                if ts3 - ti > 0.005 and len(slow_iters) < 10:
                    slow_iters.append({"t_s": round(t, 4), "slot_wait_ms": round((ts1 - ti) * 1e3, 3),
                                       "index_ms": round((ts2 - ts1) * 1e3, 3),
                                       "push_ms": round((ts3 - ts2) * 1e3, 3),
                                       "ticket": tk, "ts2": ts2, "ts3": ts3})
                tickets.append(tk)
                ticket_cam[tk] = c
                slot_ticket[(c, slot)] = tk
            except G.GMMError as e:
                if e.code != G.EBUDGET:
                    raise
        prev = (kind, srv.now() - ti)
    for tk in tickets:
        srv.wait(tk, 60000)
    t_end = srv.now()
    gc.enable()
    for sid in list(live.values()):
        rel_q.put(sid)
    rel_q.put(None)
    rt.join()
    st = srv.stats()
    lat = np.sort(srv.latencies_ms())
    trs = srv.traces()
    parts = latency_breakdown(trs, ticket_cam, cams, t0)
    for it in slow_iters:  # inside gmm_server_push: before / after its lock
        row = trs[trs["ticket"] == it.pop("ticket")]
        ts2, ts3 = it.pop("ts2"), it.pop("ts3")
        if row.size:
            it["to_lock_ms"] = round((float(row["t_pushed"][0]) - ts2) * 1e3, 3)
            it["after_lock_ms"] = round((ts3 - float(row["t_pushed"][0])) * 1e3, 3)
    if parts is not None:
        parts["client_stalls"] = stalls[:3]
        parts["client_slow_pushes"] = slow_iters
        parts["client_slot_waits"] = waited
    srv.close()
    lag.sort()
    admit_ms.sort()
    return st, lat, t_end - t0, lag, rel_err, admit_ms, parts


def latency_breakdown(tr, ticket_cam, cams, t0):
    """Where the frames' latency went (from the engine's per-frame traces):
    waiting to be batched (pushed -> taken into a tick), submission (taken
    -> the tick's copies and launch queued), device (queued -> last download
    seen complete); and the same split over the slowest 1% of frames. The
    wait is split further into the client's lateness (arrival -> pushed)
    and the engine's (pushed -> taken into a tick)."""
    import numpy as np
    if tr.size == 0:
        return None
    late = (tr["t_pushed"] - tr["t_arrival"]) * 1e3
    wait = (tr["t_batched"] - tr["t_pushed"]) * 1e3
    sub = (tr["t_submitted"] - tr["t_batched"]) * 1e3
    dev = (tr["t_done"] - tr["t_submitted"]) * 1e3
    tot = (tr["t_done"] - tr["t_arrival"]) * 1e3
    tail = tot >= np.percentile(tot, 99)
    px = np.array([H * W for (H, W, _, _) in cams] + [0])
    res = px[ticket_cam[tr["ticket"]]]  # -1 (unknown) picks the trailing 0
    q = lambda x, p: float(np.percentile(x, p))
    win = np.floor((tr["t_arrival"][tail] - t0) / 0.1)  # 100 ms windows
    return {"client_late_ms": {"p50": q(late, 50), "p99": q(late, 99), "max": float(late.max())},
            "wait_ms": {"p50": q(wait, 50), "p99": q(wait, 99)},
            "submit_ms": {"p50": q(sub, 50), "p99": q(sub, 99)},
            "device_ms": {"p50": q(dev, 50), "p99": q(dev, 99)},
            "tick_frames": {"p50": q(tr["tick_frames"], 50), "p99": q(tr["tick_frames"], 99)},
            "slowest_1pct": {"frames": int(tail.sum()),
                             "client_late_ms": float(late[tail].mean()),
                             "wait_ms": float(wait[tail].mean()),
                             "submit_ms": float(sub[tail].mean()),
                             "device_ms": float(dev[tail].mean()),
                             "tick_frames": float(tr["tick_frames"][tail].mean()),
                             "share_1080p": float((res[tail] == 1920 * 1080).mean()),
                             "windows_100ms": int(np.unique(win).size)}}


def run_serving(args, wl):
    import torch
    import paper_2110_14934_gb300 as G

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    cams, ring = serving_setup(G, torch, wl, rank, dev)
    duration = args.serve_seconds or wl["duration_s"]
    barrier(world, dev)
    transfer = G.SERVE_COPY if args.serve_copy else G.SERVE_ZERO_COPY
    st, lat, wall, lag, rel_err, admit_ms, parts = serve_run(G, torch, cams, ring, wl,
                                            int(wl["budget_gb"] * 1e9), duration, 2021 + rank,
                                            transfer=transfer)
    wall = reduce_max(wall, world, dev)
    pixels = st["pixels"]
    total_px = pixels * world  # weak scaling: every rank serves its own cameras
    value = total_px / wall / 1e6
    st2, lat2, _, _, _, _, _ = serve_run(G, torch, cams, ring, wl, int(wl["tight_budget_gb"] * 1e9),
                                   wl["tight_duration_s"], 77 + rank, transfer=transfer)
    # a genlocked rig: the cameras live at the start deliver their frames
    # together every period, so each period opens with one large burst
    st3, lat3, _, _, _, _, parts3 = serve_run(G, torch, cams, ring, wl, int(wl["budget_gb"] * 1e9),
                                              wl["tight_duration_s"], 2021 + rank, genlocked=True,
                                              transfer=transfer)
    ev3 = serving_schedule(len(cams), wl["tight_duration_s"], wl["fps"],
                           wl["session_frames"] / wl["fps"], wl["live_fraction"], 2021 + rank, True)
    burst_px = sum(cams[c][0] * cams[c][1] for (t, kind, c, _) in ev3 if t == 0.0 and kind == 0)
    mean_bpp = sum(H * W * bytes_per_pixel(M, wl["prec"]) for (H, W, M, _) in cams) / \
        sum(H * W for (H, W, _, _) in cams)
    achieved = pixels * mean_bpp / wall / 1e9
    peak, peak_src = measured_hbm_peak()
    cpu = (oracle_many_cameras(wl, args.cpu_seconds)
           if rank == 0 and world == 1 and args.cpu_seconds > 0 else None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": st["ticks"], "warmup": 0, "ms_per_step": wall / max(st["ticks"], 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"c4: {wl['name']}", "cameras_per_gpu": len(cams),
                       "duration_s": duration, "state": "f16/bf16",
                       "parallelism": f"camera-sharded x{world}"},
            "latency_ms": {"p50": fnum(pct(list(lat), 50)), "p99": fnum(pct(list(lat), 99)),
                           "p999": fnum(pct(list(lat), 99.9)),
                           "max": float(lat[-1]) if lat.size else None,
                           "what": "frame arrival to fused mask in host memory",
                           "breakdown": parts},
            "serving": {"transfer": "copy" if args.serve_copy else "zero-copy",
                        "frames_completed": st["completed"], "frames_dropped": st["dropped"],
                        "sessions_admitted": st["admitted"], "admissions_rejected": st["rejected"],
                        "ticks": st["ticks"], "mean_frames_per_tick": st["completed"] / max(st["ticks"], 1),
                        "driver_lag_ms_p99": fnum(pct(lag, 99)),
                        "driver_lag_ms_max": fnum(lag[-1]) if lag else None,
                        "engine_gap_ms_max": st.get("max_engine_gap_ms"), "release_errors": len(rel_err),
                        "admit_ms_p50": fnum(pct(admit_ms, 50)), "admit_ms_max":
                            fnum(admit_ms[-1]) if admit_ms else None,
                        "budget_gb": wl["budget_gb"]},
            "tight_budget": {"budget_gb": wl["tight_budget_gb"], "duration_s": wl["tight_duration_s"],
                             "sessions_admitted": st2["admitted"], "admissions_rejected": st2["rejected"],
                             "frames_completed": st2["completed"],
                             "latency_ms_p99": fnum(pct(list(lat2), 99))},
            "genlocked": {"duration_s": wl["tight_duration_s"], "frames_completed": st3["completed"],
                          "burst_mpx_at_start": burst_px / 1e6,
                          "latency_ms": {"p50": fnum(pct(list(lat3), 50)),
                                         "p99": fnum(pct(list(lat3), 99)),
                                         "p999": fnum(pct(list(lat3), 99.9)),
                                         "max": float(lat3[-1]) if lat3.size else None},
                          "slowest_1pct": parts3["slowest_1pct"] if parts3 else None},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                         "note": "offered-load bound: the cameras offer far less than the GPU "
                                 "can serve, so this is utilisation, not a kernel limit"},
            "e2e": {"value": value, "unit": UNIT,
                    "h2d_bytes_per_step": int(pixels * 5 / max(st["ticks"], 1)),
                    "d2h_bytes_per_step": int(pixels / 8 / max(st["ticks"], 1)),
                    "path": "page-locked host frames -> gmm_server_push -> masks in host memory"},
            "cpu_baseline": cpu,
            "gpu_launches": st["ticks"],
            "clocks": None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def fnum(x):
    return None if x is None else float(x)


def pct(sorted_vals, p):
    if not sorted_vals:
        return None
    i = min(len(sorted_vals) - 1, max(0, int(round(p / 100.0 * (len(sorted_vals) - 1)))))
    return sorted_vals[i]


def run_e2e(G, torch, g_args, frames, dev, steps, warmup, world, kernel, morph=False):
    """Host frames (pinned) -> C-ABI pipelined path -> host masks. Timed from
    the first submit to the last mask in host memory; per-frame latency from a
    separate unpipelined pass (submit, wait)."""
    H, W, M, prec = g_args
    rgb_d, dep_d = frames
    n_host = min(32, rgb_d.shape[0])
    rgb_h = torch.empty((n_host, H, W, 3), dtype=torch.uint8).pin_memory()
    dep_h = torch.empty((n_host, H, W), dtype=torch.int16).pin_memory()
    rgb_h.copy_(rgb_d[:n_host])
    dep_h.copy_(dep_d[:n_host])
    ring = 8
    masks = torch.empty((ring, H, G.mask_words_per_row(W)), dtype=torch.int32).pin_memory()
    g = G.GMM(H, W, M, precision=prec, device=dev, morph_open=morph, **PARAMS)
    g.set_kernel(*kernel)
    g.set_stream(torch.cuda.current_stream(dev))
    pending = []

    def submit(k):
        pending.append(g.pipe_submit(rgb_h[k % n_host], dep_h[k % n_host], masks[k % ring]))
        if len(pending) >= G.PIPE_DEPTH:
            g.pipe_wait(pending.pop(0), 60000)

    for k in range(warmup):
        submit(k)
    while pending:
        g.pipe_wait(pending.pop(0), 60000)
    barrier(world, dev)
    t = time.perf_counter()
    for k in range(steps):
        submit(warmup + k)
    while pending:
        g.pipe_wait(pending.pop(0), 60000)
    dt = time.perf_counter() - t
    barrier(world, dev)
    dt = reduce_max(dt, world, dev)
    lat = []
    for k in range(min(200, steps)):
        t0 = time.perf_counter()
        tk = g.pipe_submit(rgb_h[k % n_host], dep_h[k % n_host], masks[k % ring])
        g.pipe_wait(tk, 60000)
        lat.append((time.perf_counter() - t0) * 1e3)
    lat.sort()
    g.close()
    # zero-copy: gmm_apply on the same page-locked host frames and masks, the
    # kernel reading the frame and writing the mask over the host link
    zg = G.GMM(H, W, M, precision=prec, device=dev, morph_open=morph, **PARAMS)
    zg.set_kernel(*kernel)
    stream = torch.cuda.current_stream(dev)
    for k in range(warmup):
        zg.apply(rgb_h[k % n_host], dep_h[k % n_host], masks[k % ring], stream=stream)
    torch.cuda.synchronize()
    barrier(world, dev)
    t = time.perf_counter()
    for k in range(steps):
        zg.apply(rgb_h[(warmup + k) % n_host], dep_h[(warmup + k) % n_host],
                 masks[(warmup + k) % ring], stream=stream)
    torch.cuda.synchronize()
    dz = time.perf_counter() - t
    barrier(world, dev)
    dz = reduce_max(dz, world, dev)
    zg.close()
    return {"value": world * steps * H * W / dt / 1e6, "h2d": H * W * 5,
            "d2h": H * G.mask_words_per_row(W) * 4, "lat_p50": pct(lat, 50), "lat_p99": pct(lat, 99),
            "zero_copy": world * steps * H * W / dz / 1e6}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gmm", "reference"], default="gmm")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="0: --steps, at least 200 (pooled workloads: at most 600)")
    ap.add_argument("--kernel", choices=sorted(KERNELS), default="direct")
    ap.add_argument("--variant", type=int, default=0, help="staged tile shape 0-3")
    ap.add_argument("--ctas", type=int, default=0, help="staged CTAs per SM (0: as many as fit)")
    ap.add_argument("--precision", choices=["default", "f32", "f16"], default="default",
                    help="override the workload's state storage precision")
    ap.add_argument("--cams-per-res", type=int, default=0,
                    help="pooled workloads: cameras per resolution (0: the workload's 16)")
    ap.add_argument("--no-graph", action="store_true", help="pooled workloads: no CUDA graph")
    ap.add_argument("--serve-seconds", type=float, default=0.0,
                    help="serving workload: simulated seconds (0: the workload's 20)")
    ap.add_argument("--serve-copy", action="store_true",
                    help="serving workload: the engine's copy mode instead of zero-copy")
    ap.add_argument("--no-autotune", action="store_true", help="pooled workloads: default launch")
    ap.add_argument("--pool-launch", default="",
                    help="pooled workloads: THREADS,CTAS_PER_SM,TILE_PIXELS instead of tuning "
                         "(CTAS_PER_SM -1: the flat form)")
    ap.add_argument("--frame-size", default="",
                    help="single-camera workloads: WIDTHxHEIGHT instead of the workload's")
    ap.add_argument("--frames", type=int, default=0,
                    help="resident frames to cycle through (0: the workload's sequence length)")
    ap.add_argument("--stochastic-weights", action="store_true",
                    help="FP16 state: store the weights with stochastic rounding")
    ap.add_argument("--morph", action="store_true",
                    help="single-camera workloads: each step adds the 3x3 opening of the mask")
    ap.add_argument("--no-extras", action="store_true",
                    help="c2: skip the extra keys (the same cameras with FP16/BF16 state, and a "
                         "short serving run)")
    ap.add_argument("--extra-serve-seconds", type=float, default=10.0,
                    help="c2: simulated seconds of the extra serving runs in the default mode "
                         "(the tight-budget and copy-mode runs take at most 6)")
    ap.add_argument("--cpu-frames", type=int, default=21, help="oracle baseline frames (0 = skip)")
    ap.add_argument("--cpu-rows", type=int, default=0, help="oracle baseline rows per frame (0 = all)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="many-camera workloads: wall seconds of the all-core oracle baseline "
                         "(0 = skip)")
    ap.add_argument("--cpu-all-frames", type=int, default=61,
                    help="frames of the all-core oracle baseline (0 = single thread only)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = dict(WORKLOADS[args.workload])
    multi = wl.get("pool") or wl.get("serve")
    if multi and (args.morph or args.frame_size or args.kernel != "direct"):
        ap.error("--morph, --frame-size and --kernel apply to the single-camera workloads "
                 "(--workload c0 or c1)")
    if args.precision != "default":
        wl["prec"] = 0 if args.precision == "f32" else 1
        wl["name"] += f" [state overridden: {args.precision}]"
    if args.frame_size and not (wl.get("pool") or wl.get("serve")):
        W_, H_ = (int(v) for v in args.frame_size.lower().split("x"))
        wl["H"], wl["W"] = H_, W_
        wl["name"] += f" [frame {W_}x{H_}]"
    if args.cams_per_res and (wl.get("pool") or wl.get("serve")):
        wl["cams_per_res"] = args.cams_per_res
        wl["name"] += f" [{args.cams_per_res} cameras per resolution]"
    if args.impl == "reference":
        return run_reference(args, wl)
    if wl.get("serve"):
        return run_serving(args, wl)
    if wl.get("pool"):
        return run_pool(args, wl)
    return run_gmm(args, wl)


if __name__ == "__main__":
    sys.exit(main())
