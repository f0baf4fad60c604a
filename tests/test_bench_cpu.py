"""Host logic of bench.py that decides what a bench line reports: the
recorded-traffic lookup and its source hash, the serving schedule, the
latency split from the engine's traces, and the pooled launch count. No GPU."""

import numpy as np

import bench
import paper_2110_14934_gb300 as G


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)
    return str(path)


def test_source_hash_ignores_comments_and_whitespace(tmp_path):
    a = _write(tmp_path / "a.cu", "int f(int x) { return x + 1; }\n")
    b = _write(tmp_path / "b.cu", "// a comment\nint f(int x) {\n    /* block */ return x + 1;\n}\n")
    c = _write(tmp_path / "c.cu", "int f(int x) { return x + 2; }\n")
    assert bench.kernel_source_hash([a]) == bench.kernel_source_hash([b])
    assert bench.kernel_source_hash([a]) != bench.kernel_source_hash([c])


def test_recorded_traffic_needs_the_capture_sources_and_scales(tmp_path, monkeypatch):
    csrc = tmp_path / "csrc"
    prof = tmp_path / "profiles"
    csrc.mkdir()
    prof.mkdir()
    for f in ("gmm_device.cuh", "gmm_kernels.cu", "gmm_pool_kernel.cu"):
        _write(csrc / f, f"// {f}\nint k_{f.split('.')[0]};\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "CSRC", str(csrc))
    tick_h = bench.kernel_source_hash([str(csrc / "gmm_device.cuh"), str(csrc / "gmm_kernels.cu")])
    pool_h = bench.kernel_source_hash([str(csrc / "gmm_device.cuh"), str(csrc / "gmm_pool_kernel.cu")])
    _write(prof / "gmm_tick_f32_m5_1920x1080.md",
           f"traffic_bytes_per_launch = 1000\nkernel_source_sha256_16 = {tick_h}\n")
    _write(prof / "gmm_pool_tick_mixed_cameras.md",
           "traffic_bytes_per_launch_f32 = 900\nalgorithmic_bytes_per_launch_f32 = 1000\n"
           "traffic_bytes_per_launch_flat_f32 = 800\nalgorithmic_bytes_per_launch_flat_f32 = 1000\n"
           f"kernel_source_sha256_16 = {pool_h}\n")
    assert bench.recorded_traffic("tick", 0, 12345.0) == 1000.0      # not scaled
    assert bench.recorded_traffic("tick", 1, 1.0) is None             # no FP16 record here
    assert bench.recorded_traffic("pool", 0, 5000.0) == 4500.0        # scaled by the bytes
    assert bench.recorded_traffic("pool_flat", 0, 2000.0) == 1600.0
    _write(csrc / "gmm_kernels.cu", "int changed;\n")                 # the code moved on
    assert bench.recorded_traffic("tick", 0, 1.0) is None
    assert bench.recorded_traffic("pool", 0, 1000.0) == 900.0         # other sources unchanged


def test_serving_schedule_phases_and_genlock():
    wl = bench.WORKLOADS["c4"]
    args = (64, 4.0, wl["fps"], wl["session_frames"] / wl["fps"], wl["live_fraction"], 7)
    free = bench.serving_schedule(*args)
    lock = bench.serving_schedule(*args, genlocked=True)
    assert [e[0] for e in free] == sorted(e[0] for e in free)
    # the same sessions either way: joins and leaves at the same times
    sess = lambda ev: [(t, k, c) for (t, k, c, _) in ev if k != 1]
    assert sess(free) == sess(lock)
    period = 1.0 / wl["fps"]
    first = {}
    for (t, kind, c, k) in free:
        if kind == 1 and k == 0 and c not in first:
            first[c] = t
    live0 = [c for (t, kind, c, _) in free if kind == 0 and t == 0.0]
    assert live0
    # cameras live at the start: free-running phases spread over the period,
    # genlocked ones all start within the jitter of 0
    ph = [first[c] for c in live0 if c in first]
    assert max(ph) - min(ph) > period / 2
    lock_first = {}
    for (t, kind, c, k) in lock:
        if kind == 1 and k == 0 and c not in lock_first:
            lock_first[c] = t
    assert all(lock_first[c] <= 0.002 + 1e-9 for c in live0 if c in lock_first)


def test_latency_breakdown_splits_each_latency():
    n = 400
    buf = (G.ServerTrace * n)()
    tr = np.ctypeslib.as_array(buf)
    rng = np.random.default_rng(3)
    tr["ticket"] = np.arange(n)
    tr["cam"] = rng.integers(0, 2, n)
    tr["tick_frames"] = rng.integers(1, 4, n)
    tr["t_arrival"] = 50.0 + np.sort(rng.random(n))
    tr["t_pushed"] = tr["t_arrival"] + 1e-5
    tr["t_batched"] = tr["t_pushed"] + 2e-5
    tr["t_submitted"] = tr["t_batched"] + 3e-5
    tr["t_done"] = (tr["t_submitted"] + 4e-4 + 1e-5 * rng.random(n)
                    + 1e-3 * (np.arange(n) == 7))                           # one slow frame
    cams = [(240, 320, 3, 0), (1080, 1920, 5, 0)]
    ticket_cam = np.array([1] * n + [-1], dtype=np.int32)
    out = bench.latency_breakdown(tr.copy(), ticket_cam, cams, 50.0)
    assert abs(out["client_late_ms"]["p50"] - 0.01) < 1e-6
    assert abs(out["wait_ms"]["p50"] - 0.02) < 1e-6
    assert abs(out["submit_ms"]["p50"] - 0.03) < 1e-6
    assert abs(out["device_ms"]["p50"] - 0.405) < 2e-3
    slow = out["slowest_1pct"]
    assert slow["frames"] == 4 and slow["share_1080p"] == 1.0 and slow["device_ms"] > 0.4


def test_pool_launch_count():
    cams = bench.camera_mix(16, 0)
    ms = {M for (_, _, M, _) in cams}
    assert bench.pool_launches(cams, None) == 1
    assert bench.pool_launches(cams, {"ctas_per_sm": 8}) == 1
    assert bench.pool_launches(cams, {"ctas_per_sm": -1}) == len(ms)
    many = cams * 3  # 192 cameras: two launches of up to 128
    assert bench.pool_launches(many, None) == 2


def test_committed_captures_match_the_kernel_sources():
    """The ncu summaries under profiles/ that the bench quotes DRAM traffic
    from were taken on the kernel sources as they stand: the single-camera
    ticks (FP32 and FP16/BF16), the pooled tick's small case in both
    precisions, and the full 64-camera launch of the default workloads (c2,
    and its cameras with FP16/BF16 state), whose algorithmic bytes must be
    exactly those of that launch."""
    cams = bench.camera_mix(16, 0)
    full = {p: sum(H * W * bench.bytes_per_pixel(M, p) for (H, W, M, _) in cams) for p in (0, 1)}
    assert full[0] == 15622348800.0 and full[1] == 8003788800.0
    for p in (0, 1):
        assert bench.recorded_traffic("tick", p, 1.0) is not None, p
        assert bench.recorded_traffic("pool", p, 1.0) is not None, p
        t = bench.recorded_traffic("pool_full", p, full[p], exact=True)
        # a capture of the whole launch: DRAM bytes within 1% of the algorithmic bytes
        assert t is not None and abs(t / full[p] - 1.0) < 0.01, (p, t)
