"""CUDA path against the FP64 oracle on identical seeded synthetic frames.

Single-step (teacher-forced) parity: before each tick the oracle is set to the
GPU's exact state, so the only differences left are the arithmetic of one
tick (FP32 on the GPU, FP64 in the oracle). Free-running parity: both run
from the first frame on their own and the pixels whose trajectories separate
(FP32 vs FP64 rounding flipping a decision) are counted; each GPU tick is
still held to the strict single-step bar. Full-size parity: the bench workload
(1920x1080, M=5) in the bench's launch configuration, checked on sampled
pixels that the oracle computes one by one.
"""
import numpy as np
import pytest

import oracle as O
import paper_2110_14934_gb300 as G
import synth
from parity import (FREE_RUN_EPS, Pair, mask_mismatch, scene_frames, state_mismatch,
                    state_mismatch_map, to_dev, words)

pytestmark = pytest.mark.gpu


def _assert_tick(pair, g, o, label):
    exempt = o["near"] != 0
    mm = mask_mismatch(g, o, exempt)
    assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, (label, mm)
    st = state_mismatch(pair.gpu.planes(), pair.orc.planes(), pair.orc.fusion_bytes(),
                        exclude=exempt)
    assert sum(st["bad"]) == 0, (label, st)
    assert np.array_equal(pair.gpu.fusion()[~exempt], pair.orc.fusion_bytes()[~exempt]), label
    return int(np.count_nonzero(exempt))


KERNELS = [pytest.param(G.KERNEL_STAGED, id="staged"), pytest.param(G.KERNEL_DIRECT, id="direct")]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("M", [3, 4, 5])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("H,W", [(45, 83), (64, 96)])
def test_single_step_parity(M, kind, H, W, kernel):
    """Oracle state after 44 frames loaded into the GPU, then ten teacher-forced
    ticks across the illumination step at frame 50."""
    rgb, depth, _ = scene_frames(100 + M, H, W, kind, 0, 55)
    pair = Pair(H, W, M, kernel=kernel)
    for t in range(45):
        pair.orc.tick(rgb[t], depth[t])
    pair.load_gpu_from_oracle()
    for t in range(45, 55):
        g, o = pair.tick(rgb[t], depth[t])
        _assert_tick(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()


def test_teacher_forced_sequence_scene1_m5():
    """100 frames of the full scene (ellipses, shadows, periodic region) at
    120x160, M=5, from the first frame, every tick checked."""
    H, W, M = 120, 160, 5
    rgb, depth, _ = scene_frames(7, H, W, 1, 0, 100)
    pair = Pair(H, W, M)
    exempt_total = 0
    for t in range(100):
        g, o = pair.tick(rgb[t], depth[t])
        exempt_total += _assert_tick(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()
    assert exempt_total < 0.001 * H * W * 100


def test_free_running_config0():
    """The 640x480, M=3, 100-frame workload, both sides free-running from the
    first frame. Every tick, a pixel whose GPU masks or state leave the
    oracle's (the two took different branches) must do so on a tick where
    the oracle saw a decision within the free-running margin of its
    threshold; it is then counted as diverged and left out afterwards. Any
    other difference fails."""
    H, W, M = 480, 640, 3
    rgb, depth, _ = scene_frames(1, H, W, 0, 0, 100)
    pair = Pair(H, W, M, eps=FREE_RUN_EPS)           # pair.orc runs free
    tf = O.OracleGMM(H, W, M, 0.01, 2.5, 0.7, 225.0, 0.05)  # teacher-forced, eps 1e-5
    diverged = np.zeros((H, W), bool)
    beyond_margin = []
    gpu_planes = gpu_fusion = None
    for t in range(100):
        gpu_before = gpu_planes
        if t > 0:
            tf.set_state(gpu_planes.astype(np.float64), gpu_fusion)
        free_before = pair.orc.planes() if t > 0 else None
        g, o = pair.tick(rgb[t], depth[t])
        otf = tf.tick(rgb[t], depth[t])
        gpu_planes, gpu_fusion = pair.gpu.planes(), pair.gpu.fusion()
        # strict: this tick of the GPU against the oracle from the same state
        ex = otf["near"] != 0
        mm = mask_mismatch(g, otf, ex)
        assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, (t, mm)
        st = state_mismatch(gpu_planes, tf.planes(), tf.fusion_bytes(), exclude=ex)
        assert sum(st["bad"]) == 0, (t, st)
        # free-running drift: pixels whose trajectories separate
        differs = state_mismatch_map(gpu_planes, pair.orc.planes(), pair.orc.fusion_bytes())
        differs |= gpu_fusion != pair.orc.fusion_bytes()
        for k in ("fused", "fg_rgb", "fg_d"):
            differs |= g[k] != o[k].astype(bool)
        new = differs & ~diverged
        for (y, x) in np.argwhere(new & (o["near"] == 0))[:3]:
            beyond_margin.append({"t": t, "y": int(y), "x": int(x),
                                  "rgb": rgb[t, y, x].tolist(), "depth": int(depth[t, y, x]),
                                  "gpu_before": None if t == 0 else gpu_before[:, :, y, x].tolist(),
                                  "free_before": None if t == 0 else free_before[:, :, y, x].tolist(),
                                  "gpu_after": gpu_planes[:, :, y, x].tolist(),
                                  "free_after": pair.orc.planes()[:, :, y, x].tolist()})
        diverged |= new
    n_beyond = len(beyond_margin)
    print(f"free-running: {int(diverged.sum())} of {H * W} pixels diverged; first divergences "
          f"outside the {FREE_RUN_EPS:g} margin: {beyond_margin[:2]}")
    assert diverged.mean() < 0.01


def test_full_size_sampled_bench_workload():
    """1920x1080, M=5, scene with ellipses/shadows/periodic region, 12 ticks
    through gmm_apply (the bench's launch), checked on 3000 sampled pixels
    plus one full row and one full column, which the oracle runs as a 1 x K
    image (pixels are independent)."""
    H, W, M, T = 1080, 1920, 5, 12
    s = synth.scene(2024, H, W, 1)
    rgb, depth, _ = synth.frames_host(s, 0, T)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, H * W, 3000), 517 * W + np.arange(W),
                                    np.arange(H) * W + 1901]))
    pair = Pair(H, W, M)
    orc = O.OracleGMM(1, idx.size, M, 0.01, 2.5, 0.7, 225.0, 0.05, eps=FREE_RUN_EPS)
    diverged = np.zeros(idx.size, bool)
    for t in range(T):
        g, _ = pair_tick_gpu_only(pair, rgb[t], depth[t])
        o = orc.tick(rgb[t].reshape(-1, 3)[idx][None], depth[t].reshape(-1)[idx][None])
        diverged |= o["near"][0] != 0
        for k in ("fused", "fg_rgb", "fg_d"):
            gm = g[k].reshape(-1)[idx]
            bad = (gm != o[k][0].astype(bool)) & ~diverged
            assert not bad.any(), (t, k, int(bad.sum()))
    planes = pair.gpu.planes().reshape(M, 8, -1)[:, :, idx].astype(np.float64)
    st = state_mismatch(planes[:, :, None, :], orc.planes(), orc.fusion_bytes(),
                        exclude=diverged[None])
    assert sum(st["bad"]) == 0, st


def pair_tick_gpu_only(pair, rgb, depth):
    import torch
    r, d = to_dev(rgb, depth)
    wpr = G.mask_words_per_row(pair.W)
    m = torch.empty((pair.H, wpr), dtype=torch.int32, device="cuda")
    fc, fd = torch.empty_like(m), torch.empty_like(m)
    pair.gpu.apply(r, d, m, fc, fd)
    torch.cuda.synchronize()
    return {"fused": G.unpack_mask(words(m), pair.H, pair.W),
            "fg_rgb": G.unpack_mask(words(fc), pair.H, pair.W),
            "fg_d": G.unpack_mask(words(fd), pair.H, pair.W)}, None


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("H,W,M", [(1, 1, 3), (1, 33, 5), (33, 1, 4), (2, 31, 3), (3, 64, 5),
                                   (7, 95, 4)])
def test_edge_shapes_teacher_forced(H, W, M, kernel):
    rgb, depth, _ = scene_frames(31 + H * W, H, W, 1, 40, 25)
    pair = Pair(H, W, M, kernel=kernel)
    for t in range(25):
        g, o = pair.tick(rgb[t], depth[t])
        _assert_tick(pair, g, o, f"{H}x{W} frame {t}")
        pair.sync_oracle_to_gpu()
    # padding bits beyond W are zero in every mask word
    import torch
    r, d = to_dev(rgb[0], depth[0])
    m = pair.gpu.apply(r, d)
    torch.cuda.synchronize()
    w = words(m).reshape(H, -1)
    if W % 32:
        assert not np.any(w[:, -1] >> np.uint32(W % 32))


def test_all_depth_invalid_and_constant_frames():
    """Degenerate inputs: depth all zero (fusion copies colour), then a
    constant frame sequence (everything background after the first frame)."""
    H, W, M = 20, 40, 3
    rgb, depth, _ = scene_frames(3, H, W, 0, 0, 12)
    depth[:] = 0
    pair = Pair(H, W, M)
    for t in range(12):
        g, o = pair.tick(rgb[t], depth[t])
        _assert_tick(pair, g, o, f"invalid depth frame {t}")
        assert np.array_equal(g["fg_d"], g["fg_rgb"]) and np.array_equal(g["fused"], g["fg_rgb"])
        pair.sync_oracle_to_gpu()
    const_rgb = np.full((H, W, 3), 77, np.uint8)
    const_d = np.full((H, W), 2100, np.uint16)
    pair2 = Pair(H, W, M)
    for t in range(6):
        g, o = pair2.tick(const_rgb, const_d)
        _assert_tick(pair2, g, o, f"constant frame {t}")
        assert not g["fused"].any()


def test_parameters_reach_the_kernel():
    """Non-default parameters (alpha, k, T, variances, floors) change the
    result and still match the oracle."""
    H, W, M = 40, 64, 4
    rgb, depth, _ = scene_frames(9, H, W, 1, 0, 30)
    kw = dict(alpha=0.05, match_k=2.0, bg_T=0.6, init_var=100.0, init_w=0.1, init_var_d=400.0,
              v_min_c=4.0, v_min_d=9.0)
    pair = Pair(H, W, M, **kw)
    for t in range(30):
        g, o = pair.tick(rgb[t], depth[t])
        _assert_tick(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()


def test_reset_reinitialises():
    H, W, M = 16, 48, 3
    rgb, depth, _ = scene_frames(4, H, W, 0, 0, 8)
    pair = Pair(H, W, M)
    for t in range(5):
        pair.tick(rgb[t], depth[t])
    pair.gpu.reset()
    pair.orc = O.OracleGMM(H, W, M, 0.01, 2.5, 0.7, 225.0, 0.05)
    for t in range(5, 8):
        g, o = pair.tick(rgb[t], depth[t])
        exempt = o["near"] != 0
        assert mask_mismatch(g, o, exempt)["fused"] == 0
    # depth planes of pixels whose depth model did not restart are not compared
    st = state_mismatch(pair.gpu.planes(), pair.orc.planes(), pair.orc.fusion_bytes())
    assert sum(st["bad"]) == 0, st


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp16_state_single_step(kernel):
    """FP16 means/variances, BF16 weights, FP32 arithmetic: one tick from a
    state rounded to the storage types, against the oracle from the same
    rounded state; the tolerance is the storage rounding (half an ulp of
    float16 / bfloat16)."""
    H, W, M = 48, 96, 5
    rgb, depth, _ = scene_frames(12, H, W, 1, 0, 50)
    pair = Pair(H, W, M, precision=G.PREC_F16, kernel=kernel)
    for t in range(40):
        pair.orc.tick(rgb[t], depth[t])
    pair.load_gpu_from_oracle()
    floors = np.array([1e-3, 1.0, 1.0, 1.0, 1.0, 1e-3, 1.0, 1.0])
    for t in range(40, 50):
        g, o = pair.tick(rgb[t], depth[t])
        exempt = o["near"] != 0
        mm = mask_mismatch(g, o, exempt)
        assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, mm
        gp = pair.gpu.planes()
        op = pair.orc.planes()
        fus = pair.orc.fusion_bytes()
        for f, tol in ((0, 2 ** -8), (5, 2 ** -8), (1, 2 ** -11), (4, 2 ** -11), (6, 2 ** -11),
                       (7, 2 ** -11)):
            st = state_mismatch(gp, op, fus, exclude=exempt, rtol=tol * 1.01, floors=floors)
            assert st["bad"][f] == 0, (t, f, st)
        pair.sync_oracle_to_gpu()


@pytest.mark.parametrize("prec", [G.PREC_F32, G.PREC_F16])
@pytest.mark.parametrize("H,W,M", [(120, 160, 5), (45, 83, 3), (37, 1000, 4), (1, 1, 5)])
def test_staged_variants_match_direct(H, W, M, prec):
    """Every staged tile shape computes exactly what the direct kernel does
    (same arithmetic, different data movement): masks and state bit-equal
    over ticks that cross the illumination step, with ragged last tiles."""
    import torch
    rgb, depth, _ = scene_frames(900 + M, H, W, 1, 44, 9)
    ref = G.GMM(H, W, M, precision=prec)
    ref.set_kernel(G.KERNEL_DIRECT)
    staged = []
    for variant in range(4):
        g = G.GMM(H, W, M, precision=prec)
        g.set_kernel(G.KERNEL_STAGED, variant)
        staged.append(g)
    for t in range(9):
        r, d = to_dev(rgb[t], depth[t])
        outs = []
        for g in [ref] + staged:
            m = g.new_mask(); fc = g.new_mask(); fd = g.new_mask()
            g.apply(r, d, m, fc, fd)
            outs.append((m, fc, fd))
        torch.cuda.synchronize()
        for v, o in enumerate(outs[1:]):
            for a, b in zip(outs[0], o):
                assert torch.equal(a, b), (t, v)
    for v, g in enumerate(staged):
        assert np.array_equal(g.planes(), ref.planes()), v
        assert np.array_equal(g.fusion(), ref.fusion()), v
        g.sync()  # also reports a pipeline wait that ran out


@pytest.mark.parametrize("prec", [G.PREC_F32, G.PREC_F16])
def test_large_frame_rows(prec):
    """A frame near the size limit (11000 x 11001: 121 M padded pixels,
    ragged rows; 11.6 GB of FP32 state), frames generated on the device. The
    first, a middle and the last row must equal, bit for bit over four ticks,
    the same rows run as 1-row cameras (pixels are independent; this checks
    the large-index arithmetic against the small one), and in FP32 they must
    match the oracle (free-running: pixels near a threshold at the
    free-running margin are left out once flagged)."""
    import torch
    H, W, M, T = 11000, 11001, 3, 4
    s = synth.scene(77, H, W, 1)
    rgb_d, dep_d, _ = synth.frames_device(s, 0, T, with_gt=False)
    g = G.GMM(H, W, M, precision=prec)
    rows = [0, H // 2, H - 1]
    host = [synth.rows_host(s, 0, T, y, 1) for y in rows]
    small = [G.GMM(1, W, M, precision=prec) for _ in rows]
    orcs = [O.OracleGMM(1, W, M, 0.01, 2.5, 0.7, 225.0, 0.05, eps=FREE_RUN_EPS) for _ in rows]
    diverged = [np.zeros((1, W), bool) for _ in rows]
    for t in range(T):
        m = g.apply(rgb_d[t], dep_d[t])
        torch.cuda.synchronize()
        for k, y in enumerate(rows):
            r1, d1 = to_dev(host[k][0][t], host[k][1][t])
            m1 = small[k].apply(r1, d1)
            torch.cuda.synchronize()
            assert np.array_equal(words(m[y:y + 1]), words(m1)), (t, y)
            if prec == G.PREC_F32:
                o = orcs[k].tick(host[k][0][t], host[k][1][t])
                diverged[k] |= o["near"] != 0
                got = G.unpack_mask(words(m1), 1, W)
                bad = (got != o["fused"].astype(bool)) & ~diverged[k]
                assert not bad.any(), (t, y, int(bad.sum()))
    del rgb_d, dep_d
    g.close()
