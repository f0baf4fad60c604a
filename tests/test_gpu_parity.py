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
import json

import numpy as np
import pytest

import oracle as O
import paper_2110_14934_gb300 as G
import synth
from parity import (FREE_RUN_EPS, FreeRun, Pair, mask_mismatch, scene_frames, state_mismatch,
                    to_dev, words)

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
    first frame, every difference classified (parity.FreeRun): each GPU tick
    is held to the strict single-step bar against the oracle restarted from
    the GPU's state; a pixel whose decisions leave the free-running oracle's
    must do so where that oracle's margin is within FREE_RUN_EPS (it is then
    left out afterwards, and fewer than 1% of pixels may be); every other
    pixel's state must stay within FREE_RUN_STATE_RTOL of the oracle's."""
    H, W, M = 480, 640, 3
    rgb, depth, _ = scene_frames(1, H, W, 0, 0, 100)
    gpu = G.GMM(H, W, M)
    gpu.set_kernel(G.KERNEL_DIRECT, 0)
    fr = FreeRun(H, W, M)
    before = None
    for t in range(100):
        g = _gpu_tick(gpu, rgb[t], depth[t])
        after = (gpu.planes(), gpu.fusion())
        fr.step(rgb[t], depth[t], g, before, after)
        before = after
    s = fr.check()
    print("free-running 640x480 M=3, 100 frames:", json.dumps(s))


def _gpu_tick(gpu, rgb, depth):
    """One tick of a GPU camera from host frames; its three masks as bool."""
    import torch
    r, d = to_dev(rgb, depth)
    m, fc, fd = gpu.new_mask(), gpu.new_mask(), gpu.new_mask()
    gpu.apply(r, d, m, fc, fd)
    torch.cuda.synchronize()
    return {k: G.unpack_mask(words(v), gpu.H, gpu.W) for k, v in
            (("fused", m), ("fg_rgb", fc), ("fg_d", fd))}


def _sample_index(H, W, seed, n):
    """n random pixels plus one full row and one full column (flat indices)."""
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, H * W, n), 517 * W + np.arange(W),
                                     np.arange(H) * W + 1901]))


class _Shadow:
    """Sampled pixels of a full-size camera run again, on the GPU, as a
    1 x K camera (pixels are independent, so the two must agree bit for
    bit); the shadow's state is small enough to read back every tick."""

    def __init__(self, K, M, precision):
        self.g = G.GMM(1, K, M, precision=precision)
        self.g.set_kernel(G.KERNEL_DIRECT, 0)

    def tick(self, rgb_t, dep_t, idx_t):
        K = idx_t.numel()
        rs = rgb_t.reshape(-1, 3)[idx_t].reshape(1, K, 3).contiguous()
        ds = dep_t.reshape(-1)[idx_t].reshape(1, K).contiguous()
        m, fc, fd = self.g.new_mask(), self.g.new_mask(), self.g.new_mask()
        self.g.apply(rs, ds, m, fc, fd)
        return rs, ds, (m, fc, fd)


def _full_size_sampled(prec, T):
    """1920x1080, M=5, kind-1 scene (ellipses, shadows, periodic region),
    T ticks through gmm_apply in the bench's launch configuration, with a
    1 x K shadow camera on the sampled pixels. Yields per tick the shadow's
    host frames, its masks and its state before and after."""
    import torch
    H, W, M = 1080, 1920, 5
    s = synth.scene(2024, H, W, 1)
    rgb_d, dep_d, _ = synth.frames_device(s, 0, T, with_gt=False)
    idx = _sample_index(H, W, 5, 4000)
    idx_t = torch.from_numpy(idx).cuda()
    full = G.GMM(H, W, M, precision=prec)
    full.set_kernel(G.KERNEL_DIRECT, 0)
    sh = _Shadow(idx.size, M, prec)
    m = full.new_mask()
    before = None
    for t in range(T):
        full.apply(rgb_d[t], dep_d[t], m)
        rs, ds, sm = sh.tick(rgb_d[t], dep_d[t], idx_t)
        torch.cuda.synchronize()
        g = {k: G.unpack_mask(words(v), 1, idx.size) for k, v in zip(("fused", "fg_rgb", "fg_d"), sm)}
        # the bench's launch and the shadow agree bit for bit on the samples
        assert np.array_equal(G.unpack_mask(words(m), H, W).reshape(-1)[idx], g["fused"][0]), t
        after = (sh.g.planes(), sh.g.fusion())
        yield t, rs.cpu().numpy(), ds.cpu().numpy().view(np.uint16), g, before, after
        before = after
    fp = full.planes().reshape(M, 8, -1)[:, :, idx]
    assert np.array_equal(fp, sh.g.planes().reshape(M, 8, -1))
    assert np.array_equal(full.fusion().reshape(-1)[idx], sh.g.fusion().reshape(-1))
    del rgb_d, dep_d
    full.close()


def test_full_size_sampled_bench_workload():
    """The bench workload (1920x1080, M=5, FP32 state) for its whole
    300-frame sequence through gmm_apply in the bench's launch, checked on
    4000 random pixels plus a full row and a full column: the launch equals
    a 1 x K camera on those pixels bit for bit (masks every tick, state at
    the end), and that camera is held to free-running parity with every
    difference classified (parity.FreeRun)."""
    fr = None
    for t, rgb, dep, g, before, after in _full_size_sampled(G.PREC_F32, 300):
        if fr is None:
            fr = FreeRun(1, rgb.shape[1], 5)
        fr.step(rgb, dep, g, before, after)
    s = fr.check()
    print("free-running 1920x1080 M=5 sampled, 300 frames:", json.dumps(s))


FP16_TOL = {0: 2 ** -8, 5: 2 ** -8, 1: 2 ** -11, 2: 2 ** -11, 3: 2 ** -11, 4: 2 ** -11,
            6: 2 ** -11, 7: 2 ** -11}


def test_full_size_sampled_fp16_teacher_forced():
    """The bench workload with FP16 means/variances and BF16 weights, the
    whole 300-frame sequence through gmm_apply in the bench's launch, on
    sampled pixels (bit-equal to a 1 x K camera): every tick, the oracle
    restarted from the GPU's stored state must give the same masks (outside
    decisions within 1e-5 of a threshold) and every state value within the
    storage rounding (half an ulp of bfloat16 for weights, of float16 for
    means and variances)."""
    floors = np.array([1e-3, 1.0, 1.0, 1.0, 1.0, 1e-3, 1.0, 1.0])
    tf = None
    exempt_total = 0
    for t, rgb, dep, g, before, after in _full_size_sampled(G.PREC_F16, 300):
        K = rgb.shape[1]
        if tf is None:
            tf = O.OracleGMM(1, K, 5, 0.01, 2.5, 0.7, 225.0, 0.05)
        if before is not None:
            tf.set_state(before[0].astype(np.float64), before[1])
        o = tf.tick(rgb, dep, report=True)
        exempt = o["near"] != 0
        exempt_total += int(exempt.sum())
        mm = mask_mismatch(g, o, exempt)
        assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, (t, mm)
        for f, tol in FP16_TOL.items():
            st = state_mismatch(after[0], tf.planes(), tf.fusion_bytes(), exclude=exempt,
                                rtol=tol * 1.01, floors=floors)
            if st["bad"][f]:
                err = np.abs(after[0][:, f, 0].astype(np.float64) - tf.planes()[:, f, 0]) / \
                    np.maximum(np.abs(tf.planes()[:, f, 0]), floors[f])
                k = int(np.argmax(err.max(axis=0) * ~exempt[0]))
                detail = {"pixel": k, "rgb": rgb[0, k].tolist(), "depth": int(dep[0, k]),
                          "before": before[0][:, :, 0, k].tolist() if before else None,
                          "gpu": after[0][:, :, 0, k].tolist(),
                          "oracle": tf.planes()[:, :, 0, k].tolist(),
                          "dec": o["dec"][0, k].tolist(), "margin": float(o["margin_c"][0, k])}
                raise AssertionError((t, f, st, detail))
    assert exempt_total < 0.001 * K * 300


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
        for f, tol in FP16_TOL.items():
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
