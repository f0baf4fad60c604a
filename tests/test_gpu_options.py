"""The readings §III.A leaves open and the augmentation alternative of §III.B,
on the GPU against the FP64 oracle.

- GMM_FLAG_RHO_ETA (rho = alpha * eta, Stauffer-Grimson's second learning
  rate) and GMM_FLAG_VAR_PER_CHANNEL (v is the per-channel variance), alone
  and together, in both tick kernels: teacher-forced single-step parity with
  the same bar as the default reading.
- GMM_MODE_AUGMENTED (one mixture over R, G, B and the scaled depth):
  teacher-forced parity from the first frame, FP32 and FP16 state; the
  staged kernel selection falls back to the direct kernel for it.
- The multi-camera pool with cameras of every variant in one tick: each
  camera's masks and state equal its run alone.
- GMM_FLAG_STOCHASTIC_WEIGHTS (a storage option of FP16/BF16 state): single
  step within one bfloat16 step, unbiased where round-to-nearest stalls,
  and the same bits in a pool as alone.
"""
import numpy as np
import pytest

import oracle as O
import paper_2110_14934_gb300 as G
from parity import (AUG_PLANES, AugPair, Pair, aug_state_mismatch, mask_mismatch,
                    scene_frames, state_mismatch, to_dev, words)

pytestmark = pytest.mark.gpu

PRM = dict(alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05)

KERNELS = [pytest.param(G.KERNEL_STAGED, id="staged"), pytest.param(G.KERNEL_DIRECT, id="direct")]
FLAGS = [pytest.param(G.FLAG_RHO_ETA, id="rho_eta"),
         pytest.param(G.FLAG_VAR_PER_CHANNEL, id="var_per_channel"),
         pytest.param(G.FLAG_RHO_ETA | G.FLAG_VAR_PER_CHANNEL, id="both")]


def _assert_tick(pair, g, o, label):
    exempt = o["near"] != 0
    mm = mask_mismatch(g, o, exempt)
    assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, (label, mm)
    st = state_mismatch(pair.gpu.planes(), pair.orc.planes(), pair.orc.fusion_bytes(),
                        exclude=exempt)
    assert sum(st["bad"]) == 0, (label, st)
    assert np.array_equal(pair.gpu.fusion()[~exempt], pair.orc.fusion_bytes()[~exempt]), label
    return int(np.count_nonzero(exempt))


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("M,H,W", [(3, 45, 83), (5, 64, 96)])
def test_options_single_step_parity(flags, kernel, M, H, W):
    """Oracle state after 44 frames (same reading) loaded into the GPU, then
    ten teacher-forced ticks across the illumination step at frame 50."""
    rgb, depth, _ = scene_frames(300 + M, H, W, 1, 0, 55)
    pair = Pair(H, W, M, kernel=kernel, flags=flags)
    for t in range(45):
        pair.orc.tick(rgb[t], depth[t])
    pair.load_gpu_from_oracle()
    for t in range(45, 55):
        g, o = pair.tick(rgb[t], depth[t])
        _assert_tick(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()


def test_options_from_first_frame_and_effect():
    """Both options from the first frame, 40 teacher-forced ticks; and the
    options do change the trajectory (the flags reach the kernel)."""
    H, W, M = 48, 64, 4
    rgb, depth, _ = scene_frames(31, H, W, 1, 0, 40)
    flags = G.FLAG_RHO_ETA | G.FLAG_VAR_PER_CHANNEL
    pair = Pair(H, W, M, flags=flags)
    plain = G.GMM(H, W, M)
    for t in range(40):
        g, o = pair.tick(rgb[t], depth[t])
        _assert_tick(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()
        r, d = to_dev(rgb[t], depth[t])
        plain.apply(r, d)
    diff = np.abs(pair.gpu.planes() - plain.planes())
    assert diff[:, G.PLANE_V_C].max() > 1.0


def _aug_assert(pair, g, o, label, tols=None):
    exempt = o["near"] != 0
    fg = o["fg"].astype(bool)
    for k in ("fused", "fg_rgb", "fg_d"):
        bad = int(np.count_nonzero((g[k] != fg) & ~exempt))
        assert bad == 0, (label, k, bad)
    gp, op = pair.gpu.planes(), pair.orc.planes()
    if tols is None:
        st = aug_state_mismatch(gp, op, exclude=exempt)
        assert sum(st["bad"].values()) == 0, (label, st)
    else:
        for f in AUG_PLANES:
            st = aug_state_mismatch(gp, op, exclude=exempt, rtol=tols[f])
            assert st["bad"][f] == 0, (label, f, st)
    return int(np.count_nonzero(exempt))


@pytest.mark.parametrize("M", [3, 4, 5])
@pytest.mark.parametrize("flags", [0, G.FLAG_RHO_ETA | G.FLAG_VAR_PER_CHANNEL])
def test_augmented_teacher_forced_from_first_frame(M, flags):
    """60 frames of the full scene (shadows, illumination step, invalid depth
    patches) at 56x72, every tick checked against the oracle continuing from
    the GPU's state. Planes W_D and V_D stay zero."""
    H, W = 56, 72
    rgb, depth, _ = scene_frames(40 + M, H, W, 1, 0, 60)
    pair = AugPair(H, W, M, flags=flags)
    exempt_total = 0
    for t in range(60):
        g, o = pair.tick(rgb[t], depth[t])
        exempt_total += _aug_assert(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()
    gp = pair.gpu.planes()
    assert not gp[:, G.PLANE_W_D].any() and not gp[:, G.PLANE_V_D].any()
    assert exempt_total < 0.001 * H * W * 60
    # the depth channel is live: the scaled depth mean tracks the scene
    assert gp[0, G.PLANE_MU_D].max() > 10.0


def test_augmented_depth_scale_and_invalid_depth():
    """A non-default depth scale reaches the kernel, and a frame with no valid
    depth imputes the best component's depth mean (no depth foreground)."""
    H, W, M = 40, 50, 3
    rgb, depth, _ = scene_frames(77, H, W, 1, 0, 30)
    depth = depth.copy()
    depth[20:] = 0
    pair = AugPair(H, W, M, depth_scale=0.25)
    for t in range(30):
        g, o = pair.tick(rgb[t], depth[t])
        _aug_assert(pair, g, o, f"frame {t}")
        pair.sync_oracle_to_gpu()


def test_augmented_fp16_single_step():
    """FP16 means/variances, BF16 weights: the tolerance is the storage
    rounding, as for the fused model."""
    H, W, M = 48, 96, 5
    rgb, depth, _ = scene_frames(13, H, W, 1, 0, 50)
    pair = AugPair(H, W, M, precision=G.PREC_F16)
    for t in range(40):
        pair.orc.tick(rgb[t], depth[t])
    pair.load_gpu_from_oracle()
    tols = {0: 2 ** -8 * 1.01, 1: 2 ** -11 * 1.01, 2: 2 ** -11 * 1.01, 3: 2 ** -11 * 1.01,
            4: 2 ** -11 * 1.01, 6: 2 ** -11 * 1.01}
    for t in range(40, 50):
        g, o = pair.tick(rgb[t], depth[t])
        _aug_assert(pair, g, o, f"frame {t}", tols=tols)
        pair.sync_oracle_to_gpu()


def test_augmented_ignores_staged_selection():
    import torch
    H, W, M = 64, 96, 4
    rgb, depth, _ = scene_frames(5, H, W, 1, 0, 12)
    a = G.GMM(H, W, M, mode=G.MODE_AUGMENTED)
    b = G.GMM(H, W, M, mode=G.MODE_AUGMENTED)
    b.set_kernel(G.KERNEL_STAGED, 2)
    for t in range(12):
        r, d = to_dev(rgb[t], depth[t])
        ma, mb = a.apply(r, d), b.apply(r, d)
        torch.cuda.synchronize()
        assert torch.equal(ma, mb), t
    assert np.array_equal(a.planes(), b.planes())
    b.sync()


CAMS = [  # (H, W, M, options)
    (45, 83, 3, {}),
    (64, 96, 5, {"flags": G.FLAG_RHO_ETA}),
    (33, 40, 4, {"mode": G.MODE_AUGMENTED}),
    (50, 70, 5, {"flags": G.FLAG_RHO_ETA | G.FLAG_VAR_PER_CHANNEL, "mode": G.MODE_AUGMENTED}),
    (20, 33, 3, {"flags": G.FLAG_VAR_PER_CHANNEL}),
]


@pytest.mark.parametrize("precision", [G.PREC_F32, G.PREC_F16])
def test_pool_mixed_variants_equal_alone(precision):
    """Cameras of every variant share each tick of the pool (the kernel
    instance that dispatches per camera); a default-only tick follows. Every
    camera's masks and state equal its run alone, bit for bit."""
    import torch
    n = 8
    frames = [scene_frames(600 + i, H, W, 1, 0, n) for i, (H, W, M, _) in enumerate(CAMS)]
    alone = {}
    for i, (H, W, M, opt) in enumerate(CAMS):
        g = G.GMM(H, W, M, precision=precision, **opt)
        for t in range(n):
            if t >= n - 2 and i != 0:
                continue
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            alone[(i, t)] = words(g.apply(r, d)).copy()
        torch.cuda.synchronize()
        alone[i] = g.planes()
    pool = G.Pool(precision=precision, max_cams=8)
    ids = [pool.admit(H, W, M, **opt) for (H, W, M, opt) in CAMS]
    pooled = {}
    for t in range(n):
        active = [0] if t >= n - 2 else range(len(CAMS))  # last two ticks: default only
        masks = {}
        for i in active:
            H, W, M, _ = CAMS[i]
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            masks[i] = (torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32,
                                    device="cuda"), r, d)
            pool.submit(ids[i], r, d, masks[i][0])
        pool.tick()
        torch.cuda.synchronize()
        for i in active:
            pooled[(i, t)] = words(masks[i][0]).copy()
    for i in range(len(CAMS)):
        pooled[i] = pool.planes(ids[i])
    pool.close()
    assert alone.keys() == pooled.keys()
    for key in alone:
        assert np.array_equal(alone[key], pooled[key]), key


def test_stochastic_weights_single_step():
    """FP16/BF16 state with stochastically rounded weights: one tick from a
    stored state against the oracle from the same state. Masks as for round
    to nearest (rounding happens after every decision of the tick); weights
    within one bfloat16 step, means and variances within half a float16 step."""
    H, W, M = 48, 96, 5
    rgb, depth, _ = scene_frames(14, H, W, 1, 0, 50)
    pair = Pair(H, W, M, precision=G.PREC_F16)
    pair.gpu = G.GMM(H, W, M, precision=G.PREC_F16, flags=G.FLAG_STOCHASTIC_WEIGHTS, **PRM)
    for t in range(40):
        pair.orc.tick(rgb[t], depth[t])
    pair.load_gpu_from_oracle()
    floors = np.array([1e-3, 1.0, 1.0, 1.0, 1.0, 1e-3, 1.0, 1.0])
    for t in range(40, 50):
        g, o = pair.tick(rgb[t], depth[t])
        exempt = o["near"] != 0
        mm = mask_mismatch(g, o, exempt)
        assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, mm
        gp, op, fus = pair.gpu.planes(), pair.orc.planes(), pair.orc.fusion_bytes()
        for f, tol in ((0, 2 ** -7), (5, 2 ** -7), (1, 2 ** -11), (4, 2 ** -11), (6, 2 ** -11),
                       (7, 2 ** -11)):
            st = state_mismatch(gp, op, fus, exclude=exempt, rtol=tol * 1.01, floors=floors)
            assert st["bad"][f] == 0, (t, f, st)
        pair.sync_oracle_to_gpu()


def test_stochastic_weights_are_unbiased():
    """Identical constant frames at every pixel: the matched component's
    weight follows w_t = 1 - (1 - w_0)(1 - alpha)^t in the oracle. Stored in
    bfloat16 with round-to-nearest it stalls once an update is below half a
    step; with stochastic rounding its mean over the pixels follows the
    oracle, and the pixels that share a tick draw different rounding."""
    import torch
    H, W, M, T = 64, 64, 3, 300
    rgb = np.full((H, W, 3), 120, np.uint8)
    depth = np.full((H, W), 2000, np.uint16)
    r, d = to_dev(rgb, depth)
    orc = O.OracleGMM(1, 1, M, **PRM)
    rn = G.GMM(H, W, M, precision=G.PREC_F16, **PRM)
    sr = G.GMM(H, W, M, precision=G.PREC_F16, flags=G.FLAG_STOCHASTIC_WEIGHTS, **PRM)
    for t in range(T):
        rn.apply(r, d)
        sr.apply(r, d)
        orc.tick(rgb[:1, :1], depth[:1, :1])
    torch.cuda.synchronize()
    w_ref = orc.planes()[0, G.PLANE_W_C].item()
    w_rn = rn.planes()[0, G.PLANE_W_C]
    w_sr = sr.planes()[0, G.PLANE_W_C]
    err_rn = abs(float(w_rn.mean()) - w_ref)
    err_sr = abs(float(w_sr.mean()) - w_ref)
    print("oracle %.5f  nearest %.5f  stochastic %.5f" % (w_ref, w_rn.mean(), w_sr.mean()))
    assert np.unique(w_rn).size == 1              # round to nearest: every pixel alike
    assert np.unique(w_sr).size > 1               # stochastic: pixels draw differently
    assert err_sr < 0.25 * err_rn
    assert err_sr < 2 ** -9


def test_pool_stochastic_weights_equal_alone():
    """Stochastic rounding draws from the model's own tick count, so a camera
    gives the same bits in a pool as alone."""
    import torch
    shapes = [(45, 83, 3), (64, 96, 5)]
    n = 6
    frames = [scene_frames(700 + i, H, W, 1, 0, n) for i, (H, W, M) in enumerate(shapes)]
    alone = []
    for i, (H, W, M) in enumerate(shapes):
        g = G.GMM(H, W, M, precision=G.PREC_F16, flags=G.FLAG_STOCHASTIC_WEIGHTS)
        for t in range(n):
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            g.apply(r, d)
        torch.cuda.synchronize()
        alone.append(g.planes())
    pool = G.Pool(precision=G.PREC_F16, max_cams=4)
    ids = [pool.admit(H, W, M, flags=G.FLAG_STOCHASTIC_WEIGHTS) for (H, W, M) in shapes]
    keep = []
    for t in range(n):
        for i, (H, W, M) in enumerate(shapes):
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            m = torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
            keep.append((r, d, m))
            pool.submit(ids[i], r, d, m)
        pool.tick()
    torch.cuda.synchronize()
    for i in range(len(shapes)):
        assert np.array_equal(pool.planes(ids[i]), alone[i]), i
    pool.close()
