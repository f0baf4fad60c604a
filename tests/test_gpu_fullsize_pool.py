"""The many-camera workloads at full size, in the launch configuration the
bench times: 64 cameras (16 each at 320x240, 640x480, 1280x720, 1920x1080,
M from {3, 5} by seed) in one pool, CUDA graph requested, launch shape chosen
by the online tuner during the first ticks. Checked on sampled outputs the
oracle computes one by one: a band of two full rows per camera.

FP32 state, the whole 300-frame sequences: the bands of all cameras with the
same M run again, on the GPU, as one 1 x K camera (pixels are independent, so
the pool's band masks must equal it bit for bit every tick, and its band
state at the end); that camera is held to free-running parity against the
oracle with every difference classified (parity.FreeRun): each tick at the
strict single-step bar against the oracle restarted from the GPU's state, a
branch difference only where the free oracle's margin is within
FREE_RUN_EPS (fewer than 1% of pixels left out), value drift within
FREE_RUN_STATE_RTOL.
FP16/BF16 state, the whole sequences the same way: every tick teacher-forced
(the oracle continues from the GPU's stored band state) and held to the
storage-rounding tolerance."""
import numpy as np
import pytest

import bench
import oracle as O
import paper_2110_14934_gb300 as G
import synth
from parity import FreeRun, state_mismatch, words

pytestmark = pytest.mark.gpu

PRM = dict(alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05)
BAND = 2        # rows per camera checked against the oracle


FRAMES = 300
CHUNK = 30      # frames generated on the device at a time


def _bands_run(prec):
    """The 64-camera pool at full size for FRAMES ticks, with every camera's
    band (BAND rows at mid height) run again as one 1 x K shadow camera per
    M. Yields, per tick and M group, the shadow's host frames, masks and
    state before and after; checks every tick that the pool's bands equal
    the shadow bit for bit, and at the end the band state of one camera per
    resolution and M."""
    import torch
    cams = bench.camera_mix(16, 0)
    pool = G.Pool(precision=prec, max_cams=len(cams))
    ids = [pool.admit(H, W, M, **PRM) for (H, W, M, _) in cams]
    pool.use_graph(True)
    pool.autotune_online(1)
    scenes = [synth.scene(seed, H, W, 1) for (H, W, M, seed) in cams]
    masks = [torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
             for (H, W, _, _) in cams]
    groups = {}
    for i, (H, W, M, _) in enumerate(cams):
        y0 = H // 2
        band = torch.arange(y0 * W, (y0 + BAND) * W, device="cuda")
        groups.setdefault(M, []).append((i, band))
    shadow, before = {}, {}
    for M, members in groups.items():
        K = sum(b.numel() for _, b in members)
        shadow[M] = G.GMM(1, K, M, precision=prec)
        shadow[M].set_kernel(G.KERNEL_DIRECT, 0)
        before[M] = None
    for f0 in range(0, FRAMES, CHUNK):
        batch = [synth.frames_device(s, f0, CHUNK, with_gt=False) for s in scenes]
        for k in range(CHUNK):
            for i, cam in enumerate(ids):
                pool.submit(cam, batch[i][0][k], batch[i][1][k], masks[i])
            pool.tick()
            for M, members in groups.items():
                rs = torch.cat([batch[i][0][k].reshape(-1, 3)[b] for i, b in members]).reshape(1, -1, 3)
                ds = torch.cat([batch[i][1][k].reshape(-1)[b] for i, b in members]).reshape(1, -1)
                g = shadow[M]
                m, fc, fd = g.new_mask(), g.new_mask(), g.new_mask()
                g.apply(rs.contiguous(), ds.contiguous(), m, fc, fd)
                torch.cuda.synchronize()
                K = rs.shape[1]
                gm = {n: G.unpack_mask(words(v), 1, K) for n, v in
                      (("fused", m), ("fg_rgb", fc), ("fg_d", fd))}
                o = 0
                for i, b in members:
                    H, W = cams[i][:2]
                    y0 = H // 2
                    got = G.unpack_mask(words(masks[i][y0:y0 + BAND]), BAND, W).reshape(-1)
                    assert np.array_equal(got, gm["fused"][0, o:o + b.numel()]), (f0 + k, i)
                    o += b.numel()
                after = (g.planes(), g.fusion())
                yield M, rs.cpu().numpy(), ds.cpu().numpy().view(np.uint16), gm, before[M], after
                before[M] = after
        del batch
    assert not pool.tuning()[0]
    for M, members in groups.items():
        planes = before[M][0].reshape(M, 8, -1)
        o, seen = 0, set()
        for i, b in members:
            H, W = cams[i][:2]
            if (H, W) not in seen:
                seen.add((H, W))
                y0 = H // 2
                p = pool.planes(ids[i])[:, :, y0:y0 + BAND, :].reshape(M, 8, -1)
                assert np.array_equal(p, planes[:, :, o:o + b.numel()]), (i, (H, W, M))
            o += b.numel()
    pool.close()


def test_full_size_pool_fp32():
    import json
    fr = {}
    for M, rgb, dep, g, before, after in _bands_run(G.PREC_F32):
        if M not in fr:
            fr[M] = FreeRun(1, rgb.shape[1], M)
        fr[M].step(rgb, dep, g, before, after)
    for M in sorted(fr):
        s = fr[M].check()
        print(f"free-running pool bands M={M}, {FRAMES} frames:", json.dumps(s))


FP16_TOL = {0: 2 ** -8, 5: 2 ** -8, 1: 2 ** -11, 2: 2 ** -11, 3: 2 ** -11, 4: 2 ** -11,
            6: 2 ** -11, 7: 2 ** -11}


def test_full_size_pool_fp16_teacher_forced():
    """FP16 means/variances and BF16 weights: every tick of the 300-frame
    sequences, the oracle restarted from the GPU's stored band state must
    give the same masks (outside decisions within 1e-5 of a threshold) and
    every state value within the storage rounding."""
    floors = np.array([1e-3, 1.0, 1.0, 1.0, 1.0, 1e-3, 1.0, 1.0])
    tf, exempt_total, n_total = {}, 0, 0
    for M, rgb, dep, g, before, after in _bands_run(G.PREC_F16):
        K = rgb.shape[1]
        if M not in tf:
            tf[M] = O.OracleGMM(1, K, M, **PRM)
        o_ = tf[M]
        if before is not None:
            o_.set_state(before[0].astype(np.float64), before[1])
        o = o_.tick(rgb, dep)
        exempt = o["near"] != 0
        exempt_total += int(exempt.sum())
        n_total += K
        for key in ("fused", "fg_rgb", "fg_d"):
            bad = (g[key] != o[key].astype(bool)) & ~exempt
            assert not bad.any(), (M, key, int(bad.sum()))
        for f, tol in FP16_TOL.items():
            st = state_mismatch(after[0], o_.planes(), o_.fusion_bytes(), exclude=exempt,
                                rtol=tol * 1.01, floors=floors)
            assert st["bad"][f] == 0, (M, f, st)
    assert exempt_total < 0.001 * n_total
