"""Storage precision study: the same cameras run for 1000 frames with FP16
means/variances and BF16 weights (FP32 arithmetic), with FP32 state, and in
the FP64 oracle (on sampled pixels, which the oracle runs as a 1 x K image
since pixels are independent). Reports, per parameter, the drift of each
GPU run from the oracle at frames 100, 300 and 1000, the fraction of
sampled pixel-frames whose masks disagree with the oracle, and the fraction
of all pixel-frames where the FP16 and FP32 runs disagree. Set
GMM_DRIFT_REPORT to a path to get the numbers as JSON."""
import json
import os

import numpy as np
import pytest

import oracle as O
import paper_2110_14934_gb300 as G
import synth

pytestmark = pytest.mark.gpu

CAMS = [(240, 320, 3, 41), (480, 640, 5, 42), (720, 1280, 3, 43), (1080, 1920, 5, 44)]
FRAMES = 1000
CHECKPOINTS = (100, 300, 1000)
SAMPLES = 2048
PRM = dict(alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05)


def _drift(gpu_planes, orc_planes, orc_fusion):
    """Relative error |g - o| / max(|o|, floor) per plane over sampled pixels
    (depth planes only where the depth model has started)."""
    floors = [1e-3, 1.0, 1.0, 1.0, 1.0, 1e-3, 1.0, 1.0]
    started = ((orc_fusion >> 4) & 1).astype(bool)
    out = {}
    for f, name in enumerate(G.PLANES):
        o = orc_planes[:, f]
        signed = (gpu_planes[:, f] - o) / np.maximum(np.abs(o), floors[f])
        if f >= 5:
            signed = signed[:, started]
        signed = signed.reshape(-1)
        e = np.abs(signed)
        out[name] = {"median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
                     "max": float(e.max()), "mean_signed": float(signed.mean())}
    return out


# The runs compared: storage precision and flags.
RUNS = {"f16": (G.PREC_F16, 0), "f32": (G.PREC_F32, 0),
        "f16sr": (G.PREC_F16, G.FLAG_STOCHASTIC_WEIGHTS)}


def test_fp16_state_drift_and_mask_disagreement():
    import torch
    dev = torch.device("cuda")
    pools = {n: G.Pool(precision=prec, max_cams=len(CAMS)) for n, (prec, _) in RUNS.items()}
    ids = {n: [pools[n].admit(H, W, M, flags=RUNS[n][1], **PRM) for (H, W, M, _) in CAMS]
           for n in pools}
    scenes = [synth.scene(seed, H, W, 1) for (H, W, M, seed) in CAMS]
    rng = np.random.default_rng(8)
    idx = [np.sort(rng.choice(H * W, SAMPLES, replace=False)) for (H, W, _, _) in CAMS]
    idx_t = [torch.from_numpy(i).to(dev) for i in idx]
    orcs = [O.OracleGMM(1, SAMPLES, M, **PRM) for (H, W, M, _) in CAMS]
    masks = {n: [torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device=dev)
                 for (H, W, _, _) in CAMS] for n in pools}
    dis_orc = {n: 0 for n in pools}
    dis_vs_32 = {"f16": 0, "f16sr": 0}
    px_total = sum(H * W for (H, W, _, _) in CAMS) * FRAMES
    report = {"frames": FRAMES, "cameras": [list(c[:3]) for c in CAMS], "samples_per_camera": SAMPLES,
              "drift": {}, "bytes_per_pixel": {
                  "f16": [32 * M + 7.125 for (_, _, M, _) in CAMS],
                  "f32": [64 * M + 7.125 for (_, _, M, _) in CAMS]}}
    chunk = 50
    for f0 in range(0, FRAMES, chunk):
        batch = [synth.frames_device(s, f0, chunk, device=dev, with_gt=False) for s in scenes]
        for k in range(chunk):
            t = f0 + k
            for n in pools:
                for c, (H, W, _, _) in enumerate(CAMS):
                    r, d, _ = batch[c]
                    pools[n].submit(ids[n][c], r[k], d[k], masks[n][c])
                pools[n].tick()
            for c, (H, W, M, _) in enumerate(CAMS):
                r, d, _ = batch[c]
                rs = r[k].reshape(-1, 3)[idx_t[c]].cpu().numpy()[None]
                ds = d[k].reshape(-1)[idx_t[c]].cpu().numpy().view(np.uint16)[None]
                o = orcs[c].tick(rs, ds)["fused"][0].astype(bool)
                for n in pools:
                    g = G.unpack_mask(masks[n][c].cpu().numpy().view(np.uint32), H, W).reshape(-1)
                    dis_orc[n] += int(np.count_nonzero(g[idx[c]] != o))
                b = masks["f32"][c].cpu().numpy().view(np.uint32)
                for n in dis_vs_32:
                    a = masks[n][c].cpu().numpy().view(np.uint32)
                    dis_vs_32[n] += int(np.unpackbits((a ^ b).view(np.uint8)).sum())
            if t + 1 in CHECKPOINTS:
                entry = {}
                for n in pools:
                    per_cam = []
                    for c, (H, W, M, _) in enumerate(CAMS):
                        pl = pools[n].planes(ids[n][c]).reshape(M, 8, -1)[:, :, idx[c]]
                        per_cam.append(_drift(pl.astype(np.float64), orcs[c].planes()[:, :, 0, :],
                                              orcs[c].fusion_bytes()[0]))
                    entry[n] = per_cam
                report["drift"][str(t + 1)] = entry
    sampled = SAMPLES * len(CAMS) * FRAMES
    report["mask_disagreement_vs_oracle"] = {n: dis_orc[n] / sampled for n in pools}
    report["mask_disagreement_vs_f32"] = {n: v / px_total for n, v in dis_vs_32.items()}
    print(json.dumps(report["mask_disagreement_vs_oracle"]),
          json.dumps(report["mask_disagreement_vs_f32"]))
    # FP32 state follows the oracle closely over 1000 frames; FP16/BF16 state
    # drifts (weights near 1 move in 2^-8 steps against updates of 0.01) but
    # must stay a usable model.
    assert report["mask_disagreement_vs_oracle"]["f32"] < 0.005
    assert report["mask_disagreement_vs_oracle"]["f16"] < 0.10
    assert report["mask_disagreement_vs_oracle"]["f16sr"] < 0.10
    # stochastic rounding removes the weights' rounding bias: averaged over
    # the cameras, the mean signed error of the colour weights at the last
    # checkpoint is smaller than with round-to-nearest
    last = report["drift"][str(CHECKPOINTS[-1])]
    bias = {n: np.mean([abs(last[n][c]["w_c"]["mean_signed"]) for c in range(len(CAMS))])
            for n in ("f16", "f16sr")}
    report["weight_bias_at_last_checkpoint"] = bias
    print("mean |signed colour-weight error|:", bias)
    path = os.environ.get("GMM_DRIFT_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(report, fh, indent=1)
    assert bias["f16sr"] < bias["f16"]
    for p in pools.values():
        p.close()
