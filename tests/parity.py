"""Side-by-side runs of the CUDA path and the FP64 oracle on the same seeded
synthetic frames, and the comparison rules.

Tolerances (the spec contract for this path):
  - state: |gpu - oracle| <= 1e-4 * max(|oracle|, floor), floors 1e-3 for
    weights, 1 for means and variances (FP32 state);
  - masks: bit-exact, except pixels where the oracle flags a decision within
    1e-5 relative of its threshold at that tick (match distance vs k^2 v,
    rank-prefix weight vs T, two sort keys); those are counted and reported.
"""
from __future__ import annotations

import numpy as np

import oracle as O
import paper_2110_14934_gb300 as G
import synth

RTOL = 1e-4
FLOORS = np.array([1e-3, 1.0, 1.0, 1.0, 1.0, 1e-3, 1.0, 1.0])  # per plane, PLANES order
DEFAULTS = dict(alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05)


def to_dev(rgb, depth):
    import torch
    r = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
    d = torch.from_numpy(np.ascontiguousarray(depth).view(np.int16)).cuda()
    return r, d


def words(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


class Pair:
    """A GPU model and an oracle model with the same parameters."""

    def __init__(self, H, W, M, precision=G.PREC_F32, eps=1e-5, kernel=G.KERNEL_DIRECT,
                 variant=0, flags=0, **kw):
        p = dict(DEFAULTS)
        p.update(kw)
        self.H, self.W, self.M = H, W, M
        self.gpu = G.GMM(H, W, M, precision=precision, flags=flags, **p)
        self.gpu.set_kernel(kernel, variant)
        self.orc = O.OracleGMM(H, W, M, p["alpha"], p["match_k"], p["bg_T"], p["init_var"],
                               p["init_w"], init_var_d=p.get("init_var_d"),
                               v_min_c=p.get("v_min_c", 1.0), v_min_d=p.get("v_min_d", 1.0),
                               eps=eps, flags=flags)

    def tick(self, rgb, depth):
        """One tick on both; returns (gpu dict of bool masks, oracle dict)."""
        import torch
        r, d = to_dev(rgb, depth)
        wpr = G.mask_words_per_row(self.W)
        m = torch.empty((self.H, wpr), dtype=torch.int32, device="cuda")
        fc = torch.empty_like(m)
        fd = torch.empty_like(m)
        self.gpu.apply(r, d, m, fc, fd)
        torch.cuda.synchronize()
        g = {"fused": G.unpack_mask(words(m), self.H, self.W),
             "fg_rgb": G.unpack_mask(words(fc), self.H, self.W),
             "fg_d": G.unpack_mask(words(fd), self.H, self.W)}
        o = self.orc.tick(rgb, depth)
        return g, o

    def sync_oracle_to_gpu(self):
        """Teacher forcing: the oracle continues from the GPU's exact state."""
        self.orc.set_state(self.gpu.planes().astype(np.float64), self.gpu.fusion())

    def load_gpu_from_oracle(self):
        """Load the oracle's state (rounded to the storage type) into the GPU
        and round the oracle's copy the same way, so both start equal."""
        planes = self.orc.planes()
        fusion = self.orc.fusion_bytes()
        self.gpu.load_state(planes.astype(np.float32), fusion)
        self.orc.set_state(self.gpu.planes().astype(np.float64), self.gpu.fusion())


def mask_mismatch(g: dict, o: dict, exempt: np.ndarray) -> dict:
    out = {}
    for k in ("fused", "fg_rgb", "fg_d"):
        diff = g[k] != o[k].astype(bool)
        out[k] = int(np.count_nonzero(diff & ~exempt))
        out[k + "_exempt"] = int(np.count_nonzero(diff & exempt))
    return out


def state_mismatch(gpu_planes, orc_planes, orc_fusion, exclude=None, rtol=RTOL, floors=FLOORS):
    """Counts of state values outside tolerance, per plane; depth planes are
    compared only where the depth model has started."""
    M = gpu_planes.shape[0]
    dstarted = ((orc_fusion >> 4) & 1).astype(bool)
    bad = np.zeros(8, dtype=np.int64)
    worst = np.zeros(8)
    for f in range(8):
        o = orc_planes[:, f]
        gg = gpu_planes[:, f].astype(np.float64)
        err = np.abs(gg - o) / np.maximum(np.abs(o), floors[f])
        valid = np.ones_like(err, dtype=bool)
        if f >= 5:
            valid &= dstarted[None]
        if exclude is not None:
            valid &= ~exclude[None]
        e = np.where(valid, err, 0.0)
        worst[f] = e.max() if e.size else 0.0
        bad[f] = int(np.count_nonzero(e > rtol))
    return {"bad": bad.tolist(), "worst": worst.tolist(), "components": M}


def state_mismatch_map(gpu_planes, orc_planes, orc_fusion, rtol=RTOL, floors=FLOORS):
    """Per-pixel bool: any state value outside tolerance (depth planes only
    where the depth model has started)."""
    dstarted = ((orc_fusion >> 4) & 1).astype(bool)
    out = np.zeros(orc_fusion.shape, dtype=bool)
    for f in range(8):
        o = orc_planes[:, f]
        err = np.abs(gpu_planes[:, f].astype(np.float64) - o) / np.maximum(np.abs(o), floors[f])
        bad = (err > rtol).any(axis=0)
        if f >= 5:
            bad &= dstarted
        out |= bad
    return out


# Free-running margin. FP32 state drifts from the FP64 trajectory: a depth
# mean near 2000 mm carries ~1e-6 relative error (~2e-3 mm) after tens of
# ticks, which is ~3e-4 relative on d^2 for a sample 2.5 sigma (12.5 mm)
# away; the margin takes that with a safety factor of about six. Single-step
# (teacher-forced) comparisons use the contract's 1e-5.
FREE_RUN_EPS = 2e-3


def scene_frames(seed, H, W, kind, f0, nf):
    s = synth.scene(seed, H, W, kind)
    return synth.frames_host(s, f0, nf)


AUG_PLANES = (0, 1, 2, 3, 4, 6)  # planes the augmented mixture keeps


class AugPair:
    """A GPU model in the augmentation mode and the oracle's augmented model."""

    def __init__(self, H, W, M, precision=G.PREC_F32, eps=1e-5, kernel=G.KERNEL_DIRECT,
                 flags=0, depth_scale=None, **kw):
        p = dict(DEFAULTS)
        p.update(kw)
        self.H, self.W, self.M = H, W, M
        self.gpu = G.GMM(H, W, M, precision=precision, mode=G.MODE_AUGMENTED, flags=flags,
                         depth_scale=depth_scale, **p)
        self.gpu.set_kernel(kernel, 0)
        ds = O.DEPTH_SCALE_DEFAULT if depth_scale is None else depth_scale
        self.orc = O.OracleAugmented(H, W, M, p["alpha"], p["match_k"], p["bg_T"],
                                     p["init_var"], p["init_w"], v_min=p.get("v_min_c", 1.0),
                                     eps=eps, flags=flags, depth_scale=ds)

    def tick(self, rgb, depth):
        import torch
        r, d = to_dev(rgb, depth)
        wpr = G.mask_words_per_row(self.W)
        m = torch.empty((self.H, wpr), dtype=torch.int32, device="cuda")
        fc = torch.empty_like(m)
        fd = torch.empty_like(m)
        self.gpu.apply(r, d, m, fc, fd)
        torch.cuda.synchronize()
        g = {k: G.unpack_mask(words(t), self.H, self.W)
             for k, t in (("fused", m), ("fg_rgb", fc), ("fg_d", fd))}
        return g, self.orc.tick(rgb, depth)

    def sync_oracle_to_gpu(self):
        self.orc.set_state(self.gpu.planes().astype(np.float64))

    def load_gpu_from_oracle(self):
        self.gpu.load_state(self.orc.planes().astype(np.float32),
                            np.zeros((self.H, self.W), np.uint8))
        self.sync_oracle_to_gpu()


def aug_state_mismatch(gpu_planes, orc_planes, exclude=None, rtol=RTOL):
    """Counts of out-of-tolerance values per kept plane of the augmented
    state (floors: 1e-3 for the weight, 1 for means and the variance)."""
    bad, worst = {}, {}
    for f in AUG_PLANES:
        o = orc_planes[:, f]
        err = np.abs(gpu_planes[:, f].astype(np.float64) - o) / np.maximum(np.abs(o), FLOORS[f])
        if exclude is not None:
            err = np.where(exclude[None], 0.0, err)
        bad[f] = int(np.count_nonzero(err > rtol))
        worst[f] = float(err.max()) if err.size else 0.0
    return {"bad": bad, "worst": worst}
