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


# Free-running comparison. The GPU (FP32 state) and the oracle (FP64) each
# run the sequence from the first frame on their own. Their states drift
# apart by rounding (value drift), and a decision whose quantity sits close
# to its threshold can then go the other way (a branch difference), after
# which the pixel's trajectories separate for good. FREE_RUN_EPS bounds the
# relative distance from its threshold (the oracle's margin) at which a
# branch difference is accepted; FREE_RUN_STATE_RTOL bounds the value drift
# of pixels whose decisions all agreed. Both are set from the drift measured
# on the GPU (FP32 against FP64) over the 640x480 100-frame and the 1920x1080
# 300-frame sequences, with a margin.
FREE_RUN_EPS = 5e-4
# per plane (w_c, mu_r, mu_g, mu_b, v_c, w_d, mu_d, v_d): the single-step bar,
# except for the depth variance (see below)
FREE_RUN_STATE_RTOL = np.array([1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-3])
DRIFT_BINS = np.concatenate([[0.0], 10.0 ** np.arange(-12.0, 0.01, 0.05), [np.inf]])


class FreeRun:
    """Free-running parity of a GPU camera against the FP64 oracle, with
    every difference classified.

    Two oracles run beside the GPU: `tf` restarts each tick from the GPU's
    state (teacher forcing: the GPU tick is held to the strict single-step
    bar against it), `fr` runs free from the first frame. At each tick, for
    the pixels still compared:
      - a branch difference: the two oracles' decisions (matched component,
        B, rank) differ, or the GPU's masks or List-1 byte differ from the
        free oracle's, or the teacher-forced oracle saw a decision within
        1e-5 of its threshold (the GPU may have taken the other side) while
        the GPU state left the free oracle's. It is accepted only where the
        free oracle's margin is within FREE_RUN_EPS or the teacher-forced one
        flagged it; the pixel is then left out afterwards (diverged);
      - value drift: all decisions agree; every state value must stay within
        FREE_RUN_STATE_RTOL of the free oracle's (relative, floors as for
        single steps), and its distribution is recorded per plane.
    Anything else fails."""

    def __init__(self, H, W, M, params=None, free_eps=None):
        p = dict(DEFAULTS)
        p.update(params or {})
        self.H, self.W, self.M = H, W, M
        args = (H, W, M, p["alpha"], p["match_k"], p["bg_T"], p["init_var"], p["init_w"])
        self.tf = O.OracleGMM(*args)
        self.fr = O.OracleGMM(*args, eps=FREE_RUN_EPS if free_eps is None else free_eps)
        self.free_eps = FREE_RUN_EPS if free_eps is None else free_eps
        self.diverged = np.zeros((H, W), bool)
        self.events = []        # (tick, free margin, teacher-forced near) per branch difference
        self.unexplained = []   # details of branch differences beyond the margin
        self.value_fail = []    # details of value drift beyond the bar
        self.hist = np.zeros((8, DRIFT_BINS.size - 1), np.int64)
        self.max_drift = np.zeros(8)
        self.max_tick = np.zeros(8, np.int64)
        self.t = 0

    def step(self, rgb, depth, g, gpu_before, gpu_after):
        """One tick. g: the GPU's masks (bool [H, W] each: fused, fg_rgb,
        fg_d); gpu_before / gpu_after: (planes [M, 8, H, W], List-1 bytes)
        of the GPU before and after the tick (before is None on the first
        tick)."""
        if gpu_before is not None:
            self.tf.set_state(gpu_before[0].astype(np.float64), gpu_before[1])
        otf = self.tf.tick(rgb, depth, report=True)
        ofr = self.fr.tick(rgb, depth, report=True)
        gp, gf = gpu_after
        # strict: this GPU tick against the oracle from the same state
        ex = otf["near"] != 0
        mm = mask_mismatch(g, otf, ex)
        assert mm["fused"] == 0 and mm["fg_rgb"] == 0 and mm["fg_d"] == 0, (self.t, mm)
        st = state_mismatch(gp, self.tf.planes(), self.tf.fusion_bytes(), exclude=ex)
        assert sum(st["bad"]) == 0, (self.t, st)
        assert np.array_equal(gf[~ex], self.tf.fusion_bytes()[~ex]), self.t
        # free-running
        fp, ff = self.fr.planes(), self.fr.fusion_bytes()
        err = rel_err_planes(gp, fp, ff)                    # [8, H, W]
        beyond = (err > FREE_RUN_STATE_RTOL[:, None, None]).any(axis=0)
        branch = (otf["dec"] != ofr["dec"]).any(axis=-1) | (gf != ff)
        for k in ("fused", "fg_rgb", "fg_d"):
            branch |= g[k] != ofr[k].astype(bool)
        branch |= ex & beyond
        live = ~self.diverged
        new = branch & live
        margin = np.minimum(ofr["margin_c"], ofr["margin_d"])
        ok = (margin <= self.free_eps) | ex
        for (y, x) in np.argwhere(new):
            self.events.append((self.t, float(margin[y, x]), bool(ex[y, x])))
        for (y, x) in np.argwhere(new & ~ok)[:5]:
            self.unexplained.append({"t": self.t, "y": int(y), "x": int(x),
                                     "margin": float(margin[y, x]),
                                     "dec_tf": otf["dec"][y, x].tolist(),
                                     "dec_fr": ofr["dec"][y, x].tolist()})
        self.diverged |= new
        live = ~self.diverged
        for (y, x) in np.argwhere(live & beyond)[:5]:
            self.value_fail.append({"t": self.t, "y": int(y), "x": int(x),
                                    "err": err[:, y, x].tolist()})
        for f in range(8):
            e = err[f][live]
            self.hist[f] += np.histogram(e, DRIFT_BINS)[0]
            m = float(e.max()) if e.size else 0.0
            if m > self.max_drift[f]:
                self.max_drift[f], self.max_tick[f] = m, self.t
        self.t += 1

    def summary(self):
        """Value drift per plane (max and 99.9th percentile of the relative
        error over the compared pixel-ticks), branch differences and the free
        oracle's margins at them, and the fraction of pixels left out."""
        q = []
        for f in range(8):
            c = np.cumsum(self.hist[f])
            n = c[-1]
            i = int(np.searchsorted(c, 0.999 * n)) if n else 0
            q.append(float(DRIFT_BINS[min(i + 1, DRIFT_BINS.size - 1)]))
        m = sorted(e[1] for e in self.events if not e[2])
        return {"ticks": self.t, "diverged_fraction": float(self.diverged.mean()),
                "branch_differences": len(self.events),
                "explained_by_teacher_forced_near": sum(1 for e in self.events if e[2]),
                "free_margin_max": m[-1] if m else None,
                "free_margin_median": m[len(m) // 2] if m else None,
                "value_drift_max": dict(zip(PLANE_NAMES, self.max_drift.tolist())),
                "value_drift_max_tick": dict(zip(PLANE_NAMES, self.max_tick.tolist())),
                "value_drift_p999_upper": dict(zip(PLANE_NAMES, q)),
                "unexplained": self.unexplained[:3], "value_fail": self.value_fail[:3]}

    def check(self, max_diverged=0.01):
        s = self.summary()
        assert not self.unexplained, s
        assert not self.value_fail, s
        assert s["diverged_fraction"] < max_diverged, s
        return s


PLANE_NAMES = ("w_c", "mu_r", "mu_g", "mu_b", "v_c", "w_d", "mu_d", "v_d")


def rel_err_planes(gpu_planes, orc_planes, orc_fusion, floors=FLOORS):
    """Relative error |g - o| / max(|o|, floor), reduced over components:
    [8, H, W]; depth planes are 0 where the depth model has not started."""
    dstarted = ((orc_fusion >> 4) & 1).astype(bool)
    out = np.empty((8,) + orc_fusion.shape)
    for f in range(8):
        o = orc_planes[:, f]
        e = np.abs(gpu_planes[:, f].astype(np.float64) - o) / np.maximum(np.abs(o), floors[f])
        e = e.max(axis=0)
        if f >= 5:
            e = np.where(dstarted, e, 0.0)
        out[f] = e
    return out


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
