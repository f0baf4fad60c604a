"""FP64 CPU oracle for per-pixel RGB-D Gaussian-mixture background subtraction
and List-1 fusion ("GPU based GMM segmentation of Kinect data", §III).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package. The CUDA library under
``paper_2110_14934_gb300`` never imports it, and it imports nothing from
there. The arithmetic lives in ``gmm_oracle.c`` (plain C, double precision,
compiled with FP contraction off); this module only builds it, marshals
numpy arrays and keeps the per-image state.

Parity unpinned: agreement with the paper's own (unpublished) GPU numerics and
with any particular third-party Stauffer-Grimson implementation; neither is
available, so the readings listed in ``gmm_oracle.c`` define the method here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Parameter vector layout of gmm_oracle.c.
P_ALPHA, P_K, P_T, P_INIT_VAR, P_INIT_W, P_VMIN, P_EPS, P_FLAGS = range(8)
NEAR_MATCH, NEAR_T, NEAR_KEY = 1, 2, 4
FLAG_RHO_ETA, FLAG_VAR_PER_CHANNEL = 1, 2
DEPTH_SCALE_DEFAULT = 255.0 / 4095.0

# Plane order of the product library's state (gmm.h, GMM_PLANE_*); used only
# to lay the oracle's pixel-major state out the same way for comparison.
PLANE_NAMES = ("w_c", "mu_r", "mu_g", "mu_b", "v_c", "w_d", "mu_d", "v_d")


def build(force: bool = False) -> str:
    """Compile gmm_oracle.c into a shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u16p = ctypes.POINTER(ctypes.c_uint16)


def _declare(L):
    L.oracle_param_count.restype = ctypes.c_int
    L.oracle_stream_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]
    L.oracle_stream_init.restype = None
    L.oracle_rank_order.argtypes = [ctypes.c_int, _dp, _dp, _ip]
    L.oracle_rank_order.restype = None
    L.oracle_background_count.argtypes = [ctypes.c_int, _dp, ctypes.c_double]
    L.oracle_background_count.restype = ctypes.c_int
    L.oracle_stream_step.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _ip, _dp]
    L.oracle_stream_step.restype = ctypes.c_int
    L.oracle_fuse.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip]
    L.oracle_fuse.restype = None
    L.oracle_tick.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int,
                              _dp, _dp, _dp, _dp, _dp, _dp, _i8p, _i8p, _u8p, _u8p, _u16p,
                              _u8p, _u8p, _u8p, _u8p]
    L.oracle_tick.restype = None
    L.oracle_tick_ex.argtypes = L.oracle_tick.argtypes + [_dp, _dp, _i8p]
    L.oracle_tick_ex.restype = None
    L.oracle_morph_open3.argtypes = [ctypes.c_int, ctypes.c_int, _u8p, _u8p, _u8p]
    L.oracle_morph_open3.restype = None
    L.oracle_tick_augmented.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                        ctypes.c_int, _dp, _dp, _dp, _u8p, _u16p, _u8p, _u8p]
    L.oracle_tick_augmented.restype = None
    assert L.oracle_param_count() == 8


def _ptr(a: np.ndarray, ctype):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def f32(x: float) -> float:
    """The float32 value a caller of the float C-ABI actually passes, as a double."""
    return float(np.float32(x))


def stream_params(alpha, k, T, init_var, init_w, v_min=1.0, eps=1e-5, flags=0) -> np.ndarray:
    """Parameter vector; every value is the float32 value the product library sees."""
    return np.array([f32(alpha), f32(k), f32(T), f32(init_var), f32(init_w), f32(v_min), eps,
                     float(flags)], dtype=np.float64)


# ----------------------------------------------------------------- pixel level
def stream_init(M, D, init_var, x):
    w = np.zeros(M); mu = np.zeros(M * D); v = np.zeros(M)
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(D))
    lib().oracle_stream_init(M, D, float(init_var), _ptr(w, ctypes.c_double), _ptr(mu, ctypes.c_double),
                             _ptr(v, ctypes.c_double), _ptr(xa, ctypes.c_double))
    return w, mu.reshape(M, D), v


def stream_step(prm, w, mu, v, x, with_margin=False):
    """One tick of one stream at one pixel. Arrays are updated in place
    (mu has shape (M, D)). Returns (fg, info) with info = (matched stored
    index or -1, B, rank of the matched/replaced component, near bits), and
    with_margin: (fg, info, margin), the smallest relative distance of a
    decision to its threshold."""
    M, D = mu.shape
    assert w.dtype == np.float64 and mu.dtype == np.float64 and v.dtype == np.float64
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(D))
    info = np.zeros(4, dtype=np.int32)
    mrg = np.zeros(1)
    fg = lib().oracle_stream_step(M, D, _ptr(prm, ctypes.c_double), _ptr(w, ctypes.c_double),
                                  _ptr(mu, ctypes.c_double), _ptr(v, ctypes.c_double),
                                  _ptr(xa, ctypes.c_double), _ptr(info, ctypes.c_int),
                                  _ptr(mrg, ctypes.c_double))
    if with_margin:
        return int(fg), tuple(int(i) for i in info), float(mrg[0])
    return int(fg), tuple(int(i) for i in info)


def rank_order(w, v):
    w = np.ascontiguousarray(w, dtype=np.float64); v = np.ascontiguousarray(v, dtype=np.float64)
    perm = np.zeros(len(w), dtype=np.int32)
    lib().oracle_rank_order(len(w), _ptr(w, ctypes.c_double), _ptr(v, ctypes.c_double),
                            _ptr(perm, ctypes.c_int))
    return perm


def background_count(w_ranked, T):
    w = np.ascontiguousarray(w_ranked, dtype=np.float64)
    return int(lib().oracle_background_count(len(w), _ptr(w, ctypes.c_double), float(T)))


def fuse(f_rgb, f_d, F, cpt):
    """List 1 on one pixel; returns the new (F, cpt)."""
    Fi = ctypes.c_int(F); ci = ctypes.c_int(cpt)
    lib().oracle_fuse(int(f_rgb), int(f_d), ctypes.byref(Fi), ctypes.byref(ci))
    return Fi.value, ci.value


def morph_open3(mask: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(mask.astype(np.uint8))
    H, W = m.shape
    tmp = np.zeros_like(m); out = np.zeros_like(m)
    lib().oracle_morph_open3(H, W, _ptr(m, ctypes.c_uint8), _ptr(tmp, ctypes.c_uint8),
                             _ptr(out, ctypes.c_uint8))
    return out


# ----------------------------------------------------------------- image level
class OracleGMM:
    """Whole-image oracle state: colour and depth mixtures plus List-1 state,
    pixel-major, double precision. Parameters are rounded to float32 first,
    because the product library receives them as floats."""

    def __init__(self, H, W, M, alpha, match_k, bg_T, init_var, init_w,
                 init_var_d=None, v_min_c=1.0, v_min_d=1.0, eps=1e-5, flags=0):
        if not (3 <= M <= 5):
            raise ValueError("M must be in [3, 5]")
        self.H, self.W, self.M = int(H), int(W), int(M)
        N = self.H * self.W
        iv_d = init_var if init_var_d is None else init_var_d
        self.prm_c = stream_params(alpha, match_k, bg_T, init_var, init_w, v_min_c, eps, flags)
        self.prm_d = stream_params(alpha, match_k, bg_T, iv_d, init_w, v_min_d, eps, flags)
        self.wc = np.zeros((N, M)); self.muc = np.zeros((N, M, 3)); self.vc = np.zeros((N, M))
        self.wd = np.zeros((N, M)); self.mud = np.zeros((N, M)); self.vd = np.zeros((N, M))
        self.F = np.zeros(N, dtype=np.int8); self.cpt = np.zeros(N, dtype=np.int8)
        self.dinit = np.zeros(N, dtype=np.uint8)
        self.first = True
        self.frames = 0

    def tick(self, rgb: np.ndarray, depth: np.ndarray, report: bool = False) -> dict:
        """One tick. Returns the masks and near bits; with report also the
        per-stream margins ("margin_c", "margin_d": smallest relative
        distance of a decision to its threshold, inf where the stream took no
        step) and the decisions ("dec", int8 [H, W, 6]: colour matched stored
        index or -1, B, rank of the matched or replaced component, then the
        same for depth; -2 where the stream took no step)."""
        H, W = self.H, self.W
        N = H * W
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(H, W, 3)
        depth = np.ascontiguousarray(depth, dtype=np.uint16).reshape(H, W)
        fg_rgb = np.zeros(N, np.uint8); fg_d = np.zeros(N, np.uint8)
        fused = np.zeros(N, np.uint8); near = np.zeros(N, np.uint8)
        d = ctypes.c_double
        args = [H, W, self.M, _ptr(self.prm_c, d), _ptr(self.prm_d, d), int(self.first),
                _ptr(self.wc, d), _ptr(self.muc, d), _ptr(self.vc, d),
                _ptr(self.wd, d), _ptr(self.mud, d), _ptr(self.vd, d),
                _ptr(self.F, ctypes.c_int8), _ptr(self.cpt, ctypes.c_int8),
                _ptr(self.dinit, ctypes.c_uint8), _ptr(rgb, ctypes.c_uint8),
                _ptr(depth, ctypes.c_uint16), _ptr(fg_rgb, ctypes.c_uint8),
                _ptr(fg_d, ctypes.c_uint8), _ptr(fused, ctypes.c_uint8),
                _ptr(near, ctypes.c_uint8)]
        shp = (H, W)
        out = {}
        if report:
            mc = np.zeros(N); md = np.zeros(N); dec = np.zeros(N * 6, np.int8)
            lib().oracle_tick_ex(*args, _ptr(mc, d), _ptr(md, d), _ptr(dec, ctypes.c_int8))
            out = {"margin_c": mc.reshape(shp), "margin_d": md.reshape(shp),
                   "dec": dec.reshape(H, W, 6)}
        else:
            lib().oracle_tick(*args)
        self.first = False
        self.frames += 1
        out.update({"fg_rgb": fg_rgb.reshape(shp), "fg_d": fg_d.reshape(shp),
                    "fused": fused.reshape(shp), "near": near.reshape(shp)})
        return out

    # -- state in the product library's plane layout ---------------------------
    def planes(self) -> np.ndarray:
        """State as [M, 8, H, W] float64, planes in PLANE_NAMES order."""
        H, W, M = self.H, self.W, self.M
        out = np.empty((M, 8, H, W))
        out[:, 0] = self.wc.T.reshape(M, H, W)
        for c in range(3):
            out[:, 1 + c] = self.muc[:, :, c].T.reshape(M, H, W)
        out[:, 4] = self.vc.T.reshape(M, H, W)
        out[:, 5] = self.wd.T.reshape(M, H, W)
        out[:, 6] = self.mud.T.reshape(M, H, W)
        out[:, 7] = self.vd.T.reshape(M, H, W)
        return out

    def fusion_bytes(self) -> np.ndarray:
        """List-1 state as one byte per pixel: bit 0 fused label, bits 1-3
        counter + 3, bit 4 depth model started."""
        b = (self.F.astype(np.int32) | ((self.cpt.astype(np.int32) + 3) << 1)
             | (self.dinit.astype(np.int32) << 4))
        return b.astype(np.uint8).reshape(self.H, self.W)

    def set_state(self, planes: np.ndarray, fusion: np.ndarray) -> None:
        """Load state given in the plane layout (any float dtype) and the
        fusion byte; marks the model as started."""
        H, W, M = self.H, self.W, self.M
        p = np.asarray(planes, dtype=np.float64).reshape(M, 8, H * W)
        self.wc[:] = p[:, 0].T
        for c in range(3):
            self.muc[:, :, c] = p[:, 1 + c].T
        self.vc[:] = p[:, 4].T
        self.wd[:] = p[:, 5].T
        self.mud[:] = p[:, 6].T
        self.vd[:] = p[:, 7].T
        f = np.asarray(fusion, dtype=np.int32).reshape(H * W)
        self.F[:] = (f & 1).astype(np.int8)
        self.cpt[:] = (((f >> 1) & 7) - 3).astype(np.int8)
        self.dinit[:] = ((f >> 4) & 1).astype(np.uint8)
        self.first = False


class OracleAugmented:
    """The augmentation alternative (§III.B): one mixture per pixel over R, G,
    B and depth * depth_scale; one foreground bit per pixel, no fusion."""

    def __init__(self, H, W, M, alpha, match_k, bg_T, init_var, init_w, v_min=1.0, eps=1e-5,
                 flags=0, depth_scale=DEPTH_SCALE_DEFAULT):
        self.H, self.W, self.M = int(H), int(W), int(M)
        N = self.H * self.W
        self.prm = stream_params(alpha, match_k, bg_T, init_var, init_w, v_min, eps, flags)
        self.depth_scale = f32(depth_scale)
        self.w = np.zeros((N, M)); self.mu = np.zeros((N, M, 4)); self.v = np.zeros((N, M))
        self.first = True

    def tick(self, rgb, depth) -> dict:
        H, W = self.H, self.W
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(H, W, 3)
        depth = np.ascontiguousarray(depth, dtype=np.uint16).reshape(H, W)
        fg = np.zeros(H * W, np.uint8); near = np.zeros(H * W, np.uint8)
        d = ctypes.c_double
        lib().oracle_tick_augmented(H, W, self.M, _ptr(self.prm, d), self.depth_scale, int(self.first),
                                    _ptr(self.w, d), _ptr(self.mu, d), _ptr(self.v, d),
                                    _ptr(rgb, ctypes.c_uint8), _ptr(depth, ctypes.c_uint16),
                                    _ptr(fg, ctypes.c_uint8), _ptr(near, ctypes.c_uint8))
        self.first = False
        return {"fg": fg.reshape(H, W), "near": near.reshape(H, W)}

    def planes(self) -> np.ndarray:
        """State in the library's plane layout for this mode: [M, 8, H, W] with
        w in plane 0, the R, G, B means in planes 1-3, v in plane 4 and the
        depth-channel mean in plane 6 (planes 5 and 7 unused, zero)."""
        H, W, M = self.H, self.W, self.M
        out = np.zeros((M, 8, H, W))
        out[:, 0] = self.w.T.reshape(M, H, W)
        for c in range(3):
            out[:, 1 + c] = self.mu[:, :, c].T.reshape(M, H, W)
        out[:, 4] = self.v.T.reshape(M, H, W)
        out[:, 6] = self.mu[:, :, 3].T.reshape(M, H, W)
        return out

    def set_state(self, planes: np.ndarray) -> None:
        H, W, M = self.H, self.W, self.M
        p = np.asarray(planes, dtype=np.float64).reshape(M, 8, H * W)
        self.w[:] = p[:, 0].T
        for c in range(3):
            self.mu[:, :, c] = p[:, 1 + c].T
        self.v[:] = p[:, 4].T
        self.mu[:, :, 3] = p[:, 6].T
        self.first = False


def f1_scores(pred: np.ndarray, truth: np.ndarray) -> dict:
    """Recall, precision and F1 of a binary mask against ground truth
    (Eq. 1-3, §V.A). Empty denominators give 0."""
    p = np.asarray(pred).astype(bool); t = np.asarray(truth).astype(bool)
    tp = int(np.count_nonzero(p & t)); fp = int(np.count_nonzero(p & ~t))
    fn = int(np.count_nonzero(~p & t)); tn = int(p.size - tp - fp - fn)
    R = tp / (tp + fn) if tp + fn else 0.0
    P = tp / (tp + fp) if tp + fp else 0.0
    F1 = 2 * P * R / (P + R) if P + R else 0.0
    return {"tp": tp, "fp": fp, "fn": fn, "tn": tn, "recall": R, "precision": P, "f1": F1}
