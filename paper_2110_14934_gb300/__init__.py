"""GB300 (sm_103a) per-pixel RGB-D Gaussian-mixture background subtraction
with counter-based fusion ("GPU based GMM segmentation of Kinect data").

This module is a thin binding of the C ABI in ``include/gmm.h``: it marshals
torch tensors (device memory, streams) and numpy arrays into plain pointers
and sizes. Every step of the method runs in the CUDA kernels of
``libgmm.so``; there is no CPU fallback, and using the package without the
built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["GMM", "Pool", "GMMError", "fuse_masks", "morph_open3", "mask_words_per_row",
           "state_bytes", "unpack_mask", "pack_mask", "load_library", "PLANES",
           "PREC_F32", "PREC_F16", "make_config", "MODE_FUSION", "MODE_AUGMENTED",
           "FLAG_RHO_ETA", "FLAG_VAR_PER_CHANNEL", "FLAG_STOCHASTIC_WEIGHTS", "Server",
           "SERVE_ZERO_COPY", "SERVE_COPY"]

OK, EINVAL, ENOMEM, ECUDA, EBUDGET, ETIMEOUT = 0, -1, -2, -3, -4, -5
PLANE_W_C, PLANE_MU_R, PLANE_MU_G, PLANE_MU_B, PLANE_V_C, PLANE_W_D, PLANE_MU_D, PLANE_V_D, \
    PLANE_FUSION = range(9)
PLANES = ("w_c", "mu_r", "mu_g", "mu_b", "v_c", "w_d", "mu_d", "v_d")
PREC_F32, PREC_F16 = 0, 1
PIPE_DEPTH = 3
KERNEL_STAGED, KERNEL_DIRECT = 0, 1
MODE_FUSION, MODE_AUGMENTED = 0, 1
FLAG_RHO_ETA, FLAG_VAR_PER_CHANNEL, FLAG_STOCHASTIC_WEIGHTS = 1, 2, 4
SERVE_ZERO_COPY, SERVE_COPY = 0, 1

_ERRNAMES = {EINVAL: "GMM_EINVAL", ENOMEM: "GMM_ENOMEM", ECUDA: "GMM_ECUDA",
             EBUDGET: "GMM_EBUDGET", ETIMEOUT: "GMM_ETIMEOUT"}


class GMMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class GMMConfig(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("M", ctypes.c_int),
                ("alpha", ctypes.c_float), ("match_k", ctypes.c_float), ("bg_T", ctypes.c_float),
                ("init_var", ctypes.c_float), ("init_w", ctypes.c_float),
                ("init_var_d", ctypes.c_float), ("v_min_c", ctypes.c_float),
                ("v_min_d", ctypes.c_float), ("precision", ctypes.c_int),
                ("morph_open", ctypes.c_int), ("mode", ctypes.c_int),
                ("depth_scale", ctypes.c_float), ("flags", ctypes.c_uint)]


class ServerStats(ctypes.Structure):
    _fields_ = [("pushed", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("dropped", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("released", ctypes.c_longlong),
                ("ticks", ctypes.c_longlong), ("pixels", ctypes.c_longlong),
                ("live_cams", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
                ("used_bytes", ctypes.c_size_t), ("max_engine_gap_ms", ctypes.c_double)]


class ServerTrace(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_longlong), ("cam", ctypes.c_int),
                ("tick_frames", ctypes.c_int), ("t_arrival", ctypes.c_double),
                ("t_pushed", ctypes.c_double), ("t_batched", ctypes.c_double), ("t_submitted", ctypes.c_double),
                ("t_done", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def load_library(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libgmm.so (building it first when stale). Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libgmm.so is not built ({_build.LIB}); run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    sig = {
        "gmm_config_init": (None, [ctypes.POINTER(GMMConfig), ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int] + [ctypes.c_float] * 5),
        "gmm_create": (_vp, [ctypes.c_int] * 3 + [ctypes.c_float] * 5),
        "gmm_create_ex": (_vp, [ctypes.POINTER(GMMConfig)]),
        "gmm_set_stream": (ctypes.c_int, [_vp, _vp]),
        "gmm_set_kernel": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "gmm_wait_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double)]),
        "gmm_inject_cuda_error": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_pool_inject_cuda_error": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_apply": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
        "gmm_apply_ex": (ctypes.c_int, [_vp] * 6),
        "gmm_apply_host": (ctypes.c_int, [_vp] * 4),
        "gmm_pipe_submit": (ctypes.c_longlong, [_vp] * 4),
        "gmm_pipe_wait": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_int]),
        "gmm_state_get": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t]),
        "gmm_state_set": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t]),
        "gmm_reset": (ctypes.c_int, [_vp]),
        "gmm_sync": (ctypes.c_int, [_vp]),
        "gmm_destroy": (ctypes.c_int, [_vp]),
        "gmm_last_error": (ctypes.c_char_p, []),
        "gmm_mask_words_per_row": (ctypes.c_int, [ctypes.c_int]),
        "gmm_state_bytes": (ctypes.c_size_t, [ctypes.c_int] * 4),
        "gmm_fuse_masks": (ctypes.c_int, [_vp] * 4 + [ctypes.c_int, ctypes.c_int, _vp]),
        "gmm_morph_open3": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp]),
        "gmm_pack_mask": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp]),
        "gmm_mask_confusion": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
        "gmm_apply_open3_noalloc": (ctypes.c_int, [ctypes.POINTER(GMMConfig), _vp, ctypes.c_int,
                                                   _vp, _vp, _vp, _vp]),
        "gmm_pool_create": (_vp, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
        "gmm_pool_admit": (ctypes.c_int, [_vp, ctypes.POINTER(GMMConfig)]),
        "gmm_pool_release": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_pool_submit": (ctypes.c_int, [_vp, ctypes.c_int] + [_vp] * 5),
        "gmm_pool_submit_many": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
                                 + [ctypes.POINTER(ctypes.c_void_p)] * 3),
        "gmm_pool_tick": (ctypes.c_int, [_vp]),
        "gmm_pool_set_stream": (ctypes.c_int, [_vp, _vp]),
        "gmm_pool_set_launch": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "gmm_pool_autotune": (ctypes.c_int, [_vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3),
        "gmm_pool_autotune_online": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_pool_tuning": (ctypes.c_int, [_vp] + [ctypes.POINTER(ctypes.c_int)] * 3),
        "gmm_pool_use_graph": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_pool_set_prefetch": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_pool_state_get": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                              ctypes.c_size_t]),
        "gmm_pool_state_used": (ctypes.c_size_t, [_vp]),
        "gmm_pool_sync": (ctypes.c_int, [_vp]),
        "gmm_pool_destroy": (ctypes.c_int, [_vp]),
        "gmm_server_create": (_vp, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "gmm_server_admit": (ctypes.c_int, [_vp, ctypes.POINTER(GMMConfig)]),
        "gmm_server_set_transfer": (ctypes.c_int, [_vp, ctypes.c_int]),
        "gmm_server_release": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
        "gmm_server_push": (ctypes.c_longlong, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_double]),
        "gmm_server_done": (ctypes.c_int, [_vp, ctypes.c_longlong]),
        "gmm_server_wait": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_int]),
        "gmm_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)]),
        "gmm_server_latencies": (ctypes.c_size_t, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
        "gmm_server_reserve": (ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.c_size_t]),
        "gmm_pool_reserve": (ctypes.c_int, [_vp, ctypes.c_size_t]),
        "gmm_server_traces": (ctypes.c_size_t, [_vp, ctypes.POINTER(ServerTrace), ctypes.c_size_t]),
        "gmm_server_now": (ctypes.c_double, []),
        "gmm_server_destroy": (ctypes.c_int, [_vp, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _err() -> str:
    return (load_library().gmm_last_error() or b"").decode(errors="replace")


def _check(rc: int) -> int:
    if rc < 0:
        raise GMMError(rc, _err())
    return rc


def mask_words_per_row(W: int) -> int:
    return (int(W) + 31) // 32


def state_bytes(H: int, W: int, M: int, precision: int = PREC_F32) -> int:
    return int(load_library().gmm_state_bytes(H, W, M, precision))


def unpack_mask(words, H: int, W: int) -> np.ndarray:
    """Bit-packed mask (H rows of ceil(W/32) uint32, LSB first) -> bool [H, W]."""
    a = np.asarray(words).astype(np.uint32, copy=False).reshape(H, mask_words_per_row(W))
    bits = np.unpackbits(a.view(np.uint8).reshape(H, -1), axis=1, bitorder="little")
    return bits[:, :W].astype(bool)


def pack_mask(mask: np.ndarray) -> np.ndarray:
    """bool [H, W] -> uint32 [H, ceil(W/32)] in the library's mask layout."""
    m = np.asarray(mask).astype(bool)
    H, W = m.shape
    wpr = mask_words_per_row(W)
    padded = np.zeros((H, wpr * 32), dtype=np.uint8)
    padded[:, :W] = m
    return np.packbits(padded, axis=1, bitorder="little").view(np.uint32).reshape(H, wpr)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr()


def _stream_ptr(stream, device) -> int:
    import torch
    s = torch.cuda.current_stream(device) if stream is None else stream
    return s.cuda_stream


def _check_frame(rgb, depth, H, W):
    if tuple(rgb.shape[-3:]) != (H, W, 3) or rgb.element_size() != 1:
        raise ValueError(f"rgb must be uint8 [{H}, {W}, 3]")
    if tuple(depth.shape[-2:]) != (H, W) or depth.element_size() != 2:
        raise ValueError(f"depth must be a 16-bit [{H}, {W}] tensor")


def make_config(H, W, M=3, alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05,
                init_var_d=None, v_min_c=1.0, v_min_d=1.0, precision=PREC_F32, morph_open=False,
                mode=MODE_FUSION, depth_scale=None, flags=0) -> GMMConfig:
    """gmm_config from gmm_config_init's defaults and the given overrides
    (None keeps the default: init_var_d = init_var, depth_scale = 255/4095)."""
    cfg = GMMConfig()
    load_library().gmm_config_init(ctypes.byref(cfg), H, W, M, alpha, match_k, bg_T, init_var,
                                   init_w)
    if init_var_d is not None:
        cfg.init_var_d = init_var_d
    cfg.v_min_c = v_min_c
    cfg.v_min_d = v_min_d
    cfg.precision = precision
    cfg.morph_open = int(bool(morph_open))
    cfg.mode = mode
    if depth_scale is not None:
        cfg.depth_scale = depth_scale
    cfg.flags = flags
    return cfg


class GMM:
    """One camera's resident model (FP32 or FP16/BF16 state) on a CUDA device."""

    def __init__(self, H, W, M=3, alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0,
                 init_w=0.05, init_var_d=None, v_min_c=1.0, v_min_d=1.0,
                 precision=PREC_F32, morph_open=False, mode=MODE_FUSION, depth_scale=None,
                 flags=0, device=None):
        import torch
        L = load_library()
        self.device = torch.device("cuda" if device is None else device)
        cfg = make_config(H, W, M, alpha, match_k, bg_T, init_var, init_w, init_var_d, v_min_c,
                          v_min_d, precision, morph_open, mode, depth_scale, flags)
        self.cfg = cfg
        self.H, self.W, self.M = int(H), int(W), int(M)
        self.wpr = mask_words_per_row(W)
        with torch.cuda.device(self.device):
            h = L.gmm_create_ex(ctypes.byref(cfg))
        if not h:
            raise GMMError(EINVAL, _err())
        self._h = h

    # -- ticks -----------------------------------------------------------------
    def new_mask(self):
        import torch
        return torch.empty((self.H, self.wpr), dtype=torch.int32, device=self.device)

    def apply(self, rgb, depth, mask=None, fg_rgb=None, fg_d=None, stream=None):
        """One tick on device tensors; returns the mask tensor (int32 words)."""
        _check_frame(rgb, depth, self.H, self.W)
        mask = self.new_mask() if mask is None else mask
        L = load_library()
        _check(L.gmm_set_stream(self._h, _stream_ptr(stream, self.device)))
        _check(L.gmm_apply_ex(self._h, _ptr(rgb), _ptr(depth), _ptr(mask), _ptr(fg_rgb),
                              _ptr(fg_d)))
        return mask

    def apply_host(self, rgb: np.ndarray, depth: np.ndarray, mask: np.ndarray | None = None):
        """One tick from host memory (copies inside); returns the host mask words."""
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        depth = np.ascontiguousarray(depth).view(np.uint16)
        if mask is None:
            mask = np.empty((self.H, self.wpr), dtype=np.uint32)
        _check(load_library().gmm_apply_host(self._h, _ptr(rgb), _ptr(depth), _ptr(mask)))
        return mask

    def pipe_submit(self, rgb, depth, mask) -> int:
        """Queue a host-memory tick (buffers: pinned torch CPU tensors or numpy)."""
        return _check(load_library().gmm_pipe_submit(self._h, _ptr(rgb), _ptr(depth), _ptr(mask)))

    def pipe_wait(self, ticket: int, timeout_ms: int = -1) -> None:
        _check(load_library().gmm_pipe_wait(self._h, ticket, timeout_ms))

    def set_stream(self, stream) -> None:
        _check(load_library().gmm_set_stream(self._h, _stream_ptr(stream, self.device)))

    def set_kernel(self, kind: int = KERNEL_DIRECT, variant: int = 0, ctas_per_sm: int = 0) -> None:
        _check(load_library().gmm_set_kernel(self._h, kind, variant, ctas_per_sm))

    # -- state -----------------------------------------------------------------
    def state_get(self, plane: int, component: int = 0) -> np.ndarray:
        out = np.empty((self.H, self.W), dtype=np.float32)
        _check(load_library().gmm_state_get(self._h, plane, component, _ptr(out), out.size))
        return out

    def state_set(self, plane: int, component: int, values: np.ndarray) -> None:
        v = np.ascontiguousarray(values, dtype=np.float32).reshape(self.H, self.W)
        _check(load_library().gmm_state_set(self._h, plane, component, _ptr(v), v.size))

    def planes(self) -> np.ndarray:
        """Whole state as float32 [M, 8, H, W] (planes in PLANES order)."""
        return np.stack([np.stack([self.state_get(f, i) for f in range(8)]) for i in range(self.M)])

    def fusion(self) -> np.ndarray:
        return self.state_get(PLANE_FUSION).astype(np.uint8)

    def load_state(self, planes: np.ndarray, fusion: np.ndarray) -> None:
        planes = np.asarray(planes, dtype=np.float32).reshape(self.M, 8, self.H, self.W)
        for i in range(self.M):
            for f in range(8):
                self.state_set(f, i, planes[i, f])
        self.state_set(PLANE_FUSION, 0, np.asarray(fusion, dtype=np.float32))

    def reset(self) -> None:
        _check(load_library().gmm_reset(self._h))

    def sync(self) -> None:
        _check(load_library().gmm_sync(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            load_library().gmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """Many cameras with resident models advanced together, one persistent
    launch per tick."""

    def __init__(self, budget_bytes=0, precision=PREC_F32, max_cams=256, device=None):
        import torch
        L = load_library()
        self.device = torch.device("cuda" if device is None else device)
        self.precision = precision
        with torch.cuda.device(self.device):
            p = L.gmm_pool_create(budget_bytes, precision, max_cams)
        if not p:
            raise GMMError(EINVAL, _err())
        self._p = p
        self.cams = {}

    def admit(self, H, W, M=3, alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05,
              init_var_d=None, v_min_c=1.0, v_min_d=1.0, mode=MODE_FUSION, depth_scale=None,
              flags=0) -> int:
        """Returns the camera id; raises GMMError (code EBUDGET) when the state
        budget is exhausted."""
        L = load_library()
        cfg = make_config(H, W, M, alpha, match_k, bg_T, init_var, init_w, init_var_d, v_min_c,
                          v_min_d, self.precision, False, mode, depth_scale, flags)
        cam = _check(L.gmm_pool_admit(self._p, ctypes.byref(cfg)))
        self.cams[cam] = (int(H), int(W), int(M))
        return cam

    def release(self, cam: int) -> None:
        _check(load_library().gmm_pool_release(self._p, cam))
        self.cams.pop(cam, None)

    def submit(self, cam, rgb, depth, mask, fg_rgb=None, fg_d=None) -> None:
        H, W, _ = self.cams[cam]
        _check_frame(rgb, depth, H, W)
        _check(load_library().gmm_pool_submit(self._p, cam, _ptr(rgb), _ptr(depth), _ptr(mask),
                                              _ptr(fg_rgb), _ptr(fg_d)))

    def submit_many(self, cams, rgb_ptrs, depth_ptrs, mask_ptrs) -> None:
        """Submit many cameras at once from raw device pointers (ints)."""
        n = len(cams)
        ca = (ctypes.c_int * n)(*cams)
        ra = (ctypes.c_void_p * n)(*rgb_ptrs)
        da = (ctypes.c_void_p * n)(*depth_ptrs)
        ma = (ctypes.c_void_p * n)(*mask_ptrs)
        _check(load_library().gmm_pool_submit_many(self._p, n, ca, ra, da, ma))

    def tick(self, stream=None) -> None:
        L = load_library()
        _check(L.gmm_pool_set_stream(self._p, _stream_ptr(stream, self.device)))
        _check(L.gmm_pool_tick(self._p))

    def set_stream(self, stream) -> None:
        _check(load_library().gmm_pool_set_stream(self._p, _stream_ptr(stream, self.device)))

    def reserve(self, nbytes: int) -> None:
        """Map nbytes of device memory for camera state up front."""
        _check(load_library().gmm_pool_reserve(self._p, int(nbytes)))

    def set_launch(self, threads=0, ctas_per_sm=0, tile_pixels=0) -> None:
        """Launch shape: block size; persistent CTAs per SM and tile size, or
        ctas_per_sm=-1 for the flat form (one chunk per warp). 0 keeps."""
        _check(load_library().gmm_pool_set_launch(self._p, threads, ctas_per_sm, tile_pixels))

    def autotune(self, iters=3):
        t, c, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load_library().gmm_pool_autotune(self._p, iters, ctypes.byref(t), ctypes.byref(c),
                                                ctypes.byref(p)))
        return {"threads": t.value, "ctas_per_sm": c.value, "tile_pixels": p.value}

    def autotune_online(self, ticks_per_shape=3) -> None:
        """Arm online tuning: the next ticks try the candidate shapes in turn."""
        _check(load_library().gmm_pool_autotune_online(self._p, int(ticks_per_shape)))

    def tuning(self):
        """(still tuning?, current shape dict)."""
        t, c, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = _check(load_library().gmm_pool_tuning(self._p, ctypes.byref(t), ctypes.byref(c),
                                                   ctypes.byref(p)))
        return bool(rc), {"threads": t.value, "ctas_per_sm": c.value, "tile_pixels": p.value}

    def use_graph(self, enable=True) -> None:
        _check(load_library().gmm_pool_use_graph(self._p, int(bool(enable))))

    def set_prefetch(self, enable=True) -> None:
        """FP16/BF16 next-tile L2 prefetch (on by default); turn it off when
        frames are uploaded on a copy stream beside every tick."""
        _check(load_library().gmm_pool_set_prefetch(self._p, int(bool(enable))))

    def state_get(self, cam, plane, component=0) -> np.ndarray:
        H, W, _ = self.cams[cam]
        out = np.empty((H, W), dtype=np.float32)
        _check(load_library().gmm_pool_state_get(self._p, cam, plane, component, _ptr(out),
                                                 out.size))
        return out

    def planes(self, cam) -> np.ndarray:
        H, W, M = self.cams[cam]
        return np.stack([np.stack([self.state_get(cam, f, i) for f in range(8)]) for i in range(M)])

    def fusion(self, cam) -> np.ndarray:
        return self.state_get(cam, PLANE_FUSION).astype(np.uint8)

    def state_used(self) -> int:
        return int(load_library().gmm_pool_state_used(self._p))

    def sync(self) -> None:
        _check(load_library().gmm_pool_sync(self._p))

    def close(self) -> None:
        if getattr(self, "_p", None):
            load_library().gmm_pool_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving engine: cameras join and leave, frames
    arrive in page-locked host memory, one pooled launch per tick.
    transfer: SERVE_ZERO_COPY (the kernel reads frames and writes masks in
    host memory) or SERVE_COPY (uploads and downloads on copy streams)."""

    def __init__(self, budget_bytes=0, precision=PREC_F16, max_cams=256, queue_depth=4,
                 device=None, transfer=None):
        import torch
        L = load_library()
        self.device = torch.device("cuda" if device is None else device)
        self.precision = precision
        with torch.cuda.device(self.device):
            s = L.gmm_server_create(budget_bytes, precision, max_cams, queue_depth)
        if not s:
            raise GMMError(EINVAL, _err())
        self._s = s
        self.cams = {}
        if transfer is not None:
            _check(L.gmm_server_set_transfer(s, transfer))

    @staticmethod
    def now() -> float:
        return float(load_library().gmm_server_now())

    def admit(self, H, W, M=3, alpha=0.01, match_k=2.5, bg_T=0.7, init_var=225.0, init_w=0.05,
              init_var_d=None, v_min_c=1.0, v_min_d=1.0, mode=MODE_FUSION, depth_scale=None,
              flags=0) -> int:
        """Camera id; raises GMMError with code EBUDGET when rejected."""
        L = load_library()
        cfg = make_config(H, W, M, alpha, match_k, bg_T, init_var, init_w, init_var_d, v_min_c,
                          v_min_d, self.precision, False, mode, depth_scale, flags)
        cam = _check(L.gmm_server_admit(self._s, ctypes.byref(cfg)))
        self.cams[cam] = (int(H), int(W), int(M))
        return cam

    def reserve(self, state_bytes: int, staging_bytes: int) -> None:
        """Map device memory for camera state and staging up front."""
        _check(load_library().gmm_server_reserve(self._s, int(state_bytes), int(staging_bytes)))

    def release(self, cam: int, timeout_ms: int = -1) -> None:
        _check(load_library().gmm_server_release(self._s, cam, timeout_ms))
        self.cams.pop(cam, None)

    def push(self, cam, rgb, depth, mask, t_arrival=None) -> int:
        """Queue a frame (page-locked host tensors or arrays); returns a
        ticket. Raises GMMError(EBUDGET) when the camera's queue is full."""
        t = self.now() if t_arrival is None else float(t_arrival)
        return _check(load_library().gmm_server_push(self._s, cam, _ptr(rgb), _ptr(depth),
                                                     _ptr(mask), t))

    def done(self, ticket: int) -> bool:
        return bool(_check(load_library().gmm_server_done(self._s, ticket)))

    def wait(self, ticket: int, timeout_ms: int = -1) -> None:
        _check(load_library().gmm_server_wait(self._s, ticket, timeout_ms))

    def stats(self) -> dict:
        st = ServerStats()
        _check(load_library().gmm_server_stats_get(self._s, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def latencies_ms(self) -> np.ndarray:
        L = load_library()
        n = int(L.gmm_server_latencies(self._s, None, 0))
        out = np.empty(n, dtype=np.float32)
        if n:
            L.gmm_server_latencies(self._s, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n)
        return out

    def traces(self) -> np.ndarray:
        """Per completed frame, in completion order: ticket, camera, frames in
        its tick, and the arrival / pushed / batched / submitted / done times
        (seconds, gmm_server_now clock)."""
        L = load_library()
        n = int(L.gmm_server_traces(self._s, None, 0))
        buf = (ServerTrace * max(n, 1))()
        if n:
            n = int(min(n, L.gmm_server_traces(self._s, buf, n)))
        return np.ctypeslib.as_array(buf)[:n].copy()

    def close(self, timeout_ms: int = 60000) -> None:
        if getattr(self, "_s", None):
            s, self._s = self._s, None
            _check(load_library().gmm_server_destroy(s, timeout_ms))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fuse_masks(fg_rgb, fg_d, fusion, mask_out, H, W, stream=None) -> None:
    """List 1 alone on bit-packed device masks; fusion bytes updated in place."""
    _check(load_library().gmm_fuse_masks(_ptr(fg_rgb), _ptr(fg_d), _ptr(fusion), _ptr(mask_out),
                                         H, W, _stream_ptr(stream, fusion.device)))


def pack_mask_device(byte_mask, H, W, out=None, stream=None):
    """Byte mask tensor [H, W] (device) -> bit-packed int32 words (device)."""
    import torch
    if out is None:
        out = torch.empty((H, mask_words_per_row(W)), dtype=torch.int32, device=byte_mask.device)
    _check(load_library().gmm_pack_mask(_ptr(byte_mask), _ptr(out), H, W,
                                        _stream_ptr(stream, byte_mask.device)))
    return out


def mask_scores(pred, truth, H, W, counts=None, stream=None) -> dict:
    """TP/FP/FN/TN of bit-packed device masks counted on the GPU, with recall,
    precision and F1 (Eq. 1-3, §V.A). Synchronises the stream."""
    import torch
    if counts is None:
        counts = torch.empty(4, dtype=torch.int64, device=pred.device)
    s = torch.cuda.current_stream(pred.device) if stream is None else stream
    _check(load_library().gmm_mask_confusion(_ptr(pred), _ptr(truth), H, W, _ptr(counts),
                                             s.cuda_stream))
    s.synchronize()
    tp, fp, fn, tn = (int(v) for v in counts.cpu().tolist())
    R = tp / (tp + fn) if tp + fn else 0.0
    P = tp / (tp + fp) if tp + fp else 0.0
    F1 = 2 * P * R / (P + R) if P + R else 0.0
    return {"tp": tp, "fp": fp, "fn": fn, "tn": tn, "recall": R, "precision": P, "f1": F1}


def wait_selftest(timeout_ms: int = 200) -> dict:
    """Run the bounded-wait self-test on the current CUDA device: a device
    wait that nothing completes must give up after timeout_ms and report it."""
    t, w = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load_library().gmm_wait_selftest(int(timeout_ms), ctypes.byref(t), ctypes.byref(w)))
    return {"timed_out": bool(t.value), "waited_ms": w.value}


def morph_open3(mask_in, mask_out, H, W, stream=None) -> None:
    """3x3 opening of a bit-packed device mask."""
    _check(load_library().gmm_morph_open3(_ptr(mask_in), _ptr(mask_out), H, W,
                                          _stream_ptr(stream, mask_in.device)))
