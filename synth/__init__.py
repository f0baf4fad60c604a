"""Seeded synthetic RGB-D scenes (integer-exact; identical on host and device).

The generator stands in for the paper's Kinect captures, which are not
available. It is the one module shared by the oracle side and the CUDA side of
the tests: it draws frames and ground-truth masks and holds none of the
background-subtraction arithmetic. ``synth_core.h`` defines every pixel;
``synth.c`` builds scenes and host frames; ``synth_dev.cu`` produces the same
frames in device memory.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_OUT = os.path.join(_HERE, "_build")
_HOST_LIB = os.path.join(_OUT, "libsynth.so")
_DEV_LIB = os.path.join(_OUT, "libsynth_dev.so")
_lock = threading.Lock()
_host = None
_dev = None

SYNTH_MAX_ELLIPSES = 8
SYNTH_LUT = 1024


class Ellipse(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("cx0", "cy0", "vx", "vy", "a", "b", "sx", "sy", "r", "g", "bl", "depth")]


class Scene(ctypes.Structure):
    """Mirror of ``synth_scene``; fields may be edited before generating."""
    _fields_ = [
        ("seed", ctypes.c_uint64), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
        ("bg_base", ctypes.c_int32 * 3), ("bg_gx", ctypes.c_int32 * 3), ("bg_gy", ctypes.c_int32 * 3),
        ("d_base", ctypes.c_int32), ("d_gx", ctypes.c_int32), ("d_gy", ctypes.c_int32),
        ("rect_x0", ctypes.c_int32), ("rect_y0", ctypes.c_int32), ("rect_w", ctypes.c_int32),
        ("rect_h", ctypes.c_int32), ("rect_speed", ctypes.c_int32),
        ("rect_rgb", ctypes.c_int32 * 3), ("rect_depth", ctypes.c_int32),
        ("n_ellipses", ctypes.c_int32), ("ell", Ellipse * SYNTH_MAX_ELLIPSES),
        ("periodic", ctypes.c_int32), ("per_x0", ctypes.c_int32), ("per_y0", ctypes.c_int32),
        ("per_w", ctypes.c_int32), ("per_h", ctypes.c_int32), ("per_num", ctypes.c_int32),
        ("per_den", ctypes.c_int32), ("lut", ctypes.c_int8 * SYNTH_LUT),
        ("illum_frame", ctypes.c_int32), ("illum_delta", ctypes.c_int32),
        ("noise_c_k", ctypes.c_int64), ("noise_d_k", ctypes.c_int64),
        ("invalid_per_10000", ctypes.c_int32),
    ]


def _compile(cmd, out):
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(cmd + ["-o", tmp], check=True, cwd=_HERE)
    os.replace(tmp, out)


def _stale(out, srcs):
    return (not os.path.exists(out)) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in srcs)


def host_build_cmd():
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
            os.path.join(_HERE, "synth.c"), "-lm"]


def dev_build_cmd(arch="103a"):
    return ["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC", "-std=c++17",
            f"-gencode=arch=compute_{arch},code=sm_{arch}", "-lineinfo",
            os.path.join(_HERE, "synth_dev.cu")]


def build(device: bool = True, force: bool = False) -> None:
    os.makedirs(_OUT, exist_ok=True)
    hdr = os.path.join(_HERE, "synth_core.h")
    if force or _stale(_HOST_LIB, [os.path.join(_HERE, "synth.c"), hdr]):
        _compile(host_build_cmd(), _HOST_LIB)
    if device and (force or _stale(_DEV_LIB, [os.path.join(_HERE, "synth_dev.cu"), hdr])):
        _compile(dev_build_cmd(), _DEV_LIB)


def host_lib():
    global _host
    with _lock:
        if _host is None:
            build(device=False)
            L = ctypes.CDLL(_HOST_LIB)
            L.synth_scene_size.restype = ctypes.c_int
            L.synth_scene_init.argtypes = [ctypes.POINTER(Scene), ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int]
            L.synth_scene_init.restype = ctypes.c_int
            L.synth_frames_host.argtypes = [ctypes.POINTER(Scene), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.synth_frames_host.restype = ctypes.c_int
            L.synth_rows_host.argtypes = [ctypes.POINTER(Scene), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
            L.synth_rows_host.restype = ctypes.c_int
            if L.synth_scene_size() != ctypes.sizeof(Scene):
                raise RuntimeError("synth_scene layout mismatch")
            _host = L
        return _host


def dev_lib():
    global _dev
    with _lock:
        if _dev is None:
            build(device=True)
            L = ctypes.CDLL(_DEV_LIB)
            L.synth_frames_device.argtypes = [ctypes.POINTER(Scene), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]
            L.synth_frames_device.restype = ctypes.c_int
            _dev = L
        return _dev


def scene(seed: int, H: int, W: int, kind: int = 0) -> Scene:
    """kind 0: gradient + moving rectangle + illumination step; kind 1: adds
    6 ellipses with shadows and a quasi-periodic region."""
    s = Scene()
    if host_lib().synth_scene_init(ctypes.byref(s), seed, H, W, kind) != 0:
        raise ValueError("bad scene arguments")
    return s


def frames_host(s: Scene, f0: int, nf: int):
    """Returns (rgb [nf,H,W,3] u8, depth [nf,H,W] u16, gt [nf,H,W] u8)."""
    H, W = s.H, s.W
    rgb = np.empty((nf, H, W, 3), np.uint8)
    depth = np.empty((nf, H, W), np.uint16)
    gt = np.empty((nf, H, W), np.uint8)
    rc = host_lib().synth_frames_host(ctypes.byref(s), f0, nf, rgb.ctypes.data,
                                      depth.ctypes.data, gt.ctypes.data)
    if rc != 0:
        raise RuntimeError("synth_frames_host failed")
    return rgb, depth, gt


def rows_host(s: Scene, f0: int, nf: int, y0: int, rows: int):
    """Rows y0..y0+rows-1 of frames f0..f0+nf-1 (same bytes as frames_host)."""
    W = s.W
    rgb = np.empty((nf, rows, W, 3), np.uint8)
    depth = np.empty((nf, rows, W), np.uint16)
    gt = np.empty((nf, rows, W), np.uint8)
    rc = host_lib().synth_rows_host(ctypes.byref(s), f0, nf, y0, rows, rgb.ctypes.data,
                                    depth.ctypes.data, gt.ctypes.data)
    if rc != 0:
        raise ValueError("bad row range")
    return rgb, depth, gt


def frames_device(s: Scene, f0: int, nf: int, device=None, stream=None, with_gt=True):
    """Same frames as frames_host, generated in device memory (torch tensors)."""
    import torch
    dev = torch.device("cuda" if device is None else device)
    H, W = s.H, s.W
    rgb = torch.empty((nf, H, W, 3), dtype=torch.uint8, device=dev)
    depth = torch.empty((nf, H, W), dtype=torch.int16, device=dev)  # bit pattern of uint16
    gt = torch.empty((nf, H, W), dtype=torch.uint8, device=dev) if with_gt else None
    st = torch.cuda.current_stream(dev) if stream is None else stream
    rc = dev_lib().synth_frames_device(ctypes.byref(s), f0, nf, rgb.data_ptr(), depth.data_ptr(),
                                       gt.data_ptr() if gt is not None else None, st.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_frames_device failed: cudaError {rc}")
    return rgb, depth, gt
