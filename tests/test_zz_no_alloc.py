"""The allocation-free entry point gmm_apply_open3_noalloc, called through the
C ABI, against the regular path (a handle created with morph_open = 1, whose
gmm_apply keeps the unopened mask in a buffer it allocated).

The allocation-free call exists for callers that must not allocate device
memory (an application that reserves the GPU's memory up front, a real-time
loop that may not wait on the allocator, code where allocation calls are not
allowed): it keeps the unopened mask in a fixed array inside the library and
takes the model state from the caller. Both paths run the same kernels, so
the masks and the state must agree exactly, on two calls in a row (the first
initialises the caller's state, the second updates it).

The file name sorts last, so pytest collects it after every other test: this
test was added on its own, and should it fail in a run that stops at the first
failure (-x), every other test has already run. It passes in either order:
alone in a fresh process, and after the rest of the suite."""
import ctypes

import numpy as np
import pytest

import paper_2110_14934_gb300 as G
from parity import scene_frames, to_dev, words

pytestmark = pytest.mark.gpu


def _config(L, H, W, M, prec):
    cfg = G.GMMConfig()
    L.gmm_config_init(ctypes.byref(cfg), H, W, M, 0.01, 2.5, 0.7, 225.0, 0.05)
    cfg.precision = prec
    return cfg


def _caller_plane(state, H, W, M, prec, comp, field):
    """Decode one plane of the caller-owned state (layout of gmm.h)."""
    import torch
    w_pad = ((W + 31) // 32) * 32
    n_tiles = (H * w_pad + 255) // 256
    if prec == G.PREC_F32:
        flat = state.view(torch.float32)
    elif field in (G.PLANE_W_C, G.PLANE_W_D):
        flat = state.view(torch.bfloat16)
    else:
        flat = state.view(torch.float16)
    if prec == G.PREC_F32:
        tiles = flat[:n_tiles * 8 * M * 256].reshape(n_tiles, 8 * M, 256)
        plane = tiles[:, 8 * comp + field, :].reshape(-1)[:H * w_pad]
    else:
        group, slot = {G.PLANE_W_C: (0, 0), G.PLANE_W_D: (0, 1), G.PLANE_MU_R: (0, 2),
                       G.PLANE_MU_G: (0, 3), G.PLANE_MU_B: (1, 0), G.PLANE_V_C: (1, 1),
                       G.PLANE_MU_D: (1, 2), G.PLANE_V_D: (1, 3)}[field]
        tiles = flat[:n_tiles * 8 * M * 256].reshape(n_tiles, 2 * M, 256, 4)
        plane = tiles[:, 2 * comp + group, :, slot].reshape(-1)[:H * w_pad]
    return plane.float().reshape(H, w_pad)[:, :W].cpu().numpy()


@pytest.mark.parametrize("H,W,M,prec", [(45, 83, 3, G.PREC_F32), (120, 160, 5, G.PREC_F32),
                                        (64, 96, 4, G.PREC_F16), (1, 1, 3, G.PREC_F32)])
def test_noalloc_matches_handle_path_two_calls(H, W, M, prec):
    import torch
    L = G.load_library()
    rgb, depth, _ = scene_frames(77 + M + H, H, W, 1, 48, 2)
    ref = G.GMM(H, W, M, precision=prec, morph_open=True)
    cfg = _config(L, H, W, M, prec)
    # caller-owned state, deliberately not cleared: the first call initialises it
    state = torch.full((G.state_bytes(H, W, M, prec),), 0xAB, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for t in range(2):
        r, d = to_dev(rgb[t], depth[t])
        want = ref.apply(r, d)
        got = torch.full_like(want, -1)
        rc = L.gmm_apply_open3_noalloc(ctypes.byref(cfg), state.data_ptr(), 1 if t == 0 else 0,
                                       r.data_ptr(), d.data_ptr(), got.data_ptr(),
                                       stream.cuda_stream)
        assert rc == G.OK, L.gmm_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(words(got), words(want)), f"mask differs on call {t}"
        for comp in range(M):
            for field in range(8):
                a = _caller_plane(state, H, W, M, prec, comp, field)
                b = ref.state_get(field, comp)
                assert np.array_equal(a, b), (t, comp, G.PLANES[field])


def test_noalloc_rejects_frames_above_the_scratch_limit():
    L = G.load_library()
    cfg = _config(L, 4096, 4097, 3, G.PREC_F32)  # 4096 * 129 words > 2^18
    rc = L.gmm_apply_open3_noalloc(ctypes.byref(cfg), None, 1, None, None, None, None)
    assert rc == G.EINVAL
    assert "GMM_NOALLOC_MAX_MASK_WORDS" in L.gmm_last_error().decode()


@pytest.mark.parametrize("H,W,M,prec", [(1, 33, 5, G.PREC_F16), (33, 1, 4, G.PREC_F32),
                                        (7, 1000, 3, G.PREC_F16)])
def test_noalloc_state_and_mask_stay_in_bounds(H, W, M, prec):
    """The caller-owned state and the mask sit between canary bytes: three
    calls at ragged sizes leave the canaries intact."""
    import torch
    L = G.load_library()
    guard, canary = 4096, 0xA5
    nbytes = G.state_bytes(H, W, M, prec)
    sbuf = torch.full((guard + nbytes + guard,), canary, dtype=torch.uint8, device="cuda")
    state = sbuf[guard:guard + nbytes]
    mwords = H * G.mask_words_per_row(W)
    mbuf = torch.full((guard + 4 * mwords + guard,), canary, dtype=torch.uint8, device="cuda")
    mask = mbuf[guard:guard + 4 * mwords]
    cfg = _config(L, H, W, M, prec)
    rgb, depth, _ = scene_frames(5 + H, H, W, 1, 0, 3)
    stream = torch.cuda.current_stream()
    for t in range(3):
        r, d = to_dev(rgb[t], depth[t])
        rc = L.gmm_apply_open3_noalloc(ctypes.byref(cfg), state.data_ptr(), 1 if t == 0 else 0,
                                       r.data_ptr(), d.data_ptr(), mask.data_ptr(),
                                       stream.cuda_stream)
        assert rc == G.OK, L.gmm_last_error()
    torch.cuda.synchronize()
    for buf, n in ((sbuf, nbytes), (mbuf, 4 * mwords)):
        b = buf.cpu().numpy()
        assert (b[:guard] == canary).all() and (b[guard + n:] == canary).all()


def test_noalloc_calls_allocate_no_device_memory():
    """After one warm-up call (the first call in a context looks up the
    scratch array and, under lazy module loading, loads the module that holds
    it), further calls leave both torch's allocator and the device's free
    memory exactly where they were."""
    import torch
    L = G.load_library()
    H, W, M, prec = 96, 160, 5, G.PREC_F32
    rgb, depth, _ = scene_frames(303, H, W, 1, 10, 6)
    frames = [to_dev(rgb[t], depth[t]) for t in range(6)]
    state = torch.empty((G.state_bytes(H, W, M, prec),), dtype=torch.uint8, device="cuda")
    mask = torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
    cfg = _config(L, H, W, M, prec)
    stream = torch.cuda.current_stream()

    def call(t):
        r, d = frames[t]
        rc = L.gmm_apply_open3_noalloc(ctypes.byref(cfg), state.data_ptr(), 1 if t == 0 else 0,
                                       r.data_ptr(), d.data_ptr(), mask.data_ptr(),
                                       stream.cuda_stream)
        assert rc == G.OK, L.gmm_last_error()

    call(0)
    torch.cuda.synchronize()
    allocated = torch.cuda.memory_allocated()
    free_before = torch.cuda.mem_get_info()[0]
    for t in range(1, 6):
        call(t)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == allocated
    assert torch.cuda.mem_get_info()[0] == free_before
