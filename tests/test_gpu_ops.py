"""GPU tests of the standalone operators (List 1 alone, 3x3 opening), the
host-memory paths, the device frame generator and the host-side argument
checks that must stop bad calls before any launch."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_2110_14934_gb300 as G
import synth
from parity import Pair, scene_frames, to_dev, words

pytestmark = pytest.mark.gpu


def test_fuse_masks_exhaustive_sequences():
    """Every (colour, depth) sequence of length 6 from both initial labels,
    one pixel per sequence, stepped through gmm_fuse_masks; bit-exact against
    List 1 in the oracle."""
    import torch
    L = 6
    seqs = list(itertools.product(range(4), repeat=L))
    n = 2 * len(seqs)
    H, W = 1, n
    F0 = np.array([0] * len(seqs) + [1] * len(seqs))
    steps = np.array(seqs + seqs)  # [n, L]
    fusion = torch.from_numpy((F0 | (3 << 1)).astype(np.uint8)).cuda()
    out = torch.empty((1, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
    Fo = F0.copy(); co = np.zeros(n, int)
    for t in range(L):
        rgb_bits = (steps[:, t] >> 1) & 1
        d_bits = steps[:, t] & 1
        fr = torch.from_numpy(G.pack_mask(rgb_bits[None].astype(bool)).view(np.int32)).cuda()
        fd = torch.from_numpy(G.pack_mask(d_bits[None].astype(bool)).view(np.int32)).cuda()
        G.fuse_masks(fr, fd, fusion, out, H, W)
        for i in range(n):
            Fo[i], co[i] = O.fuse(int(rgb_bits[i]), int(d_bits[i]), int(Fo[i]), int(co[i]))
        torch.cuda.synchronize()
        got = G.unpack_mask(words(out), H, W)[0]
        assert np.array_equal(got, Fo.astype(bool)), t
        fb = fusion.cpu().numpy().astype(int)
        assert np.array_equal(fb & 1, Fo) and np.array_equal(((fb >> 1) & 7) - 3, co), t


def test_fuse_masks_matches_the_tick_at_full_size():
    """At 1920x1080, gmm_fuse_masks applied to a tick's colour and depth
    masks and the List-1 bytes from before the tick gives the tick's fused
    mask and List-1 state (label and counter, the low four bits) exactly: the
    operator and the fused kernel run the same List 1. (Bit 4, the depth
    model's start, belongs to the tick, not to List 1.)"""
    import torch
    H, W, M = 1080, 1920, 5
    s = synth.scene(606, H, W, 1)
    rgb, dep, _ = synth.frames_device(s, 40, 4, with_gt=False)
    g = G.GMM(H, W, M)
    out = g.new_mask()
    for t in range(4):
        before = torch.from_numpy(g.fusion()).cuda()
        m, fc, fd = g.new_mask(), g.new_mask(), g.new_mask()
        g.apply(rgb[t], dep[t], m, fc, fd)
        torch.cuda.synchronize()
        if t == 0:
            continue  # the first tick initialises the models
        G.fuse_masks(fc, fd, before, out, H, W)
        torch.cuda.synchronize()
        assert torch.equal(out, m), t
        assert np.array_equal(before.cpu().numpy() & 15, g.fusion() & 15), t


@pytest.mark.parametrize("H,W", [(1, 1), (1, 40), (5, 1), (9, 13), (33, 65), (100, 1000)])
def test_morph_open3_matches_oracle(H, W):
    import torch
    rng = np.random.default_rng(H * 1000 + W)
    for p in (0.4, 0.8, 0.97):
        m = rng.random((H, W)) < p
        packed = G.pack_mask(m)
        # garbage in the padding bits must not leak into the result
        if W % 32:
            packed[:, -1] |= np.uint32(0xFFFFFFFF) << np.uint32(W % 32)
        src = torch.from_numpy(packed.view(np.int32)).cuda()
        dst = torch.zeros_like(src)
        G.morph_open3(src, dst, H, W)
        torch.cuda.synchronize()
        got = G.unpack_mask(words(dst), H, W)
        assert np.array_equal(got, O.morph_open3(m.astype(np.uint8)).astype(bool))
        if W % 32:
            assert not np.any(words(dst)[:, -1] >> np.uint32(W % 32))


def test_handle_with_morph_open():
    import torch
    H, W, M = 60, 90, 3
    rgb, depth, _ = scene_frames(21, H, W, 0, 0, 8)
    plain = G.GMM(H, W, M)
    opened = G.GMM(H, W, M, morph_open=True)
    for t in range(8):
        r, d = to_dev(rgb[t], depth[t])
        a = plain.apply(r, d)
        b = opened.apply(r, d)
        torch.cuda.synchronize()
        ref = O.morph_open3(G.unpack_mask(words(a), H, W).astype(np.uint8)).astype(bool)
        assert np.array_equal(G.unpack_mask(words(b), H, W), ref)


@pytest.mark.parametrize("prec,morph,reuse", [(G.PREC_F32, False, False), (G.PREC_F16, False, False),
                                              (G.PREC_F32, True, False), (G.PREC_F32, False, True),
                                              (G.PREC_F16, True, True)])
def test_back_to_back_ticks_equal_synchronised_ticks(prec, morph, reuse):
    """Consecutive ticks (and openings) are launched as programmatic
    dependents of the kernel before them. Queued back to back with no host
    synchronisation (directly one after another, or with each frame copied
    into one reused input buffer, and that buffer cleared after the tick, by
    ordinary stream work in between), the masks and the final state equal a
    run that synchronises the device after every tick."""
    import torch
    H, W, M, n = 96, 160, 5, 24
    rgb, depth, _ = scene_frames(31, H, W, 1, 0, n)
    frames = [to_dev(rgb[t], depth[t]) for t in range(n)]
    ref_g = G.GMM(H, W, M, precision=prec, morph_open=morph)
    ref = []
    for t in range(n):
        ref.append(words(ref_g.apply(*frames[t])).copy())
        torch.cuda.synchronize()
    g = G.GMM(H, W, M, precision=prec, morph_open=morph)
    r_buf, d_buf = torch.empty_like(frames[0][0]), torch.empty_like(frames[0][1])
    outs = [g.new_mask() for _ in range(n)]
    for t in range(n):
        if reuse:
            r_buf.copy_(frames[t][0])
            d_buf.copy_(frames[t][1])
            g.apply(r_buf, d_buf, outs[t])
            r_buf.zero_()  # may only land after this tick read the frame
        else:
            g.apply(*frames[t], outs[t])
    torch.cuda.synchronize()
    for t in range(n):
        assert np.array_equal(words(outs[t]), ref[t]), t
    assert np.array_equal(g.planes(), ref_g.planes())


@pytest.mark.parametrize("prec", [G.PREC_F32, G.PREC_F16])
def test_zero_copy_host_buffers_match_device_path(prec):
    """gmm_apply on page-locked host frames and a page-locked host mask (the
    kernel reads and writes them over the host link) equals the device path."""
    import torch
    H, W, M = 70, 100, 5
    rgb, depth, _ = scene_frames(41, H, W, 1, 0, 6)
    dev = G.GMM(H, W, M, precision=prec)
    zc = G.GMM(H, W, M, precision=prec)
    for t in range(6):
        ref = words(dev.apply(*to_dev(rgb[t], depth[t]))).copy()
        r = torch.from_numpy(rgb[t].copy()).pin_memory()
        d = torch.from_numpy(depth[t].view(np.int16).copy()).pin_memory()
        m = torch.zeros((H, G.mask_words_per_row(W)), dtype=torch.int32).pin_memory()
        zc.apply(r, d, m)
        torch.cuda.synchronize()
        assert np.array_equal(m.numpy().view(np.uint32), ref), t
    assert np.array_equal(zc.planes(), dev.planes())


def test_host_path_and_pipeline_match_device_path():
    import torch
    H, W, M = 50, 70, 4
    rgb, depth, _ = scene_frames(8, H, W, 1, 0, 10)
    dev = G.GMM(H, W, M)
    host = G.GMM(H, W, M)
    pipe = G.GMM(H, W, M)
    ref = []
    for t in range(10):
        r, d = to_dev(rgb[t], depth[t])
        ref.append(words(dev.apply(r, d)).copy())
    for t in range(10):
        assert np.array_equal(host.apply_host(rgb[t], depth[t]), ref[t])
    # pipelined: pinned buffers, several frames in flight
    rgb_p = [torch.from_numpy(rgb[t].copy()).pin_memory() for t in range(10)]
    dep_p = [torch.from_numpy(depth[t].view(np.int16).copy()).pin_memory() for t in range(10)]
    masks = [torch.zeros((H, G.mask_words_per_row(W)), dtype=torch.int32).pin_memory()
             for _ in range(10)]
    tickets = [pipe.pipe_submit(rgb_p[t], dep_p[t], masks[t]) for t in range(10)]
    for t, tk in enumerate(tickets):
        pipe.pipe_wait(tk, 10000)
        assert np.array_equal(masks[t].numpy().view(np.uint32), ref[t]), t
    assert np.array_equal(dev.planes(), pipe.planes())


def test_host_side_checks_reject_bad_calls():
    """Plain host pointers, misaligned pointers and wrong planes are refused
    on the host; the handle stays usable afterwards."""
    import torch
    H, W = 8, 40
    g = G.GMM(H, W, 3)
    L = G.load_library()
    rgb = np.zeros((H, W, 3), np.uint8); dep = np.zeros((H, W), np.uint16)
    mask = np.zeros((H, 2), np.uint32)
    assert L.gmm_apply(g._h, rgb.ctypes.data, dep.ctypes.data, mask.ctypes.data) == G.EINVAL
    r = torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")
    d = torch.zeros((H * W + 1,), dtype=torch.int16, device="cuda")
    m = torch.zeros((H, 2), dtype=torch.int32, device="cuda")
    bytes_d = d.view(torch.uint8).reshape(-1)
    bytes_m = m.view(torch.uint8).reshape(-1)
    assert (bytes_d[1:].data_ptr() - d.data_ptr()) == 1
    assert (bytes_m[2:].data_ptr() - m.data_ptr()) == 2
    assert L.gmm_apply(g._h, r.data_ptr(), bytes_d[1:].data_ptr(), m.data_ptr()) == G.EINVAL
    assert L.gmm_apply(g._h, r.data_ptr(), d.data_ptr(), bytes_m[2:].data_ptr()) == G.EINVAL
    out = np.zeros(H * W, np.float32)
    assert L.gmm_state_get(g._h, 9, 0, out.ctypes.data, out.size) == G.EINVAL
    assert L.gmm_state_get(g._h, 0, 3, out.ctypes.data, out.size) == G.EINVAL
    assert L.gmm_state_get(g._h, 0, 0, out.ctypes.data, out.size - 1) == G.EINVAL
    g.apply(r, d[:H * W].view(H, W))
    g.sync()


def test_device_generator_matches_host():
    import torch
    for seed, H, W, kind in ((1, 48, 64, 0), (2, 37, 51, 1), (3, 1080, 1920, 1)):
        s = synth.scene(seed, H, W, kind)
        f0 = 45
        rgb, dep, gt = synth.frames_host(s, f0, 3)
        rd, dd, gd = synth.frames_device(s, f0, 3)
        torch.cuda.synchronize()
        assert np.array_equal(rd.cpu().numpy(), rgb)
        assert np.array_equal(dd.cpu().numpy().view(np.uint16), dep)
        assert np.array_equal(gd.cpu().numpy(), gt)


def test_bounded_wait_runs_out_and_reports():
    """Failure detection without a GPU fault: a device wait on a barrier that
    nothing completes (the same time-bounded wait the staged kernel's
    pipeline uses) gives up after its limit, the kernel reports it and
    returns, and the context keeps working."""
    import torch
    for ms in (50, 300):
        r = G.wait_selftest(ms)
        assert r["timed_out"], r
        assert ms <= r["waited_ms"] < ms + 500, r
    g = G.GMM(45, 83, 3)
    rgb, depth, _ = scene_frames(3, 45, 83, 0, 0, 2)
    for t in range(2):
        r_, d_ = to_dev(rgb[t], depth[t])
        g.apply(r_, d_)
    torch.cuda.synchronize()
    g.sync()


def test_sticky_cuda_error_through_the_test_hook():
    """A CUDA failure recorded on a handle (injected on the host, no GPU
    fault) makes every later launching or copying call fail with GMM_ECUDA
    and a message naming the error; destroying the handle still works. The
    same for a pool."""
    import torch
    H, W = 24, 40
    rgb, depth, _ = scene_frames(4, H, W, 0, 0, 2)
    g = G.GMM(H, W, 3)
    r, d = to_dev(rgb[0], depth[0])
    g.apply(r, d)
    torch.cuda.synchronize()
    L = G.load_library()
    assert L.gmm_inject_cuda_error(g._h, 999) == G.OK  # cudaErrorUnknown
    with pytest.raises(G.GMMError) as ei:
        g.apply(r, d)
    assert ei.value.code == G.ECUDA and "earlier CUDA failure" in str(ei.value)
    with pytest.raises(G.GMMError) as ei:
        g.sync()
    assert ei.value.code == G.ECUDA
    g.close()
    assert L.gmm_inject_cuda_error(None, 999) == G.EINVAL
    pool = G.Pool(max_cams=2)
    cam = pool.admit(H, W, 3)
    m = torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
    pool.submit(cam, r, d, m)
    pool.tick()
    assert L.gmm_pool_inject_cuda_error(pool._p, 999) == G.OK
    pool.submit(cam, r, d, m)
    with pytest.raises(G.GMMError) as ei:
        pool.tick()
    assert ei.value.code == G.ECUDA
    pool.close()
