"""The serving engine (continuous batching over the camera pool). Each
camera's results must be the same alone and in any mix of cameras sharing
ticks; admission follows the memory budget; full queues drop frames; every
frame gets a latency."""
import random
import time

import numpy as np
import pytest

import paper_2110_14934_gb300 as G
from parity import scene_frames, to_dev, words

pytestmark = pytest.mark.gpu

CAMS = [(45, 83, 3), (64, 96, 5), (33, 40, 4), (120, 160, 5), (1, 1, 3), (240, 320, 3)]


def _pinned(frames):
    import torch
    rgb, depth, _ = frames
    r = torch.from_numpy(np.ascontiguousarray(rgb)).pin_memory()
    d = torch.from_numpy(np.ascontiguousarray(depth).view(np.int16)).pin_memory()
    return r, d


TRANSFER = [pytest.param(G.SERVE_ZERO_COPY, id="zero_copy"), pytest.param(G.SERVE_COPY, id="copy")]


@pytest.mark.parametrize("transfer", TRANSFER)
@pytest.mark.parametrize("prec", [G.PREC_F16, G.PREC_F32])
def test_server_results_equal_alone_in_a_changing_mix(prec, transfer):
    import torch
    n = 10
    frames = [scene_frames(700 + i, H, W, 1, 40, n) for i, (H, W, M) in enumerate(CAMS)]
    alone = {}
    for i, (H, W, M) in enumerate(CAMS):
        g = G.GMM(H, W, M, precision=prec)
        for t in range(n):
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            alone[(i, t)] = words(g.apply(r, d)).copy()
    srv = G.Server(precision=prec, max_cams=8, queue_depth=n, transfer=transfer)
    ids = [srv.admit(H, W, M) for (H, W, M) in CAMS]
    pinned = [_pinned(f) for f in frames]
    masks = {(i, t): torch.zeros((H, G.mask_words_per_row(W)), dtype=torch.int32).pin_memory()
             for i, (H, W, M) in enumerate(CAMS) for t in range(n)}
    order = [(i, t) for t in range(n) for i in range(len(CAMS))]
    rng = random.Random(4)
    # frames of a camera stay in order; cameras interleave irregularly, with
    # pauses so that ticks see different subsets of cameras
    pos = [0] * len(CAMS)
    tickets = []
    while any(p < n for p in pos):
        i = rng.choice([k for k in range(len(CAMS)) if pos[k] < n])
        t = pos[i]
        tickets.append(srv.push(ids[i], pinned[i][0][t], pinned[i][1][t], masks[(i, t)]))
        pos[i] += 1
        if rng.random() < 0.2:
            time.sleep(rng.choice([0.0, 0.0005, 0.002]))
    for tk in tickets:
        srv.wait(tk, 30000)
    for key in alone:
        assert np.array_equal(masks[key].numpy().view(np.uint32), alone[key]), key
    st = srv.stats()
    assert st["completed"] == len(order) and st["dropped"] == 0 and st["ticks"] >= n
    lat = srv.latencies_ms()
    assert lat.size == len(order) and np.all(lat > 0) and np.all(lat < 30000)
    # the traces: one per completed frame, in the same order, times in order
    tr = srv.traces()
    assert tr.size == lat.size
    assert sorted(tr["ticket"].tolist()) == sorted(tickets)
    assert np.all(tr["t_arrival"] <= tr["t_pushed"]) and np.all(tr["t_pushed"] <= tr["t_batched"])
    assert np.all(tr["t_batched"] <= tr["t_submitted"])
    assert np.all(tr["t_submitted"] <= tr["t_done"])
    assert np.allclose((tr["t_done"] - tr["t_arrival"]) * 1e3, lat, rtol=1e-5, atol=1e-3)
    assert np.all((tr["tick_frames"] >= 1) & (tr["tick_frames"] <= len(CAMS)))
    assert set(tr["cam"].tolist()) == set(ids)
    srv.close()


@pytest.mark.parametrize("transfer", TRANSFER)
def test_server_budget_admission_and_release(transfer):
    per = G.state_bytes(120, 160, 5, G.PREC_F16)
    srv = G.Server(budget_bytes=int(2.5 * per) + 400000, precision=G.PREC_F16, max_cams=4,
                   transfer=transfer)
    a = srv.admit(120, 160, 5)
    b = srv.admit(120, 160, 5)
    with pytest.raises(G.GMMError) as e:
        srv.admit(120, 160, 5)
    assert e.value.code == G.EBUDGET
    st = srv.stats()
    assert st["admitted"] == 2 and st["rejected"] == 1 and st["live_cams"] == 2
    srv.release(a, 10000)
    c = srv.admit(120, 160, 5)
    st = srv.stats()
    assert st["admitted"] == 3 and st["released"] == 1 and st["live_cams"] == 2
    srv.release(b, 10000)
    srv.release(c, 10000)
    assert srv.stats()["used_bytes"] == 0
    srv.close()


@pytest.mark.parametrize("transfer", TRANSFER)
def test_server_full_queue_drops_frames(transfer):
    import torch
    H, W, M = 720, 1280, 5
    rgb, depth = _pinned(scene_frames(3, H, W, 1, 0, 2))
    srv = G.Server(precision=G.PREC_F16, max_cams=2, queue_depth=1, transfer=transfer)
    cam = srv.admit(H, W, M)
    mask = torch.zeros((H, G.mask_words_per_row(W)), dtype=torch.int32).pin_memory()
    tickets, drops = [], 0
    for k in range(40):
        try:
            tickets.append(srv.push(cam, rgb[k % 2], depth[k % 2], mask))
        except G.GMMError as e:
            assert e.code == G.EBUDGET
            drops += 1
    for tk in tickets:
        srv.wait(tk, 30000)
    st = srv.stats()
    assert drops >= 1 and st["dropped"] == drops
    assert st["pushed"] == len(tickets) and st["completed"] == len(tickets)
    srv.release(cam, 10000)
    srv.close()


def test_server_transfer_mode_rules():
    """The mode is fixed once a camera is admitted; the zero-copy mode takes
    only host memory the device can reach (pageable memory is refused at
    push, with no frame queued), while the copy mode uploads from it."""
    import torch
    H, W, M = 48, 64, 3
    rgb, depth, _ = scene_frames(9, H, W, 1, 0, 1)
    srv = G.Server(precision=G.PREC_F16, max_cams=2)
    cam = srv.admit(H, W, M)
    with pytest.raises(G.GMMError) as e:
        G._check(G.load_library().gmm_server_set_transfer(srv._s, G.SERVE_COPY))
    assert e.value.code == G.EINVAL
    pageable_mask = np.zeros((H, G.mask_words_per_row(W)), np.uint32)
    with pytest.raises(G.GMMError) as e:
        srv.push(cam, np.ascontiguousarray(rgb[0]), np.ascontiguousarray(depth[0]), pageable_mask)
    assert e.value.code == G.EINVAL and srv.stats()["pushed"] == 0
    srv.close()
    srv = G.Server(precision=G.PREC_F16, max_cams=2, transfer=G.SERVE_COPY)
    cam = srv.admit(H, W, M)
    want = G.GMM(H, W, M, precision=G.PREC_F16)
    r, d = to_dev(rgb[0], depth[0])
    ref = words(want.apply(r, d))
    srv.wait(srv.push(cam, np.ascontiguousarray(rgb[0]), np.ascontiguousarray(depth[0]),
                      pageable_mask), 30000)
    assert np.array_equal(pageable_mask, ref)
    srv.close()
