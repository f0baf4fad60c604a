"""The multi-camera pool: one persistent launch per tick over every camera
with a submitted frame. Results must equal each camera run alone (same
kernel arithmetic, so bit-identical), whatever mix of cameras shares a tick,
and must match the oracle."""
import numpy as np
import pytest

import paper_2110_14934_gb300 as G
from parity import FreeRun, scene_frames, to_dev, words

pytestmark = pytest.mark.gpu

CAMS = [(45, 83, 3), (64, 96, 5), (33, 40, 4), (1, 1, 3), (120, 160, 5)]


def _frames(n):
    return [scene_frames(500 + i, H, W, i % 2, 0, n) for i, (H, W, M) in enumerate(CAMS)]


def _alone(frames, schedule, precision=G.PREC_F32):
    """Each camera in its own handle, fed only on the ticks it is scheduled."""
    import torch
    out = {}
    for i, (H, W, M) in enumerate(CAMS):
        g = G.GMM(H, W, M, precision=precision)
        k = 0
        for t, active in enumerate(schedule):
            if i in active:
                r, d = to_dev(frames[i][0][k], frames[i][1][k])
                out[(i, t)] = words(g.apply(r, d)).copy()
                k += 1
        torch.cuda.synchronize()
        out[i] = g.planes()
    return out


def _pooled(frames, schedule, graph=False, launch=None, precision=G.PREC_F32, online=0,
            prefetch=True):
    import torch
    pool = G.Pool(precision=precision, max_cams=8)
    pool.set_prefetch(prefetch)
    if graph:
        pool.use_graph(True)
    if launch:
        pool.set_launch(*launch)
    if online:
        pool.autotune_online(online)
    ids = [pool.admit(H, W, M) for (H, W, M) in CAMS]
    out = {}
    pos = [0] * len(CAMS)
    for t, active in enumerate(schedule):
        masks = {}
        for i in active:
            H, W, M = CAMS[i]
            r, d = to_dev(frames[i][0][pos[i]], frames[i][1][pos[i]])
            masks[i] = (torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda"), r, d)
            pool.submit(ids[i], r, d, masks[i][0])
            pos[i] += 1
        pool.tick()
        torch.cuda.synchronize()
        for i in active:
            out[(i, t)] = words(masks[i][0]).copy()
    for i in range(len(CAMS)):
        out[i] = pool.planes(ids[i])
    return out, pool, ids


def test_pool_equals_alone_every_tick():
    n = 12
    frames = _frames(n)
    schedule = [set(range(len(CAMS)))] * n
    a = _alone(frames, schedule)
    b, _, _ = _pooled(frames, schedule)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_pool_equals_alone_in_a_changing_mix():
    """Cameras join the tick on different schedules (continuous batching):
    every camera's masks and state equal its run alone."""
    n = 14
    frames = _frames(n)
    rng = np.random.default_rng(3)
    schedule = [set(int(i) for i in np.nonzero(rng.random(len(CAMS)) < 0.6)[0]) for _ in range(n)]
    a = _alone(frames, schedule)
    b, _, _ = _pooled(frames, schedule)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def _valid_shape(shape):
    """A persistent shape (tiles a multiple of the block) or the flat form."""
    return shape["threads"] in (64, 128, 256) and (
        shape["ctas_per_sm"] == -1 or shape["tile_pixels"] % shape["threads"] == 0)


@pytest.mark.parametrize("launch", [(128, 1, 128), (256, 2, 2048), (256, 0, 32768), (64, 6, 2048),
                                    (64, 0, 64), (64, -1, 0), (256, -1, 0)])
def test_pool_graph_and_launch_shapes(launch):
    n = 6
    frames = _frames(n)
    schedule = [set(range(len(CAMS)))] * 3 + [{0, 2, 4}] * 3
    a = _alone(frames, schedule)
    b, _, _ = _pooled(frames, schedule, graph=True, launch=launch)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("launch", [(128, 8, 1024), (64, -1, 0), (256, -1, 0)])
def test_pool_fp16_launch_shapes(launch):
    """FP16/BF16 state: the persistent and the flat form (two pixels per
    lane, a half chunk at each camera's end) equal each camera alone."""
    n = 5
    frames = _frames(n)
    schedule = [set(range(len(CAMS)))] * 3 + [{1, 3, 4}] * 2
    a = _alone(frames, schedule, precision=G.PREC_F16)
    b, _, _ = _pooled(frames, schedule, graph=True, launch=launch, precision=G.PREC_F16)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_pool_matches_oracle():
    """Every camera of a pooled tick against the oracle, free-running with
    every difference classified (parity.FreeRun)."""
    import torch
    n = 10
    frames = _frames(n)
    pool = G.Pool(max_cams=8)
    ids = [pool.admit(H, W, M) for (H, W, M) in CAMS]
    frs = [FreeRun(H, W, M) for (H, W, M) in CAMS]
    before = [None] * len(CAMS)
    for t in range(n):
        outs = []
        for i, (H, W, M) in enumerate(CAMS):
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            ms = [torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
                  for _ in range(3)]
            pool.submit(ids[i], r, d, *ms)
            outs.append(ms + [r, d])  # the frames stay alive until the tick has run
        pool.tick()
        torch.cuda.synchronize()
        for i, (H, W, M) in enumerate(CAMS):
            g = {k: G.unpack_mask(words(v), H, W)
                 for k, v in zip(("fused", "fg_rgb", "fg_d"), outs[i][:3])}
            after = (pool.planes(ids[i]), pool.fusion(ids[i]))
            frs[i].step(frames[i][0][t], frames[i][1][t], g, before[i], after)
            before[i] = after
    for f in frs:
        f.check()


def test_pool_budget_and_release():
    per = G.state_bytes(64, 96, 5)
    pool = G.Pool(budget_bytes=2 * per + 10, max_cams=4)
    a = pool.admit(64, 96, 5)
    b = pool.admit(64, 96, 5)
    with pytest.raises(G.GMMError) as e:
        pool.admit(64, 96, 5)
    assert e.value.code == G.EBUDGET
    assert pool.state_used() == 2 * per
    pool.release(a)
    c = pool.admit(64, 96, 5)
    assert c == a and pool.state_used() == 2 * per
    pool.release(b)
    pool.release(c)
    assert pool.state_used() == 0
    pool.sync()


def test_pool_autotune_leaves_state_unchanged():
    import torch
    frames = _frames(4)
    pool = G.Pool(max_cams=8)
    ids = [pool.admit(H, W, M) for (H, W, M) in CAMS]
    keep = []
    for t in range(2):
        for i, (H, W, M) in enumerate(CAMS):
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            m = torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
            keep.append((r, d, m))
            pool.submit(ids[i], r, d, m)
        if t == 0:
            pool.tick()
    before = [pool.planes(c) for c in ids]
    shape = pool.autotune(iters=2)
    assert _valid_shape(shape)
    after = [pool.planes(c) for c in ids]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    pool.tick()  # the submission survives the autotuner
    pool.sync()


def test_pool_online_tuning_changes_nothing_but_speed():
    """Online tuning runs real ticks under every candidate launch shape (30
    of them, one tick each here, then 4 finalists two ticks each; graphs
    requested): the results still equal each camera run alone, tuning
    finishes, and graph use resumes."""
    n = 50
    frames = _frames(n)
    schedule = [set(range(len(CAMS)))] * n
    a = _alone(frames, schedule)
    b, pool, _ = _pooled(frames, schedule, graph=True, online=1)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    tuning, shape = pool.tuning()
    assert not tuning
    assert _valid_shape(shape)
    pool.sync()


@pytest.mark.parametrize("graph,launch", [(False, None), (True, None), (True, (128, -1, 0))])
def test_pool_more_cameras_than_one_launch_holds(graph, launch):
    """A tick with more cameras than one launch's parameter block holds (128)
    is split into several launches; every camera still equals its run alone,
    in ticks of changing size (the graph's nodes updated or rebuilt)."""
    import torch
    n_cams, n = 131, 4
    shapes = [(8 + (i % 3), 33 + 7 * (i % 5), 3 + (i % 3)) for i in range(n_cams)]
    frames = [scene_frames(3000 + i, H, W, i % 2, 0, n) for i, (H, W, M) in enumerate(shapes)]
    schedule = [set(range(n_cams)), set(range(n_cams)), set(range(0, n_cams, 2)),
                set(range(n_cams))]
    alone = {}
    for i, (H, W, M) in enumerate(shapes):
        g = G.GMM(H, W, M)
        k = 0
        for t, active in enumerate(schedule):
            if i in active:
                r, d = to_dev(frames[i][0][k], frames[i][1][k])
                alone[(i, t)] = words(g.apply(r, d)).copy()
                k += 1
        torch.cuda.synchronize()
        alone[i] = g.planes()
        g.close()
    pool = G.Pool(max_cams=n_cams)
    pool.use_graph(graph)
    if launch:
        pool.set_launch(*launch)
    ids = [pool.admit(H, W, M) for (H, W, M) in shapes]
    pos = [0] * n_cams
    got = {}
    for t, active in enumerate(schedule):
        masks = {}
        for i in sorted(active):
            H, W, M = shapes[i]
            r, d = to_dev(frames[i][0][pos[i]], frames[i][1][pos[i]])
            m = torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
            masks[i] = (m, r, d)
            pool.submit(ids[i], r, d, m)
            pos[i] += 1
        pool.tick()
        torch.cuda.synchronize()
        for i in active:
            got[(i, t)] = words(masks[i][0]).copy()
    for i in range(n_cams):
        got[i] = pool.planes(ids[i])
    pool.close()
    assert alone.keys() == got.keys()
    for key in alone:
        assert np.array_equal(alone[key], got[key]), key


def test_two_pools_on_two_streams():
    """Two pools ticking on two streams without synchronising in between
    (their launches share the device's argument bank, taken in turn): each
    camera still equals its run alone."""
    import torch
    n = 6
    frames = _frames(n)
    a = _alone(frames, [set(range(len(CAMS)))] * n)
    halves = [list(range(0, len(CAMS), 2)), list(range(1, len(CAMS), 2))]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pools = [G.Pool(max_cams=8), G.Pool(max_cams=8)]
    pools[1].use_graph(True)
    ids = [{i: pools[h].admit(*CAMS[i]) for i in halves[h]} for h in range(2)]
    keep, masks = [], {}
    torch.cuda.synchronize()
    for t in range(n):
        for h in range(2):
            with torch.cuda.stream(streams[h]):
                for i in halves[h]:
                    H, W, M = CAMS[i]
                    r = torch.from_numpy(np.ascontiguousarray(frames[i][0][t])).cuda()
                    d = torch.from_numpy(np.ascontiguousarray(frames[i][1][t]).view(np.int16)).cuda()
                    m = torch.empty((H, G.mask_words_per_row(W)), dtype=torch.int32, device="cuda")
                    keep.append((r, d, m))
                    masks[(i, t)] = m
                    pools[h].submit(ids[h][i], r, d, m)
                pools[h].tick(streams[h])
    torch.cuda.synchronize()
    for (i, t), m in masks.items():
        assert np.array_equal(words(m), a[(i, t)]), (i, t)
    for h in range(2):
        for i in halves[h]:
            assert np.array_equal(pools[h].planes(ids[h][i]), a[i]), i
        pools[h].close()


@pytest.mark.parametrize("graph", [False, True])
def test_pool_fp16_prefetch_changes_nothing_but_speed(graph):
    """FP16/BF16 pool with tiles of one pixel per thread and one CTA per SM,
    so a tick has more than two waves of tiles and CTAs take their next tile
    early and prefetch it: masks and state equal each camera run alone, and
    the pool with the prefetch turned off, bit for bit, on every tick."""
    n = 6
    frames = _frames(n)
    schedule = [set(range(len(CAMS)))] * n
    a = _alone(frames, schedule, precision=G.PREC_F16)
    on, _, _ = _pooled(frames, schedule, graph=graph, launch=(64, 1, 64), precision=G.PREC_F16)
    off, _, _ = _pooled(frames, schedule, graph=graph, launch=(64, 1, 64), precision=G.PREC_F16,
                        prefetch=False)
    for key in a:
        assert np.array_equal(a[key], on[key]), key
        assert np.array_equal(off[key], on[key]), key
