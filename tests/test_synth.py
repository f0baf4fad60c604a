"""The seeded synthetic RGB-D generator (host build): determinism, the
scene statistics the workloads ask for, and seed independence."""
import numpy as np
import pytest

import synth


def test_deterministic_and_seeded():
    s = synth.scene(5, 48, 64, 0)
    a = synth.frames_host(s, 0, 3)
    b = synth.frames_host(synth.scene(5, 48, 64, 0), 0, 3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c = synth.frames_host(synth.scene(6, 48, 64, 0), 0, 3)
    assert not np.array_equal(a[0], c[0])
    # frames are addressable: generating frames 1..2 alone gives the same bytes
    d = synth.frames_host(s, 1, 2)
    assert np.array_equal(d[0], a[0][1:]) and np.array_equal(d[1], a[1][1:])


def test_scene0_statistics():
    s = synth.scene(1, 480, 640, 0)
    rgb, depth, gt = synth.frames_host(s, 48, 4)
    # one 80 x 120 rectangle of ground truth per frame, moving 4 px per frame
    assert gt.reshape(4, -1).sum(axis=1).tolist() == [9600] * 4
    xs = [np.nonzero(gt[f].any(axis=0))[0] for f in range(4)]
    assert all(len(x) == 80 for x in xs)
    bg = (gt[0] == 0) & (gt[1] == 0)
    dc = (rgb[0].astype(int) - rgb[1].astype(int))[bg]
    assert abs(dc.std() / np.sqrt(2) - 3.0) < 0.1     # colour noise sigma 3
    valid = (depth[0] > 0) & (depth[1] > 0) & bg
    dd = depth[0].astype(int)[valid] - depth[1].astype(int)[valid]
    assert abs(dd.std() / np.sqrt(2) - 5.0) < 0.15    # depth noise sigma 5 mm
    assert abs((depth == 0).mean() - 0.02) < 0.003   # 2% invalid depth
    bgd = depth[0][(gt[0] == 0) & (depth[0] > 0)]
    assert bgd.min() >= 1450 and bgd.max() <= 4050     # plane at 1500-4000 mm
    assert np.all(depth[0][(gt[0] == 1) & (depth[0] > 0)] < 900)  # rectangle at 800 mm
    # illumination step of +40 at frame 50
    before = synth.frames_host(s, 49, 1)[0][0].astype(float)
    after = synth.frames_host(s, 50, 1)[0][0].astype(float)
    m = (synth.frames_host(s, 49, 1)[2][0] == 0) & (synth.frames_host(s, 50, 1)[2][0] == 0)
    m &= before.max(axis=2) < 200
    assert abs((after - before)[m].mean() - 40.0) < 0.5


def test_scene1_structure():
    s = synth.scene(9, 270, 480, 1)
    assert s.n_ellipses == 6 and s.periodic == 1
    assert abs(s.per_w * s.per_h / (270 * 480) - 0.10) < 0.01  # periodic region ~10%
    rgb, depth, gt = synth.frames_host(s, 0, 2)
    assert 0 < gt.mean() < 0.5
    lut = np.array(s.lut[:], dtype=int)
    assert lut.max() == 25 and lut.min() == -25


@pytest.mark.parametrize("H,W", [(1, 1), (1, 33), (7, 1), (3, 5)])
def test_tiny_shapes(H, W):
    for kind in (0, 1):
        rgb, depth, gt = synth.frames_host(synth.scene(2, H, W, kind), 0, 2)
        assert rgb.shape == (2, H, W, 3) and depth.shape == (2, H, W)


def test_row_band_matches_whole_frames():
    s = synth.scene(4, 40, 50, 1)
    rgb, dep, gt = synth.frames_host(s, 3, 2)
    r2, d2, g2 = synth.rows_host(s, 3, 2, 11, 7)
    assert np.array_equal(r2, rgb[:, 11:18]) and np.array_equal(d2, dep[:, 11:18])
    assert np.array_equal(g2, gt[:, 11:18])
    with pytest.raises(ValueError):
        synth.rows_host(s, 0, 1, 35, 6)
