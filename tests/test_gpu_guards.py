"""Out-of-bounds writes, checked without a sanitizer: every output the
kernels write (fused mask, per-stream masks, the opened mask; pooled cameras
too) sits inside a larger device buffer whose bytes before and after it are
filled with a canary pattern, at ragged sizes (W not a multiple of 32, one
row, one column, one pixel). After several ticks the canaries must be intact
and the outputs' padding bits zero."""
import numpy as np
import pytest

import paper_2110_14934_gb300 as G
from parity import scene_frames, to_dev

pytestmark = pytest.mark.gpu

GUARD = 4096          # bytes of canary on each side
CANARY = 0xA5

SHAPES = [(1, 1, 3), (1, 33, 5), (33, 1, 4), (45, 83, 3), (3, 64, 5), (7, 1000, 4)]


class Guarded:
    """A device int32 [rows, cols] tensor with canary bytes around it."""

    def __init__(self, rows, cols):
        import torch
        self.n = rows * cols * 4
        self.buf = torch.full((GUARD + self.n + GUARD,), CANARY, dtype=torch.uint8, device="cuda")
        self.t = self.buf[GUARD:GUARD + self.n].view(torch.int32).view(rows, cols)

    def intact(self) -> bool:
        b = self.buf.cpu().numpy()
        return bool((b[:GUARD] == CANARY).all() and (b[GUARD + self.n:] == CANARY).all())


def _padding_zero(words, W):
    """Bits of the last word of each row beyond column W are zero."""
    rem = W % 32
    if rem == 0:
        return True
    last = words[:, -1].view(np.uint32)
    return bool((last >> np.uint32(rem) == 0).all())


@pytest.mark.parametrize("prec", [G.PREC_F32, G.PREC_F16])
@pytest.mark.parametrize("morph", [False, True])
@pytest.mark.parametrize("H,W,M", SHAPES)
def test_outputs_stay_in_bounds(H, W, M, prec, morph):
    import torch
    rgb, depth, _ = scene_frames(H * 131 + W, H, W, 1, 0, 4)
    g = G.GMM(H, W, M, precision=prec, morph_open=morph)
    wpr = G.mask_words_per_row(W)
    outs = [Guarded(H, wpr) for _ in range(3)]
    for t in range(4):
        r, d = to_dev(rgb[t], depth[t])
        g.apply(r, d, outs[0].t, outs[1].t, outs[2].t)
    torch.cuda.synchronize()
    for o in outs:
        assert o.intact()
        assert _padding_zero(o.t.cpu().numpy(), W)


@pytest.mark.parametrize("prec", [G.PREC_F32, G.PREC_F16])
def test_pooled_outputs_stay_in_bounds(prec):
    import torch
    pool = G.Pool(precision=prec, max_cams=len(SHAPES))
    ids = [pool.admit(H, W, M, mode=(G.MODE_AUGMENTED if i % 3 == 2 else G.MODE_FUSION))
           for i, (H, W, M) in enumerate(SHAPES)]
    frames = [scene_frames(700 + i, H, W, 1, 0, 4) for i, (H, W, M) in enumerate(SHAPES)]
    outs = [[Guarded(H, G.mask_words_per_row(W)) for _ in range(3)] for (H, W, M) in SHAPES]
    keep = []
    for t in range(4):
        for i, (H, W, M) in enumerate(SHAPES):
            r, d = to_dev(frames[i][0][t], frames[i][1][t])
            keep.append((r, d))
            pool.submit(ids[i], r, d, outs[i][0].t, outs[i][1].t, outs[i][2].t)
        pool.tick()
    torch.cuda.synchronize()
    pool.close()
    for (H, W, M), o3 in zip(SHAPES, outs):
        for o in o3:
            assert o.intact(), (H, W, M)
            assert _padding_zero(o.t.cpu().numpy(), W), (H, W, M)
