/*
 * Host side of the seeded synthetic RGB-D scene (see synth_core.h): scene
 * construction from a seed and frame generation on the CPU.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "synth_core.h"

int synth_scene_size(void) { return (int)sizeof(synth_scene); }

/* Draw i of the scene-construction stream of a seed (disjoint from the
 * per-pixel counters, which never reach the top bit). */
static uint32_t draw(uint64_t seed, int i)
{
    return (uint32_t)(synth_mix(seed, (1ull << 63) | (uint64_t)i) >> 32);
}

static int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }
static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

/* kind 0: static gradient background, one 80x120 rectangle moving 4 px per
 *         frame, +40 illumination step at frame 50, noise sigma 3 (colour)
 *         and 5 mm (depth), 2% invalid depth.
 * kind 1: kind 0 plus 6 moving ellipses with cast shadows and a
 *         quasi-periodic region (amplitude 25, period 17.3 frames) on 10% of
 *         the pixels. */
int synth_scene_init(synth_scene *s, uint64_t seed, int H, int W, int kind)
{
    if (!s || H < 1 || W < 1 || kind < 0 || kind > 1)
        return -1;
    memset(s, 0, sizeof(*s));
    s->seed = seed;
    s->H = H;
    s->W = W;
    int i = 0;
    for (int k = 0; k < 3; k++) {
        s->bg_base[k] = 50 + (int32_t)(draw(seed, i++) % 80u);
        s->bg_gx[k] = -40 + (int32_t)(draw(seed, i++) % 81u);
        s->bg_gy[k] = -40 + (int32_t)(draw(seed, i++) % 81u);
    }
    s->d_base = 1500 + (int32_t)(draw(seed, i++) % 500u);
    s->d_gx = (int32_t)(draw(seed, i++) % 1000u);
    s->d_gy = (int32_t)(draw(seed, i++) % 1000u);

    s->rect_w = imax(1, imin(80, W / 2));
    s->rect_h = imax(1, imin(120, H / 2));
    s->rect_x0 = (int32_t)(draw(seed, i++) % (uint32_t)W);
    s->rect_y0 = (int32_t)(draw(seed, i++) % (uint32_t)(H - s->rect_h + 1));
    s->rect_speed = 4;
    for (int k = 0; k < 3; k++)
        s->rect_rgb[k] = (int32_t)(draw(seed, i++) % 256u);
    s->rect_depth = 800;

    s->illum_frame = 50;
    s->illum_delta = 40;
    /* sd of a sum of four uniforms on {0..65535}: sqrt(4 (65536^2 - 1) / 12) */
    const double sd = sqrt(4.0 * (65536.0 * 65536.0 - 1.0) / 12.0);
    s->noise_c_k = (int64_t)llround(3.0 / sd * 4294967296.0);
    s->noise_d_k = (int64_t)llround(5.0 / sd * 4294967296.0);
    s->invalid_per_10000 = 200;

    if (kind == 1) {
        s->n_ellipses = 6;
        for (int e = 0; e < 6; e++) {
            synth_ellipse *el = &s->ell[e];
            el->a = imax(1, W / 40 + (int32_t)(draw(seed, i++) % (uint32_t)(W / 20 + 1)));
            el->b = imax(1, H / 30 + (int32_t)(draw(seed, i++) % (uint32_t)(H / 15 + 1)));
            el->cx0 = (int32_t)(draw(seed, i++) % (uint32_t)W);
            el->cy0 = (int32_t)(draw(seed, i++) % (uint32_t)H);
            int32_t sgn = (draw(seed, i++) & 1u) ? 1 : -1;
            el->vx = sgn * (1 + (int32_t)(draw(seed, i++) % 6u));
            el->vy = (int32_t)(draw(seed, i++) % 7u) - 3;
            el->sx = el->a / 2 + 2;
            el->sy = el->b / 3 + 2;
            el->r = (int32_t)(draw(seed, i++) % 256u);
            el->g = (int32_t)(draw(seed, i++) % 256u);
            el->bl = (int32_t)(draw(seed, i++) % 256u);
            el->depth = 700 + (int32_t)(draw(seed, i++) % 700u);
        }
        s->periodic = 1;
        s->per_w = imax(1, W / 4);
        s->per_h = imax(1, (2 * H) / 5);
        s->per_x0 = (int32_t)(draw(seed, i++) % (uint32_t)(W - s->per_w + 1));
        s->per_y0 = (int32_t)(draw(seed, i++) % (uint32_t)(H - s->per_h + 1));
        s->per_num = 10240; /* 1024 / 17.3 = 10240 / 173 phase units per frame */
        s->per_den = 173;
        for (int k = 0; k < SYNTH_LUT; k++)
            s->lut[k] = (int8_t)lrint(25.0 * sin(2.0 * 3.14159265358979323846 * k / SYNTH_LUT));
    }
    return 0;
}

/* Rows y0 .. y0+rows-1 of frames f0 .. f0+nf-1 into caller buffers: rgb
 * [nf][rows][W][3], depth [nf][rows][W], gt [nf][rows][W] (gt may be NULL). */
int synth_rows_host(const synth_scene *s, int f0, int nf, int y0, int rows,
                    uint8_t *rgb, uint16_t *depth, uint8_t *gt)
{
    if (!s || !rgb || !depth || nf < 0 || f0 < 0 || y0 < 0 || rows < 0 ||
        y0 + rows > s->H)
        return -1;
    const int64_t N = (int64_t)rows * s->W;
    for (int f = 0; f < nf; f++) {
        for (int32_t r = 0; r < rows; r++) {
            for (int32_t x = 0; x < s->W; x++) {
                int64_t n = (int64_t)f * N + (int64_t)r * s->W + x;
                uint8_t g;
                synth_pixel(s, f0 + f, x, y0 + r, rgb + 3 * n, depth + n, &g);
                if (gt)
                    gt[n] = g;
            }
        }
    }
    return 0;
}

/* Whole frames f0 .. f0+nf-1: rgb [nf][H][W][3], depth [nf][H][W], gt
 * [nf][H][W] (gt may be NULL). */
int synth_frames_host(const synth_scene *s, int f0, int nf, uint8_t *rgb,
                      uint16_t *depth, uint8_t *gt)
{
    if (!s)
        return -1;
    return synth_rows_host(s, f0, nf, 0, s->H, rgb, depth, gt);
}
