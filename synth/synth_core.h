/*
 * Seeded synthetic RGB-D scene, integer arithmetic only, so that the host
 * build (gcc) and the device build (nvcc) produce bit-identical frames.
 *
 * This module is the input generator shared by the oracle tests and the CUDA
 * path's tests and benchmark. It holds none of the background-subtraction
 * arithmetic: it only draws frames and their ground-truth foreground masks.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), evaluated at a counter:
 * the n-th output of a generator seeded with s is mix(s + n * gamma).
 *
 * Scene (stand-in for the paper's Kinect captures, which are not available):
 *   colour  smooth per-channel linear gradient, optional quasi-periodic region
 *           (sinusoidal intensity, non-integer period), moving foreground
 *           objects, cast shadows (colour x 0.7, depth unchanged), a global
 *           illumination step, then additive noise and clamping to [0, 255];
 *   depth   tilted plane in millimetres, objects at their own depth, additive
 *           noise, and a hashed fraction of invalid (zero) readings;
 *   noise   approximately Gaussian: Irwin-Hall sum of four 16-bit uniforms,
 *           rescaled to the requested standard deviation in fixed point.
 */
#ifndef SYNTH_CORE_H
#define SYNTH_CORE_H

#include <stdint.h>

#if defined(__CUDACC__)
#define SYNTH_HD __host__ __device__ __forceinline__
#else
#define SYNTH_HD static inline
#endif

#define SYNTH_MAX_ELLIPSES 8
#define SYNTH_LUT 1024

typedef struct synth_ellipse {
    int32_t cx0, cy0, vx, vy; /* centre at frame 0, velocity in px/frame */
    int32_t a, b;             /* semi-axes (x, y) */
    int32_t sx, sy;           /* shadow offset */
    int32_t r, g, bl, depth;  /* colour and depth (mm) of the object */
} synth_ellipse;

typedef struct synth_scene {
    uint64_t seed;
    int32_t H, W;
    /* background */
    int32_t bg_base[3], bg_gx[3], bg_gy[3];
    int32_t d_base, d_gx, d_gy;
    /* rectangle */
    int32_t rect_x0, rect_y0, rect_w, rect_h, rect_speed;
    int32_t rect_rgb[3], rect_depth;
    /* ellipses */
    int32_t n_ellipses;
    synth_ellipse ell[SYNTH_MAX_ELLIPSES];
    /* quasi-periodic region: phase index = (t * per_num) / per_den + (5x + 3y) */
    int32_t periodic, per_x0, per_y0, per_w, per_h, per_num, per_den;
    int8_t lut[SYNTH_LUT]; /* round(amplitude * sin(2 pi i / 1024)) */
    /* illumination step and noise */
    int32_t illum_frame, illum_delta;
    int64_t noise_c_k, noise_d_k; /* sigma in Q32 per Irwin-Hall unit */
    int32_t invalid_per_10000;
} synth_scene;

/* SplitMix64 output at counter n for seed s. */
SYNTH_HD uint64_t synth_mix(uint64_t s, uint64_t n)
{
    uint64_t z = s + (n + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Counter of the draw for (frame, pixel, channel); channel < 8. */
SYNTH_HD uint64_t synth_counter(int frame, int64_t pixel, int ch)
{
    return ((((uint64_t)(uint32_t)frame) << 32 | (uint64_t)pixel) << 3) | (uint64_t)ch;
}

/* floor(v / 2^sh) for signed v, without relying on signed shifts. */
SYNTH_HD int64_t synth_floor_shift(int64_t v, int sh)
{
    if (v >= 0)
        return (int64_t)((uint64_t)v >> sh);
    return -(int64_t)(((uint64_t)(-v) + ((1ull << sh) - 1u)) >> sh);
}

/* Approximately N(0, sigma^2) integer noise from one 64-bit draw: the four
 * 16-bit fields are summed (Irwin-Hall, n = 4) and centred, then scaled by
 * k = sigma / sd(sum) in Q32 and rounded to the nearest integer. */
SYNTH_HD int32_t synth_noise(uint64_t h, int64_t k)
{
    int64_t s = (int64_t)(h & 0xFFFF) + (int64_t)((h >> 16) & 0xFFFF) +
                (int64_t)((h >> 32) & 0xFFFF) + (int64_t)((h >> 48) & 0xFFFF);
    int64_t centred2 = 2 * s - 4 * 65535; /* 2 * (s - mean) */
    int64_t q = centred2 * k;             /* |q| < 2^18 * 2^23 */
    return (int32_t)synth_floor_shift(q + (1ll << 32), 33);
}

SYNTH_HD int32_t synth_mod(int32_t a, int32_t m)
{
    int32_t r = a % m;
    return r < 0 ? r + m : r;
}

SYNTH_HD int32_t synth_clamp(int32_t v, int32_t lo, int32_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

SYNTH_HD int synth_in_ellipse(int32_t x, int32_t y, int32_t cx, int32_t cy,
                              int32_t a, int32_t b)
{
    int64_t dx = x - cx, dy = y - cy;
    int64_t aa = (int64_t)a * a, bb = (int64_t)b * b;
    return dx * dx * bb + dy * dy * aa <= aa * bb;
}

/* One pixel of frame t: colour (3 bytes), depth (mm, 0 = invalid) and the
 * ground-truth foreground bit (1 on a moving object). */
SYNTH_HD void synth_pixel(const synth_scene *s, int t, int32_t x, int32_t y,
                          uint8_t *rgb, uint16_t *depth, uint8_t *gt)
{
    const int32_t H = s->H, W = s->W;
    const int64_t pix = (int64_t)y * W + x;
    int32_t c[3], d;
    for (int k = 0; k < 3; k++)
        c[k] = s->bg_base[k] + (s->bg_gx[k] * x) / W + (s->bg_gy[k] * y) / H;
    d = s->d_base + (s->d_gx * x) / W + (s->d_gy * y) / H;

    if (s->periodic && x >= s->per_x0 && x < s->per_x0 + s->per_w &&
        y >= s->per_y0 && y < s->per_y0 + s->per_h) {
        int32_t ph = (int32_t)(((int64_t)t * s->per_num) / s->per_den) + 5 * x + 3 * y;
        int32_t dv = s->lut[ph & (SYNTH_LUT - 1)];
        for (int k = 0; k < 3; k++)
            c[k] += dv;
    }

    int obj = 0, shadow = 0;
    int32_t oc[3] = {0, 0, 0}, od = 0;
    /* rectangle moving right and wrapping */
    {
        int32_t xs = synth_mod(s->rect_x0 + s->rect_speed * t, W);
        int32_t rx = synth_mod(x - xs, W);
        if (rx < s->rect_w && y >= s->rect_y0 && y < s->rect_y0 + s->rect_h) {
            obj = 1;
            oc[0] = s->rect_rgb[0]; oc[1] = s->rect_rgb[1]; oc[2] = s->rect_rgb[2];
            od = s->rect_depth;
        }
    }
    for (int e = 0; e < s->n_ellipses; e++) {
        const synth_ellipse *el = &s->ell[e];
        int32_t cx = synth_mod(el->cx0 + el->vx * t, W);
        int32_t cy = synth_mod(el->cy0 + el->vy * t, H);
        if (synth_in_ellipse(x, y, cx, cy, el->a, el->b)) {
            obj = 1;
            oc[0] = el->r; oc[1] = el->g; oc[2] = el->bl;
            od = el->depth;
        } else if (synth_in_ellipse(x, y, cx + el->sx, cy + el->sy, el->a, el->b)) {
            shadow = 1;
        }
    }
    if (obj) {
        c[0] = oc[0]; c[1] = oc[1]; c[2] = oc[2];
        d = od;
    } else if (shadow) {
        for (int k = 0; k < 3; k++)
            c[k] = (c[k] * 7) / 10;
    }
    if (s->illum_frame >= 0 && t >= s->illum_frame)
        for (int k = 0; k < 3; k++)
            c[k] += s->illum_delta;

    for (int k = 0; k < 3; k++) {
        uint64_t h = synth_mix(s->seed, synth_counter(t, pix, k));
        rgb[k] = (uint8_t)synth_clamp(c[k] + synth_noise(h, s->noise_c_k), 0, 255);
    }
    {
        uint64_t h = synth_mix(s->seed, synth_counter(t, pix, 3));
        d = synth_clamp(d + synth_noise(h, s->noise_d_k), 1, 65535);
        uint64_t hv = synth_mix(s->seed, synth_counter(t, pix, 4));
        if ((int32_t)(hv % 10000u) < s->invalid_per_10000)
            d = 0;
    }
    *depth = (uint16_t)d;
    *gt = (uint8_t)obj;
}

#endif /* SYNTH_CORE_H */
