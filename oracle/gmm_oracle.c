/*
 * FP64 oracle for "GPU based GMM segmentation of Kinect data" (Amamra, Mouats,
 * Aouf): per-pixel Gaussian-mixture background subtraction run separately on
 * the colour image and on the depth map (§III.A, §III.B), followed by the
 * counter-based fusion of the two binary foregrounds (List 1, §III.C).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this file. The CUDA library never links,
 * includes or calls it, and nothing here includes or calls the CUDA library.
 * It is deliberately plain and slow: one pixel at a time, double precision,
 * every step in the order the method states it, no blocking or fusion.
 *
 * The paper names the model (a mixture of M Gaussians per pixel, 3 <= M <= 5,
 * weights positive and summing to one, §III.A) and its steps (match against
 * the components from the most to the least weighted, foreground when nothing
 * matches, then update) but prints no update equations; it points to
 * Stauffer and Grimson's mixture for them (§II). The equations below are that
 * mixture written out, with these readings of what the paper leaves open:
 *   - learning rate of the matched component rho = alpha (constant);
 *   - isotropic colour variance: one scalar v per component that tracks the
 *     squared distance summed over the three channels; the match test uses the
 *     same squared distance;
 *   - components are stored in rank order (descending w / sqrt(v), stable:
 *     equal keys keep their stored order) and tested in that order, the first
 *     match wins;
 *   - on a miss every weight decays, the last-ranked component is replaced by
 *     {mu = x, v = init_var, w = init_w}, and the weights are renormalised;
 *   - weights are renormalised every tick;
 *   - background set B = the shortest rank prefix whose summed weight exceeds
 *     T (strictly); a matched pixel is background iff its component's rank
 *     after the update is below B; a miss is foreground;
 *   - variance floor v_min (per stream);
 *   - first frame: every component takes the sample, v = init_var, w = 1/M,
 *     output foreground 0; the depth model of a pixel starts at the pixel's
 *     first valid (non-zero) depth instead;
 *   - a zero depth reading is invalid: the depth model is left untouched and
 *     the depth foreground copies the colour one;
 *   - fusion follows List 1 literally, with both label and counter starting
 *     at zero.
 * Options (bits of the stream's flags parameter), each another reading:
 *   - RHO_ETA: the matched component's mean and variance move with
 *     rho = alpha * eta(x | mu, sigma), eta the isotropic Gaussian density at
 *     the sample with the component's parameters before the update
 *     (Stauffer-Grimson's second learning rate), capped at 1;
 *   - VAR_PER_CHANNEL: v tracks the squared distance divided by the number of
 *     channels (the per-channel variance sigma^2), so the match test
 *     d^2 < k^2 v is the Mahalanobis test with covariance sigma^2 I; without
 *     it v tracks the summed squared distance and sigma^2 = v / D.
 * The augmentation alternative of §III.B (one mixture over R, G, B and the
 * depth brought to the byte range) is oracle_tick_augmented below.
 *
 * Near-threshold report. For each stream step the oracle also reports, in its
 * own arithmetic, whether any decision sat within a relative distance `eps` of
 * its threshold: a tested squared distance against k^2 v (bit 0), a rank-prefix
 * weight sum against T (bit 1), or the sort keys of two components with
 * different parameters against each other (bit 2). A lower-precision implementation may legitimately decide those
 * cases the other way. It can also report the smallest of those relative
 * distances itself (the step's margin), and the decisions taken (matched
 * component, B, rank of the matched or replaced component), so that a
 * comparison of two trajectories can tell a decision that flipped near its
 * threshold from one that flipped far from it.
 */

#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORACLE_MAX_M 5

enum { NEAR_MATCH = 1, NEAR_T = 2, NEAR_KEY = 4 };
enum { FLAG_RHO_ETA = 1, FLAG_VAR_PER_CHANNEL = 2 };
static const double kPi = 3.14159265358979323846;

/* Stream parameters, in this order (a plain double array keeps the ABI
 * trivial): alpha, k, T, init_var, init_w, v_min, eps, flags. */
enum { P_ALPHA, P_K, P_T, P_INIT_VAR, P_INIT_W, P_VMIN, P_EPS, P_FLAGS, P_COUNT };

int oracle_param_count(void) { return P_COUNT; }

/* Initialisation from the first sample: every component sits on x with the
 * initial variance and equal weight 1/M (so the weights are positive and sum
 * to one from the start, §III.A). w[M], mu[M*D] component-major, v[M]. */
void oracle_stream_init(int M, int D, double init_var, double *w, double *mu,
                        double *v, const double *x)
{
    for (int i = 0; i < M; i++) {
        w[i] = 1.0 / (double)M;
        for (int c = 0; c < D; c++)
            mu[i * D + c] = x[c];
        v[i] = init_var;
    }
}

/* Ordering key of a component: weight over standard deviation, so that
 * heavy, narrow components rank first (§III.A, "based on the mean and the
 * variance"; Stauffer-Grimson's w/sigma). */
static double rank_key(double w, double v) { return w / sqrt(v); }

/* Stable descending sort of the M components by rank_key. perm[r] receives
 * the stored index that lands at rank r. Plain insertion sort: an element
 * moves left only past strictly smaller keys, so equal keys keep their
 * stored order. */
void oracle_rank_order(int M, const double *w, const double *v, int *perm)
{
    double key[ORACLE_MAX_M];
    for (int i = 0; i < M; i++) {
        perm[i] = i;
        key[i] = rank_key(w[i], v[i]);
    }
    for (int i = 1; i < M; i++) {
        int p = perm[i];
        int r = i;
        while (r > 0 && key[perm[r - 1]] < key[p]) {
            perm[r] = perm[r - 1];
            r--;
        }
        perm[r] = p;
    }
}

/* Size of the background set: the first b (1-based) for which the summed
 * weight of the b best-ranked components exceeds T (§III.A, "determining the
 * Gaussian that corresponds to the background"). If rounding keeps every
 * prefix at or below T, all M components are background. */
int oracle_background_count(int M, const double *w_ranked, double T)
{
    double s = 0.0;
    for (int b = 0; b < M; b++) {
        s += w_ranked[b];
        if (s > T)
            return b + 1;
    }
    return M;
}

/* One tick of one stream at one pixel. The state (w, mu, v) is in rank order
 * on entry and on exit. Returns the stream's foreground bit.
 * info[0]: stored index that matched before the update, -1 on a miss;
 * info[1]: B; info[2]: rank of the matched (or replaced) component after the
 * update; info[3]: near-threshold bits. margin (may be NULL): the smallest
 * relative distance of a decision to its threshold, over the same decisions
 * the near bits look at: |d^2 - k^2 v| / (k^2 v) for each tested component,
 * |k_a - k_b| / max(k_a, k_b) for each pair of components with different
 * parameters (w, v), and
 * |prefix sum - T| / T for each rank prefix. */
int oracle_stream_step(int M, int D, const double *prm, double *w, double *mu,
                       double *v, const double *x, int *info, double *margin)
{
    const double alpha = prm[P_ALPHA], k = prm[P_K], T = prm[P_T];
    const double init_var = prm[P_INIT_VAR], init_w = prm[P_INIT_W];
    const double v_min = prm[P_VMIN], eps = prm[P_EPS];
    const int flags = (int)prm[P_FLAGS];
    int near = 0;
    double mrg = INFINITY;

    /* 1. Match: distance of the sample to each mean, tested from the best
     *    ranked component down; the first one within k standard deviations
     *    (squared: d^2 < k^2 v, strict) matches (§III.A). */
    int j = -1;
    for (int i = 0; i < M && j < 0; i++) {
        double d2 = 0.0;
        for (int c = 0; c < D; c++) {
            double diff = x[c] - mu[i * D + c];
            d2 += diff * diff;
        }
        double lim = k * k * v[i];
        if (fabs(d2 - lim) <= eps * lim)
            near |= NEAR_MATCH;
        mrg = fmin(mrg, fabs(d2 - lim) / lim);
        if (d2 < lim)
            j = i;
    }
    const int matched = (j >= 0);
    info[0] = j;

    /* 2. Weights: every weight decays by (1 - alpha); the matched one gains
     *    alpha. On a miss the last-ranked component is replaced by a new one
     *    on the sample. Then the weights are renormalised to sum to one. */
    for (int i = 0; i < M; i++)
        w[i] = (1.0 - alpha) * w[i];
    if (matched) {
        w[j] = w[j] + alpha;
    } else {
        j = M - 1;
        w[j] = init_w;
        for (int c = 0; c < D; c++)
            mu[j * D + c] = x[c];
        v[j] = init_var;
    }
    double s = 0.0;
    for (int i = 0; i < M; i++)
        s += w[i];
    for (int i = 0; i < M; i++)
        w[i] = w[i] / s;

    /* 3. Matched component: mean and variance move toward the sample with
     *    rate rho (alpha, or alpha * eta with RHO_ETA); the variance uses the
     *    updated mean. */
    if (matched) {
        double rho = alpha;
        if (flags & FLAG_RHO_ETA) {
            const double s2 = (flags & FLAG_VAR_PER_CHANNEL) ? v[j] : v[j] / D;
            double d2 = 0.0;
            for (int c = 0; c < D; c++) {
                double diff = x[c] - mu[j * D + c];
                d2 += diff * diff;
            }
            const double eta = pow(2.0 * kPi * s2, -0.5 * D) * exp(-d2 / (2.0 * s2));
            rho = alpha * eta;
            if (rho > 1.0)
                rho = 1.0;
        }
        for (int c = 0; c < D; c++)
            mu[j * D + c] = (1.0 - rho) * mu[j * D + c] + rho * x[c];
        double d2 = 0.0;
        for (int c = 0; c < D; c++) {
            double diff = x[c] - mu[j * D + c];
            d2 += diff * diff;
        }
        if (flags & FLAG_VAR_PER_CHANNEL)
            d2 = d2 / D;
        double vn = (1.0 - rho) * v[j] + rho * d2;
        v[j] = vn < v_min ? v_min : vn;
    }

    /* 4. Order: stable descending sort by w / sqrt(v). */
    int perm[ORACLE_MAX_M];
    oracle_rank_order(M, w, v, perm);
    /* Near keys: two components with different parameters whose keys are
     * within eps, equal ones included (an exact tie between different w and
     * v, such as w' = 1.1 w with v' = 1.21 v, holds only in exact arithmetic;
     * rounding may break it either way). Two components with the same w and
     * v have the same key in any arithmetic: a tie the stable order settles. */
    for (int a = 0; a < M; a++) {
        for (int b = a + 1; b < M; b++) {
            double ka = rank_key(w[a], v[a]), kb = rank_key(w[b], v[b]);
            const int twins = (w[a] == w[b] && v[a] == v[b]);
            if (!twins && fabs(ka - kb) <= eps * fmax(ka, kb))
                near |= NEAR_KEY;
            if (!twins)
                mrg = fmin(mrg, fabs(ka - kb) / fmax(ka, kb));
        }
    }
    double tw[ORACLE_MAX_M], tmu[ORACLE_MAX_M * 4], tv[ORACLE_MAX_M];
    int rank_j = -1;
    for (int r = 0; r < M; r++) {
        int p = perm[r];
        tw[r] = w[p];
        tv[r] = v[p];
        for (int c = 0; c < D; c++)
            tmu[r * D + c] = mu[p * D + c];
        if (p == j)
            rank_j = r;
    }
    memcpy(w, tw, sizeof(double) * (size_t)M);
    memcpy(v, tv, sizeof(double) * (size_t)M);
    memcpy(mu, tmu, sizeof(double) * (size_t)(M * D));

    /* 5. Background set. */
    int B = oracle_background_count(M, w, T);
    double acc = 0.0;
    for (int b = 0; b < M; b++) {
        acc += w[b];
        if (fabs(acc - T) <= eps * T)
            near |= NEAR_T;
        mrg = fmin(mrg, fabs(acc - T) / T);
    }

    /* 6. Foreground: nothing matched, or the matched component is not in
     *    the background set. */
    int fg = (!matched) || (rank_j >= B);
    info[1] = B;
    info[2] = rank_j;
    info[3] = near;
    if (margin)
        *margin = mrg;
    return fg;
}

/* List 1 (§III.C), literally: agreement sets the fused label and clears the
 * counter; on disagreement a counter at +3 hands the label to the colour
 * foreground, at -3 to the depth foreground (both clear it), and otherwise the
 * counter moves up when the current label equals the colour answer and down
 * when it does not. */
void oracle_fuse(int f_rgb, int f_d, int *F, int *cpt)
{
    if (f_rgb == f_d) {
        *F = f_d;
        *cpt = 0;
    } else {
        if (*cpt == 3) {
            *F = f_rgb;
            *cpt = 0;
        } else if (*cpt == -3) {
            *F = f_d;
            *cpt = 0;
        } else if (*F == f_rgb) {
            *cpt = *cpt + 1;
        } else {
            *cpt = *cpt - 1;
        }
    }
}

/* One tick over an H x W image. Pixel n = y * W + x.
 * rgb: interleaved 8-bit, 3 per pixel; depth: 16-bit millimetres, 0 = invalid.
 * State, pixel-major, rank order inside each pixel:
 *   wc[N*M], muc[N*M*3], vc[N*M]  colour;  wd[N*M], mud[N*M], vd[N*M]  depth;
 *   F[N] fused label, cpt[N] List-1 counter, dinit[N] depth model started.
 * first != 0 starts every model from this frame.
 * Outputs (each may be NULL): fg_rgb[N], fg_d[N], fused[N], near[N]
 * (near: colour bits 0-2, depth bits 4-6); margin_c[N], margin_d[N] (the
 * stream step's margin, INFINITY where the stream took no step: first frame,
 * invalid depth, depth model starting); dec[N*6] the decisions, per pixel
 * {colour: matched stored index or -1, B, rank of the matched or replaced
 * component; depth: the same}, -2 where the stream took no step. */
void oracle_tick_ex(int H, int W, int M, const double *prm_c, const double *prm_d,
                    int first, double *wc, double *muc, double *vc, double *wd,
                    double *mud, double *vd, int8_t *F, int8_t *cpt,
                    uint8_t *dinit, const uint8_t *rgb, const uint16_t *depth,
                    uint8_t *fg_rgb, uint8_t *fg_d, uint8_t *fused, uint8_t *near,
                    double *margin_c, double *margin_d, int8_t *dec)
{
    const long N = (long)H * (long)W;
    for (long n = 0; n < N; n++) {
        double xc[3] = {(double)rgb[3 * n], (double)rgb[3 * n + 1],
                        (double)rgb[3 * n + 2]};
        double xd = (double)depth[n];
        double *w1 = wc + n * M, *m1 = muc + n * M * 3, *v1 = vc + n * M;
        double *w2 = wd + n * M, *m2 = mud + n * M, *v2 = vd + n * M;
        int info[4];
        int dc[3] = {-2, -2, -2}, dd[3] = {-2, -2, -2};
        double mc = INFINITY, md = INFINITY;
        int nbits = 0;
        int fc, fdp;

        if (first) {
            F[n] = 0;
            cpt[n] = 0;
            dinit[n] = 0;
            oracle_stream_init(M, 3, prm_c[P_INIT_VAR], w1, m1, v1, xc);
            fc = 0;
        } else {
            fc = oracle_stream_step(M, 3, prm_c, w1, m1, v1, xc, info, &mc);
            nbits |= info[3];
            dc[0] = info[0];
            dc[1] = info[1];
            dc[2] = info[2];
        }

        if (depth[n] == 0) {
            fdp = fc;
        } else if (!dinit[n]) {
            oracle_stream_init(M, 1, prm_d[P_INIT_VAR], w2, m2, v2, &xd);
            dinit[n] = 1;
            fdp = 0;
        } else {
            fdp = oracle_stream_step(M, 1, prm_d, w2, m2, v2, &xd, info, &md);
            nbits |= info[3] << 4;
            dd[0] = info[0];
            dd[1] = info[1];
            dd[2] = info[2];
        }

        int Fi = F[n], ci = cpt[n];
        oracle_fuse(fc, fdp, &Fi, &ci);
        F[n] = (int8_t)Fi;
        cpt[n] = (int8_t)ci;

        if (fg_rgb)
            fg_rgb[n] = (uint8_t)fc;
        if (fg_d)
            fg_d[n] = (uint8_t)fdp;
        if (fused)
            fused[n] = (uint8_t)Fi;
        if (near)
            near[n] = (uint8_t)nbits;
        if (margin_c)
            margin_c[n] = mc;
        if (margin_d)
            margin_d[n] = md;
        if (dec)
            for (int k = 0; k < 3; k++) {
                dec[6 * n + k] = (int8_t)dc[k];
                dec[6 * n + 3 + k] = (int8_t)dd[k];
            }
    }
}

/* oracle_tick_ex without the margins and decisions. */
void oracle_tick(int H, int W, int M, const double *prm_c, const double *prm_d,
                 int first, double *wc, double *muc, double *vc, double *wd,
                 double *mud, double *vd, int8_t *F, int8_t *cpt,
                 uint8_t *dinit, const uint8_t *rgb, const uint16_t *depth,
                 uint8_t *fg_rgb, uint8_t *fg_d, uint8_t *fused, uint8_t *near)
{
    oracle_tick_ex(H, W, M, prm_c, prm_d, first, wc, muc, vc, wd, mud, vd, F, cpt, dinit,
                   rgb, depth, fg_rgb, fg_d, fused, near, NULL, NULL, NULL);
}

/* The augmentation alternative (§III.B, Fig. 2): one mixture over four
 * channels, R, G, B and the depth reading times depth_scale (bringing
 * millimetres to the byte range of the colour channels). A zero depth reading
 * takes the depth mean of the best-ranked component (the value the model
 * expects, so the fourth channel neither adds distance nor moves), or 0 on
 * the first frame. State pixel-major: w[N*M], mu[N*M*4], v[N*M]. Output: the
 * foreground bit per pixel (no fusion); near as in oracle_tick. */
void oracle_tick_augmented(int H, int W, int M, const double *prm, double depth_scale,
                           int first, double *w, double *mu, double *v,
                           const uint8_t *rgb, const uint16_t *depth, uint8_t *fg,
                           uint8_t *near)
{
    const long N = (long)H * (long)W;
    for (long n = 0; n < N; n++) {
        double *wn = w + n * M, *mn = mu + n * M * 4, *vn = v + n * M;
        double x[4] = {(double)rgb[3 * n], (double)rgb[3 * n + 1], (double)rgb[3 * n + 2],
                       depth_scale * (double)depth[n]};
        if (depth[n] == 0)
            x[3] = first ? 0.0 : mn[3];
        int f = 0, nb = 0;
        if (first) {
            oracle_stream_init(M, 4, prm[P_INIT_VAR], wn, mn, vn, x);
        } else {
            int info[4];
            f = oracle_stream_step(M, 4, prm, wn, mn, vn, x, info, NULL);
            nb = info[3];
        }
        if (fg)
            fg[n] = (uint8_t)f;
        if (near)
            near[n] = (uint8_t)nb;
    }
}

/* 3x3 morphological opening of a binary image: erosion then dilation with a
 * 3x3 square, pixels outside the image count as 0. Not part of the paper: an
 * optional clean-up of the fused mask that is never fed back into the state. */
void oracle_morph_open3(int H, int W, const uint8_t *in, uint8_t *tmp,
                        uint8_t *out)
{
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int all = 1;
            for (int dy = -1; dy <= 1; dy++) {
                for (int dx = -1; dx <= 1; dx++) {
                    int yy = y + dy, xx = x + dx;
                    int val = 0;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                        val = in[(long)yy * W + xx] != 0;
                    if (!val)
                        all = 0;
                }
            }
            tmp[(long)y * W + x] = (uint8_t)all;
        }
    }
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int any = 0;
            for (int dy = -1; dy <= 1; dy++) {
                for (int dx = -1; dx <= 1; dx++) {
                    int yy = y + dy, xx = x + dx;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W &&
                        tmp[(long)yy * W + xx])
                        any = 1;
                }
            }
            out[(long)y * W + x] = (uint8_t)any;
        }
    }
}
