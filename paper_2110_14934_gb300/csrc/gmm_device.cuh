// Per-pixel device code shared by the single-camera tick kernel and the
// multi-camera persistent kernel: state loads/stores for both storage
// precisions, one mixture step (match, update or replace, re-rank,
// background test), List-1 fusion, and the bit-packed mask write.
//
// State layout in device memory (one camera). Pixels are numbered in padded
// row-major order p = row * w_pad + x (rows padded to a multiple of 32 pixels,
// so the 32 pixels of a warp map to one mask word) and grouped into tiles of
// kTile = 256 consecutive pixels. Each tile stores its M*8 planes
// contiguously, component-major: plane 8*i + field (fields w_c, mu_r, mu_g,
// mu_b, v_c, w_d, mu_d, v_d; i the rank), kTile elements each. Element
// (plane k, pixel p) sits at ((p / kTile) * 8M + k) * kTile + p % kTile.
// A warp reads 32 consecutive elements of a plane (one fully used 128-byte
// line in FP32); the plane offsets of a pixel are compile-time constants
// from one base address; and a tile's whole state is one contiguous block
// that a single bulk copy moves. The List-1 byte of a pixel lives in a
// separate byte array indexed by p (n_tiles * kTile bytes).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gmmdev {

constexpr int kFields = 8;
constexpr int kTile = 256; // pixels per state tile
enum { F_WC = 0, F_MUR, F_MUG, F_MUB, F_VC, F_WD, F_MUD, F_VD };
constexpr uint32_t kDepthStarted = 16u;
constexpr int kStageInputs = 1;   // CamView.flags: frame bytes staged with the state
constexpr int kModeAugmented = 2; // CamView.flags: one 4-channel mixture (R, G, B, s*depth)
constexpr uint32_t kRhoEta = 1u;        // StreamPrm.flags: rho = alpha * eta(x | mu, sigma)
constexpr uint32_t kVarPerChannel = 2u; // StreamPrm.flags: v is the per-channel variance

struct StreamPrm {
    float alpha, oma, k2, T, init_var, init_w, v_min;
    uint32_t flags; // kRhoEta | kVarPerChannel
};

// Learning rate of the matched component: alpha, or with kRhoEta
// alpha * N(x; mu, sigma^2 I) (Stauffer-Grimson's rho) from the distance d2
// and variance v before the update, sigma^2 = v (kVarPerChannel) or v / D,
// capped at 1. Returns rho and sets orho = 1 - rho (oma exactly by default).
template <int D>
__device__ __forceinline__ float match_rate(const StreamPrm &p, float d2, float v, float &orho) {
    if (!(p.flags & kRhoEta)) {
        orho = p.oma;
        return p.alpha;
    }
    const float s2 = (p.flags & kVarPerChannel) ? v : v / (float)D;
    const float base = 6.28318530717958647692f * s2;
    float norm;
    if (D == 1)
        norm = 1.0f / sqrtf(base);
    else if (D == 3)
        norm = 1.0f / (base * sqrtf(base));
    else if (D == 4)
        norm = 1.0f / (base * base);
    else
        norm = powf(base, -0.5f * (float)D);
    const float rho = fminf(p.alpha * norm * expf(-d2 / (2.0f * s2)), 1.0f);
    orho = 1.0f - rho;
    return rho;
}

// Squared distance that feeds the variance: per channel with kVarPerChannel.
template <int D>
__device__ __forceinline__ float var_sample(const StreamPrm &p, float d2) {
    return (p.flags & kVarPerChannel) ? d2 / (float)D : d2;
}

// Everything one tick of one camera needs; passed by value to the
// single-camera kernel, read from a device table by the pooled kernel.
struct CamView {
    void *planes;          // n_tiles tiles of M*8 planes of kTile elements
    uint8_t *fusion;       // n_tiles*kTile List-1 bytes, indexed by padded pixel
    const uint8_t *rgb;    // H*W*3, interleaved
    const uint16_t *depth; // H*W, millimetres, 0 = invalid
    uint32_t *mask;        // H*wpr words: fused foreground
    uint32_t *fg_rgb;      // optional colour foreground words (may be null)
    uint32_t *fg_d;        // optional depth foreground words (may be null)
    int64_t n_tiles;       // state tiles: ceil(n_pad / kTile)
    int64_t n_pad;         // H*w_pad (< 2^30)
    int H, W, w_pad, wpr;  // wpr = words per mask row = w_pad / 32
    int M, prec, first, flags; // flags: kStageInputs (staged launcher), kModeAugmented
    uint32_t wpr_mul, wpr_shift; // n / wpr == umulhi(n, wpr_mul) >> wpr_shift (wpr > 1)
    float depth_scale, pad2;     // augmented mode: depth (mm) to the colour byte range
    StreamPrm pc, pd;
};

// Row of mask word n (n < 2^31): division by the words-per-row constant as a
// multiply-high and shift. With l = ceil(log2 d) and m = ceil(2^(31+l) / d),
// m < 2^32 and floor(n m / 2^(31+l)) = floor(n / d) for every n < 2^31
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994).
__device__ __forceinline__ uint32_t div_wpr(uint32_t n, const CamView &cv) {
    return cv.wpr == 1 ? n : (__umulhi(n, cv.wpr_mul) >> cv.wpr_shift);
}

// ------------------------------------------------------------ storage types
template <int PREC> struct Storage;
template <> struct Storage<0> {
    static constexpr int kBytes = 4;
    static __device__ __forceinline__ float ldw(const void *b, int64_t o) {
        return static_cast<const float *>(b)[o];
    }
    static __device__ __forceinline__ float ldv(const void *b, int64_t o) {
        return static_cast<const float *>(b)[o];
    }
    static __device__ __forceinline__ void stw(void *b, int64_t o, float v) {
        static_cast<float *>(b)[o] = v;
    }
    static __device__ __forceinline__ void stv(void *b, int64_t o, float v) {
        static_cast<float *>(b)[o] = v;
    }
};
// Means and variances in float16, weights in bfloat16 (weights need range
// near zero more than mantissa). Values above the float16 range are clamped
// to its largest finite value instead of becoming infinite.
template <> struct Storage<1> {
    static constexpr int kBytes = 2;
    static __device__ __forceinline__ float ldw(const void *b, int64_t o) {
        return __bfloat162float(static_cast<const __nv_bfloat16 *>(b)[o]);
    }
    static __device__ __forceinline__ float ldv(const void *b, int64_t o) {
        return __half2float(static_cast<const __half *>(b)[o]);
    }
    static __device__ __forceinline__ void stw(void *b, int64_t o, float v) {
        static_cast<__nv_bfloat16 *>(b)[o] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ void stv(void *b, int64_t o, float v) {
        static_cast<__half *>(b)[o] = __float2half_rn(fminf(v, 65504.0f));
    }
};

// ------------------------------------------------------------ mixture step
template <int D> struct Comp {
    float key;
    int idx;
    float w, v;
    float mu[D];
};

template <int D>
__device__ __forceinline__ void comp_swap_if(Comp<D> &a, Comp<D> &b) {
    // a sits before b. Descending key; equal keys keep the lower stored index
    // first, which makes the order total and the network's result the stable
    // sort.
    const bool sw = (b.key > a.key) || (b.key == a.key && b.idx < a.idx);
    Comp<D> lo = sw ? b : a;
    Comp<D> hi = sw ? a : b;
    a = lo;
    b = hi;
}

// Optimal compare-exchange networks for 3, 4 and 5 elements.
template <int M, int D> __device__ __forceinline__ void rank_sort(Comp<D> (&c)[M]);
template <> __device__ __forceinline__ void rank_sort<3, 3>(Comp<3> (&c)[3]) {
    comp_swap_if(c[0], c[1]); comp_swap_if(c[0], c[2]); comp_swap_if(c[1], c[2]);
}
template <> __device__ __forceinline__ void rank_sort<3, 1>(Comp<1> (&c)[3]) {
    comp_swap_if(c[0], c[1]); comp_swap_if(c[0], c[2]); comp_swap_if(c[1], c[2]);
}
template <> __device__ __forceinline__ void rank_sort<3, 4>(Comp<4> (&c)[3]) {
    comp_swap_if(c[0], c[1]); comp_swap_if(c[0], c[2]); comp_swap_if(c[1], c[2]);
}
template <int D> __device__ __forceinline__ void net4(Comp<D> (&c)[4]) {
    comp_swap_if(c[0], c[1]); comp_swap_if(c[2], c[3]); comp_swap_if(c[0], c[2]);
    comp_swap_if(c[1], c[3]); comp_swap_if(c[1], c[2]);
}
template <> __device__ __forceinline__ void rank_sort<4, 3>(Comp<3> (&c)[4]) { net4(c); }
template <> __device__ __forceinline__ void rank_sort<4, 1>(Comp<1> (&c)[4]) { net4(c); }
template <> __device__ __forceinline__ void rank_sort<4, 4>(Comp<4> (&c)[4]) { net4(c); }
template <int D> __device__ __forceinline__ void net5(Comp<D> (&c)[5]) {
    comp_swap_if(c[0], c[1]); comp_swap_if(c[3], c[4]); comp_swap_if(c[2], c[4]);
    comp_swap_if(c[2], c[3]); comp_swap_if(c[0], c[3]); comp_swap_if(c[0], c[2]);
    comp_swap_if(c[1], c[4]); comp_swap_if(c[1], c[3]); comp_swap_if(c[1], c[2]);
}
template <> __device__ __forceinline__ void rank_sort<5, 3>(Comp<3> (&c)[5]) { net5(c); }
template <> __device__ __forceinline__ void rank_sort<5, 1>(Comp<1> (&c)[5]) { net5(c); }
template <> __device__ __forceinline__ void rank_sort<5, 4>(Comp<4> (&c)[5]) { net5(c); }

// One tick of one mixture at one pixel (§III.A). The components are in rank
// order on entry and on exit. Returns the stream's foreground bit.
// kSkipSorted: let a warp skip the sorting network when it would change
// nothing (pays where issue slots, not HBM, bound the kernel).
template <int M, int D, bool kSkipSorted, bool kOptions>
__device__ __forceinline__ int mixture_step(Comp<D> (&c)[M], const float (&x)[D],
                                            const StreamPrm &p) {
    // Match: first component, in rank order, within k standard deviations.
    int j = -1;
    float d2j = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float d2 = 0.f;
#pragma unroll
        for (int ch = 0; ch < D; ++ch) {
            const float df = x[ch] - c[i].mu[ch];
            d2 = fmaf(df, df, d2);
        }
        if (j < 0 && d2 < p.k2 * c[i].v) {
            j = i;
            d2j = d2;
        }
    }
    const bool matched = j >= 0;
    const int jj = matched ? j : M - 1;

    // Weights decay; the matched one gains alpha, or the last-ranked one is
    // replaced on a miss; then renormalise.
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float w = c[i].w * p.oma;
        if (i == jj)
            w = matched ? w + p.alpha : p.init_w;
        c[i].w = w;
        sum += w;
    }
    const float inv = 1.0f / sum;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        c[i].w *= inv;
        c[i].idx = i;
        if (i == jj) {
            if (matched) {
                float orho = p.oma, rho = p.alpha;
                if (kOptions)
                    rho = match_rate<D>(p, d2j, c[i].v, orho);
                float d2 = 0.f;
#pragma unroll
                for (int ch = 0; ch < D; ++ch) {
                    const float m = fmaf(orho, c[i].mu[ch], rho * x[ch]);
                    c[i].mu[ch] = m;
                    const float df = x[ch] - m;
                    d2 = fmaf(df, df, d2);
                }
                c[i].v = fmaxf(p.v_min, fmaf(orho, c[i].v, rho * (kOptions ? var_sample<D>(p, d2) : d2)));
            } else {
#pragma unroll
                for (int ch = 0; ch < D; ++ch)
                    c[i].mu[ch] = x[ch];
                c[i].v = p.init_var;
            }
        }
        c[i].key = c[i].w * rsqrtf(c[i].v);
    }

    // Re-rank by w / sigma (stable), then the background test. When every
    // lane's components are already in non-increasing key order (the usual
    // case: a background pixel matches its best component and the others
    // decay by the same factor), the stable network would leave them as they
    // are, so the warp skips it.
    bool sorted = true;
#pragma unroll
    for (int i = 1; i < M; ++i)
        sorted = sorted && !(c[i].key > c[i - 1].key);
    if (!kSkipSorted || __any_sync(__activemask(), !sorted))
        rank_sort<M, D>(c);
    int rank = 0, B = M;
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < M; ++r) {
        if (c[r].idx == jj)
            rank = r;
        acc += c[r].w;
        if (B == M && acc > p.T)
            B = r + 1;
    }
    return (!matched || rank >= B) ? 1 : 0;
}

// List 1 (§III.C) on the low four bits of the per-pixel byte.
__device__ __forceinline__ uint32_t fuse_list1(int fgc, int fgd, uint32_t fb) {
    int F = (int)(fb & 1u);
    int cpt = (int)((fb >> 1) & 7u) - 3;
    if (fgc == fgd) {
        F = fgd;
        cpt = 0;
    } else if (cpt == 3) {
        F = fgc;
        cpt = 0;
    } else if (cpt == -3) {
        F = fgd;
        cpt = 0;
    } else if (F == fgc) {
        cpt += 1;
    } else {
        cpt -= 1;
    }
    return (fb & ~15u) | (uint32_t)F | ((uint32_t)(cpt + 3) << 1);
}

// ------------------------------------------------------------ one pixel
// p: padded linear pixel index (row * w_pad + x). Returns bit 0 fused label,
// bit 1 colour foreground, bit 2 depth foreground (all 0 for padding).
// kVariant: 0 the paper's method with the default readings; 1 the same with
// the learning-rate and variance options of StreamPrm.flags honoured; 2 the
// augmentation alternative (options honoured too).
template <int M, int PREC, bool kSkipSorted, int kVariant>
__device__ __forceinline__ uint32_t process_pixel(const CamView &cv, int64_t p) {
    using S = Storage<PREC>;
    const uint32_t p32 = (uint32_t)p;
    const uint32_t row = div_wpr(p32 >> 5, cv);
    const uint32_t x = p32 - row * (uint32_t)cv.w_pad;
    if (x >= (uint32_t)cv.W)
        return 0u;
    const int64_t q = (int64_t)row * cv.W + x;
    const float xc[3] = {(float)cv.rgb[3 * q], (float)cv.rgb[3 * q + 1],
                         (float)cv.rgb[3 * q + 2]};
    const uint32_t draw = cv.depth[q];
    const float xd[1] = {(float)draw};
    // Element of plane 0 for this pixel; plane k lies k * kTile further on.
    const int64_t e0 = (int64_t)(p32 / kTile) * (kFields * M * kTile) + (p32 % kTile);
    const void *pl = cv.planes;

    if (kVariant == 2) {
        // The augmentation alternative (§III.B): one mixture over R, G, B and
        // the scaled depth, stored in the colour planes plus the depth-mean
        // plane. A zero reading takes the best-ranked component's depth mean.
        Comp<4> a[M];
        float xa[4] = {xc[0], xc[1], xc[2], cv.depth_scale * (float)draw};
        int fg;
        if (cv.first) {
            if (draw == 0u)
                xa[3] = 0.f;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                a[i].w = 1.0f / (float)M;
                a[i].mu[0] = xa[0]; a[i].mu[1] = xa[1]; a[i].mu[2] = xa[2]; a[i].mu[3] = xa[3];
                a[i].v = cv.pc.init_var;
            }
            fg = 0;
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const int64_t b = e0 + kFields * i * kTile;
                a[i].w = S::ldw(pl, b + F_WC * kTile);
                a[i].mu[0] = S::ldv(pl, b + F_MUR * kTile);
                a[i].mu[1] = S::ldv(pl, b + F_MUG * kTile);
                a[i].mu[2] = S::ldv(pl, b + F_MUB * kTile);
                a[i].mu[3] = S::ldv(pl, b + F_MUD * kTile);
                a[i].v = S::ldv(pl, b + F_VC * kTile);
            }
            if (draw == 0u)
                xa[3] = a[0].mu[3];
            fg = mixture_step<M, 4, kSkipSorted, true>(a, xa, cv.pc);
        }
        void *plw = cv.planes;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int64_t b = e0 + kFields * i * kTile;
            S::stw(plw, b + F_WC * kTile, a[i].w);
            S::stv(plw, b + F_MUR * kTile, a[i].mu[0]);
            S::stv(plw, b + F_MUG * kTile, a[i].mu[1]);
            S::stv(plw, b + F_MUB * kTile, a[i].mu[2]);
            S::stv(plw, b + F_MUD * kTile, a[i].mu[3]);
            S::stv(plw, b + F_VC * kTile, a[i].v);
            if (cv.first) { // the unused depth planes read as zero
                S::stw(plw, b + F_WD * kTile, 0.f);
                S::stv(plw, b + F_VD * kTile, 0.f);
            }
        }
        const uint32_t f = (uint32_t)fg;
        cv.fusion[p] = (uint8_t)f;
        return f | (f << 1) | (f << 2);
    }

    Comp<3> c[M];
    Comp<1> d[M];
    uint32_t fb;
    int fgc, fgd;
    if (cv.first) {
        fb = 0u;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            c[i].w = 1.0f / (float)M;
            c[i].mu[0] = xc[0]; c[i].mu[1] = xc[1]; c[i].mu[2] = xc[2];
            c[i].v = cv.pc.init_var;
            d[i].w = 0.f; d[i].mu[0] = 0.f; d[i].v = 0.f;
        }
        fgc = 0;
    } else {
        fb = cv.fusion[p];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int64_t b = e0 + kFields * i * kTile;
            c[i].w = S::ldw(pl, b + F_WC * kTile);
            c[i].mu[0] = S::ldv(pl, b + F_MUR * kTile);
            c[i].mu[1] = S::ldv(pl, b + F_MUG * kTile);
            c[i].mu[2] = S::ldv(pl, b + F_MUB * kTile);
            c[i].v = S::ldv(pl, b + F_VC * kTile);
            d[i].w = S::ldw(pl, b + F_WD * kTile);
            d[i].mu[0] = S::ldv(pl, b + F_MUD * kTile);
            d[i].v = S::ldv(pl, b + F_VD * kTile);
        }
        fgc = mixture_step<M, 3, kSkipSorted, (kVariant != 0)>(c, xc, cv.pc);
    }

    if (draw == 0u) {
        fgd = fgc; // no reading: depth model untouched, depth answer = colour
    } else if (!(fb & kDepthStarted)) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
            d[i].w = 1.0f / (float)M;
            d[i].mu[0] = xd[0];
            d[i].v = cv.pd.init_var;
        }
        fb |= kDepthStarted;
        fgd = 0;
    } else {
        fgd = mixture_step<M, 1, kSkipSorted, (kVariant != 0)>(d, xd, cv.pd);
    }
    fb = fuse_list1(fgc, fgd, fb);

    void *plw = cv.planes;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int64_t b = e0 + kFields * i * kTile;
        S::stw(plw, b + F_WC * kTile, c[i].w);
        S::stv(plw, b + F_MUR * kTile, c[i].mu[0]);
        S::stv(plw, b + F_MUG * kTile, c[i].mu[1]);
        S::stv(plw, b + F_MUB * kTile, c[i].mu[2]);
        S::stv(plw, b + F_VC * kTile, c[i].v);
        S::stw(plw, b + F_WD * kTile, d[i].w);
        S::stv(plw, b + F_MUD * kTile, d[i].mu[0]);
        S::stv(plw, b + F_VD * kTile, d[i].v);
    }
    cv.fusion[p] = (uint8_t)fb;
    return (fb & 1u) | ((uint32_t)fgc << 1) | ((uint32_t)fgd << 2);
}

// All 32 lanes of the warp call this for 32 consecutive padded pixels
// starting at a multiple of 32 (word index wi).
__device__ __forceinline__ void write_mask_words(const CamView &cv, int64_t wi, uint32_t bits) {
    const uint32_t F = __ballot_sync(0xffffffffu, bits & 1u);
    const uint32_t fc = __ballot_sync(0xffffffffu, bits & 2u);
    const uint32_t fd = __ballot_sync(0xffffffffu, bits & 4u);
    if ((threadIdx.x & 31u) == 0u) {
        cv.mask[wi] = F;
        if (cv.fg_rgb)
            cv.fg_rgb[wi] = fc;
        if (cv.fg_d)
            cv.fg_d[wi] = fd;
    }
}

} // namespace gmmdev
