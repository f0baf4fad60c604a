// Per-pixel device code shared by the single-camera tick kernel and the
// multi-camera persistent kernel: state loads/stores for both storage
// precisions, one mixture step (match, update or replace, re-rank,
// background test), List-1 fusion, and the bit-packed mask write.
//
// State layout in device memory (one camera). Pixels are numbered in padded
// row-major order p = row * w_pad + x (rows padded to a multiple of 32 pixels,
// so the 32 pixels of a warp map to one mask word) and grouped into tiles of
// kTile = 256 consecutive pixels. Each tile stores the 8M values of its
// pixels contiguously (8M * kTile elements), component-major (i the rank;
// fields w_c, mu_r, mu_g, mu_b, v_c, w_d, mu_d, v_d):
//   FP32: one plane per field, element (8 i + field) * kTile + t for tile
//         pixel t: a warp reads 32 consecutive floats of a plane, one fully
//         used 128-byte line;
//   FP16/BF16: two groups of four 2-byte slots per component and pixel,
//         group 0 = {w_c, w_d, mu_r, mu_g}, group 1 = {mu_b, v_c, mu_d, v_d},
//         element ((2 i + group) * kTile + t) * 4 + slot: one 8-byte access
//         moves a group (a warp: 256 contiguous bytes), and each 4-byte half
//         holds two values of one type, converted by one packed instruction.
// The offsets of a pixel's values are compile-time constants from one base
// address, and a tile's whole state is one contiguous block that a single
// bulk copy moves. The List-1 byte of a pixel lives in a separate byte array
// indexed by p (n_tiles * kTile bytes).
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
constexpr int kStochasticWeights = 4; // CamView.flags: BF16 weights stored with stochastic rounding
constexpr uint32_t kRhoEta = 1u;        // StreamPrm.flags: rho = alpha * eta(x | mu, sigma)
constexpr uint32_t kVarPerChannel = 2u; // StreamPrm.flags: v is the per-channel variance

// Group and slot of a field in the FP16/BF16 layout.
__host__ __device__ constexpr int h16_group(int f) {
    return (f == F_MUB || f == F_VC || f == F_MUD || f == F_VD) ? 1 : 0;
}
__host__ __device__ constexpr int h16_slot(int f) {
    return (f == F_WC || f == F_MUB) ? 0 : (f == F_WD || f == F_VC) ? 1
                                     : (f == F_MUR || f == F_MUD) ? 2 : 3;
}
// Element index, within its tile, of field f of component i at tile pixel t.
template <int PREC> __host__ __device__ constexpr int tile_elem(int i, int f, int t) {
    return PREC == 0 ? (kFields * i + f) * kTile + t
                     : ((2 * i + h16_group(f)) * kTile + t) * 4 + h16_slot(f);
}

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
// single-camera kernel, read from constant memory by the pooled kernel.
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
    int M, prec, first, flags; // flags: kStageInputs, kModeAugmented, kStochasticWeights
    uint32_t wpr_mul, wpr_shift; // n / wpr == umulhi(n, wpr_mul) >> wpr_shift (wpr > 1)
    float depth_scale;           // augmented mode: depth (mm) to the colour byte range
    uint32_t tick;               // ticks the model has taken (seeds stochastic rounding)
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
// FP16/BF16 state: means and variances in float16, weights in bfloat16
// (weights need range near zero more than mantissa), converted in pairs.
// bfloat16 -> float is exact (the bits move up); float -> bfloat16 rounds to
// nearest even; float -> float16 rounds to nearest even and saturates at the
// largest finite value instead of becoming infinite.
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ float2 f16x2_unpack(uint32_t u) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
__device__ __forceinline__ uint32_t bf16x2_pack(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t f16x2_pack_sat(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Stochastic rounding of non-negative floats to bfloat16 (the weights):
// adding 16 uniform random bits below the kept ones and truncating rounds up
// with probability equal to the dropped fraction, so the stored weight is
// unbiased. The bits come from a counter-based hash of (tick, pixel, value):
// MurmurHash3's 32-bit finaliser (Appleby), applied twice.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint32_t sr_bits(uint32_t tick, uint32_t p, uint32_t k) {
    return fmix32(fmix32(tick * 0x9e3779b9u + p) ^ (k * 0x27d4eb2fu));
}
__device__ __forceinline__ uint32_t bf16x2_pack_sr(float lo, float hi, uint32_t r) {
    const uint32_t l = (__float_as_uint(lo) + (r & 0xffffu)) >> 16;
    const uint32_t h = (__float_as_uint(hi) + (r >> 16)) & 0xffff0000u;
    return h | l;
}

// The eight values of one component at one pixel.
struct Fields {
    float wc, mur, mug, mub, vc, wd, mud, vd;
};

// Load / store component i of the pixel whose tile starts at element tb
// (tile index * 8M * kTile) and sits at column t of it; e0 = tb + t.
template <int PREC, int M>
__device__ __forceinline__ Fields load_fields(const void *pl, int64_t e0, int64_t tb, uint32_t t,
                                              int i) {
    Fields f;
    if constexpr (PREC == 0) {
        const float *b = static_cast<const float *>(pl) + e0 + kFields * i * kTile;
        f.wc = b[F_WC * kTile];
        f.mur = b[F_MUR * kTile];
        f.mug = b[F_MUG * kTile];
        f.mub = b[F_MUB * kTile];
        f.vc = b[F_VC * kTile];
        f.wd = b[F_WD * kTile];
        f.mud = b[F_MUD * kTile];
        f.vd = b[F_VD * kTile];
    } else {
        const uint2 *g = static_cast<const uint2 *>(pl) + (tb >> 2) + t + 2 * i * kTile;
        const uint2 g0 = g[0], g1 = g[kTile];
        f.wc = bf16_lo(g0.x);
        f.wd = bf16_hi(g0.x);
        const float2 rg = f16x2_unpack(g0.y), bv = f16x2_unpack(g1.x), dv = f16x2_unpack(g1.y);
        f.mur = rg.x; f.mug = rg.y;
        f.mub = bv.x; f.vc = bv.y;
        f.mud = dv.x; f.vd = dv.y;
    }
    return f;
}

// kDepth: also write w_d and v_d (FP32 stores them separately; FP16 always
// writes them with their group). sr: nonzero = 32 random bits for the
// stochastic rounding of the two weights (FP16/BF16 state, kSR builds only).
template <int PREC, int M, bool kDepth = true, bool kSR = false>
__device__ __forceinline__ void store_fields(void *pl, int64_t e0, int64_t tb, uint32_t t, int i,
                                             const Fields &f, uint32_t sr = 0u) {
    if constexpr (PREC == 0) {
        float *b = static_cast<float *>(pl) + e0 + kFields * i * kTile;
        b[F_WC * kTile] = f.wc;
        b[F_MUR * kTile] = f.mur;
        b[F_MUG * kTile] = f.mug;
        b[F_MUB * kTile] = f.mub;
        b[F_VC * kTile] = f.vc;
        if (kDepth)
            b[F_WD * kTile] = f.wd;
        b[F_MUD * kTile] = f.mud;
        if (kDepth)
            b[F_VD * kTile] = f.vd;
    } else {
        uint2 *g = static_cast<uint2 *>(pl) + (tb >> 2) + t + 2 * i * kTile;
        const uint32_t w = (kSR && sr) ? bf16x2_pack_sr(f.wc, f.wd, sr) : bf16x2_pack(f.wc, f.wd);
        g[0] = make_uint2(w, f16x2_pack_sat(f.mur, f.mug));
        g[kTile] = make_uint2(f16x2_pack_sat(f.mub, f.vc), f16x2_pack_sat(f.mud, f.vd));
    }
}

// ------------------------------------------------------------ mixture step
// Sort key of a component: the bits of w / sqrt(v) (a positive float, so its
// bits order like its value) with the low three bits replaced by 7 - the
// component's stored rank i. Comparing keys as unsigned integers orders by
// w / sigma and, between values that agree to 2^-20 relative (the same value
// included), puts the lower stored rank first: a total order, under which the
// network's result is the stable sort. (Two values that close lie well inside
// the 1e-5 margin at which a decision counts as near its threshold.)
__device__ __forceinline__ uint32_t rank_key(float w, float v, int i) {
    return (__float_as_uint(w * rsqrtf(v)) & ~7u) | (7u - (uint32_t)i);
}

template <int D> struct Comp {
    uint32_t key; // rank_key of the component
    float w, v;
    float mu[D];
};

template <int D>
__device__ __forceinline__ void comp_swap_if(Comp<D> &a, Comp<D> &b) {
    // a sits before b: the larger key goes first
    const bool sw = b.key > a.key;
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

// Background test (§III.A) of the changed component at rank `rank` after
// the update: it is in B (the shortest rank prefix summing past T) unless the
// prefix before it already sums past T (prefix sums of non-negative weights
// do not decrease under rounding, so this equals rank >= B). A miss is
// foreground.
template <int M, int D>
__device__ __forceinline__ int background_test(const Comp<D> (&c)[M], int rank, bool matched,
                                               float T) {
    float acc = 0.f, before = 0.f;
#pragma unroll
    for (int r = 0; r < M - 1; ++r) {
        acc += c[r].w;
        if (r + 1 == rank)
            before = acc;
    }
    return (!matched || before > T) ? 1 : 0;
}

// The update after the match (§III.A): weights, the changed component's mean
// and variance, re-ranking and the background test. hit: bit i set when
// component i lies within k standard deviations (the first set bit is the
// match); d2s: the squared distances. kJ >= 0: every lane of this call
// matched component kJ (the changed component is then known at compile time
// and needs no selects); kJ < 0: any outcome.
template <int M, int D, bool kSkipSorted, bool kOptions, int kJ>
__device__ __forceinline__ int mixture_update(Comp<D> (&c)[M], const float (&x)[D],
                                              const StreamPrm &p, uint32_t lanes, uint32_t hit,
                                              const float (&d2s)[M]) {
    const bool matched = kJ >= 0 || hit != 0u;
    const int jj = kJ >= 0 ? kJ : (matched ? __ffs(hit) - 1 : M - 1);
    float d2j = d2s[0];
    if (kOptions) {
#pragma unroll
        for (int i = 1; i < M; ++i)
            if (i == jj)
                d2j = d2s[i];
    }

    // The component that changes (matched, or the last-ranked on a miss),
    // gathered once.
    float muj[D], vj = c[0].v;
#pragma unroll
    for (int ch = 0; ch < D; ++ch)
        muj[ch] = c[0].mu[ch];
#pragma unroll
    for (int i = 1; i < M; ++i) {
        if (i == jj) {
            vj = c[i].v;
#pragma unroll
            for (int ch = 0; ch < D; ++ch)
                muj[ch] = c[i].mu[ch];
        }
    }

    // Weights decay; the matched one gains alpha, or the last-ranked one is
    // replaced on a miss; then renormalise. (Explicitly rounded operations:
    // no multiply-add contraction, so every path rounds alike.)
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float w = __fmul_rn(c[i].w, p.oma);
        if (i == jj)
            w = matched ? __fadd_rn(w, p.alpha) : p.init_w;
        c[i].w = w;
        sum = __fadd_rn(sum, w);
    }
    const float inv = __fdividef(1.0f, sum); // within 2 ulp; the sum is near 1

    // Mean and variance of the changed component (the variance from the
    // squared distance to the new mean).
    if (matched) {
        float orho = p.oma, rho = p.alpha;
        if (kOptions)
            rho = match_rate<D>(p, d2j, vj, orho);
        float d2n = 0.f;
#pragma unroll
        for (int ch = 0; ch < D; ++ch) {
            muj[ch] = fmaf(orho, muj[ch], rho * x[ch]);
            const float df = x[ch] - muj[ch];
            d2n = fmaf(df, df, d2n);
        }
        vj = fmaxf(p.v_min, fmaf(orho, vj, rho * (kOptions ? var_sample<D>(p, d2n) : d2n)));
    } else {
#pragma unroll
        for (int ch = 0; ch < D; ++ch)
            muj[ch] = x[ch];
        vj = p.init_var;
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        c[i].w *= inv;
        if (i == jj) {
#pragma unroll
            for (int ch = 0; ch < D; ++ch)
                c[i].mu[ch] = muj[ch];
            c[i].v = vj;
        }
        c[i].key = rank_key(c[i].w, c[i].v, i);
    }

    // Re-rank by w / sigma (stable), then the background test. When every
    // lane's components are already in non-increasing key order (the usual
    // case: a background pixel matches its best component and the others
    // decay by the same factor), the stable network would leave them as they
    // are, so the warp skips it and the changed component keeps its rank.
    bool sorted = true;
#pragma unroll
    for (int i = 1; i < M; ++i)
        sorted = sorted && !(c[i].key > c[i - 1].key);
    int rank = jj; // the changed component's rank after the update
    if (!kSkipSorted || __any_sync(lanes, !sorted)) {
        rank_sort<M, D>(c);
#pragma unroll
        for (int r = 0; r < M; ++r)
            if ((c[r].key & 7u) == 7u - (uint32_t)jj) // its stored rank, from the key
                rank = r;
        if (kJ >= 0) // (the specialised path keeps its rank known where no sort ran)
            return background_test<M, D>(c, rank, matched, p.T);
    }
    return background_test<M, D>(c, rank, matched, p.T);
}

// One tick of one mixture at one pixel (§III.A). The components are in rank
// order on entry and on exit. Returns the stream's foreground bit.
// kSkipSorted: let a warp skip the sorting network when it would change
// nothing (pays where issue slots, not HBM, bound the kernel); `lanes` is
// then the set of lanes of the warp that make this same call, computed by
// the caller before the code diverged (unused otherwise). kFastBest (with
// kSkipSorted): a path specialised to a match of the best-ranked component
// when every lane of the call has one (the usual case for background
// pixels); it computes exactly what the general path does.
template <int M, int D, bool kSkipSorted, bool kOptions, bool kFastBest = kSkipSorted>
__device__ __forceinline__ int mixture_step(Comp<D> (&c)[M], const float (&x)[D],
                                            const StreamPrm &p, uint32_t lanes) {
    // Match: first component, in rank order, within k standard deviations
    // (bit i of hit: component i is within; the first set bit wins).
    uint32_t hit = 0u;
    float d2s[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float d2 = 0.f;
#pragma unroll
        for (int ch = 0; ch < D; ++ch) {
            const float df = x[ch] - c[i].mu[ch];
            d2 = fmaf(df, df, d2);
        }
        d2s[i] = d2;
        if (d2 < p.k2 * c[i].v)
            hit |= 1u << i;
    }
    if (kSkipSorted && kFastBest && __all_sync(lanes, hit & 1u))
        return mixture_update<M, D, kSkipSorted, kOptions, 0>(c, x, p, lanes, hit, d2s);
    return mixture_update<M, D, kSkipSorted, kOptions, -1>(c, x, p, lanes, hit, d2s);
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

// Random bits for the weights of component i at padded pixel p when the
// view asks for stochastic rounding, else 0.
__device__ __forceinline__ uint32_t sr_weights(const CamView &cv, uint32_t p, int i) {
    if (!(cv.flags & kStochasticWeights))
        return 0u;
    const uint32_t r = sr_bits(cv.tick, p, (uint32_t)i);
    return r ? r : 1u;
}

// ------------------------------------------------------------ one pixel
// p: padded linear pixel index (row * w_pad + x). Returns bit 0 fused label,
// bit 1 colour foreground, bit 2 depth foreground (all 0 for padding).
// kVariant: 0 the paper's method with the default readings; 1 the same with
// the learning-rate and variance options of StreamPrm.flags honoured; 2 the
// augmentation alternative (options honoured too).
template <int M, int PREC, bool kSkipSorted, int kVariant>
__device__ __forceinline__ uint32_t process_pixel(const CamView &cv, int64_t p) {
    const uint32_t p32 = (uint32_t)p;
    const uint32_t row = div_wpr(p32 >> 5, cv);
    const uint32_t x = p32 - row * (uint32_t)cv.w_pad;
    // Every caller enters with whole warps; the lanes on image pixels (not
    // row padding) are the ones that run the colour (or augmented) mixture.
    const uint32_t lanes_c = kSkipSorted ? __ballot_sync(0xffffffffu, x < (uint32_t)cv.W) : 0u;
    if (x >= (uint32_t)cv.W)
        return 0u;
    const int64_t q = (int64_t)row * cv.W + x;
    const float xc[3] = {(float)cv.rgb[3 * q], (float)cv.rgb[3 * q + 1],
                         (float)cv.rgb[3 * q + 2]};
    const uint32_t draw = cv.depth[q];
    const float xd[1] = {(float)draw};
    // First element of the pixel's tile, and the pixel's column in it.
    const int64_t tb = (int64_t)(p32 / kTile) * (kFields * M * kTile);
    const uint32_t t = p32 % kTile;
    const int64_t e0 = tb + t;
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
                const Fields f = load_fields<PREC, M>(pl, e0, tb, t, i);
                a[i].w = f.wc;
                a[i].mu[0] = f.mur; a[i].mu[1] = f.mug; a[i].mu[2] = f.mub; a[i].mu[3] = f.mud;
                a[i].v = f.vc;
            }
            if (draw == 0u)
                xa[3] = a[0].mu[3];
            fg = mixture_step<M, 4, kSkipSorted, true, (PREC != 0)>(a, xa, cv.pc, lanes_c);
        }
        void *plw = cv.planes;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            // w_d and v_d are unused and read as zero
            const Fields f = {a[i].w, a[i].mu[0], a[i].mu[1], a[i].mu[2], a[i].v,
                              0.f,    a[i].mu[3], 0.f};
            if (PREC != 0 || cv.first)
                store_fields<PREC, M, true, true>(plw, e0, tb, t, i, f, sr_weights(cv, p32, i));
            else
                store_fields<PREC, M, false>(plw, e0, tb, t, i, f);
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
        if constexpr (PREC == 0) {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const Fields f = load_fields<PREC, M>(pl, e0, tb, t, i);
                c[i].w = f.wc;
                c[i].mu[0] = f.mur; c[i].mu[1] = f.mug; c[i].mu[2] = f.mub;
                c[i].v = f.vc;
                d[i].w = f.wd;
                d[i].mu[0] = f.mud;
                d[i].v = f.vd;
            }
            fgc = mixture_step<M, 3, kSkipSorted, (kVariant != 0), (PREC != 0)>(c, xc, cv.pc, lanes_c);
        } else {
            // The depth values stay packed (two registers per component
            // instead of three) while the colour mixture runs.
            uint32_t dw[M], dmv[M];
            const uint2 *g = static_cast<const uint2 *>(pl) + (tb >> 2) + t;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const uint2 g0 = g[2 * i * kTile], g1 = g[(2 * i + 1) * kTile];
                c[i].w = bf16_lo(g0.x);
                const float2 rg = f16x2_unpack(g0.y), bv = f16x2_unpack(g1.x);
                c[i].mu[0] = rg.x; c[i].mu[1] = rg.y; c[i].mu[2] = bv.x;
                c[i].v = bv.y;
                dw[i] = g0.x;
                dmv[i] = g1.y;
            }
            fgc = mixture_step<M, 3, kSkipSorted, (kVariant != 0), (PREC != 0)>(c, xc, cv.pc, lanes_c);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                d[i].w = bf16_hi(dw[i]);
                const float2 mv = f16x2_unpack(dmv[i]);
                d[i].mu[0] = mv.x;
                d[i].v = mv.y;
            }
        }
    }

    // The lanes that run the depth mixture: a reading, and a started model.
    const uint32_t lanes_d =
        kSkipSorted ? __ballot_sync(lanes_c, draw != 0u && (fb & kDepthStarted)) : 0u;
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
        fgd = mixture_step<M, 1, kSkipSorted, (kVariant != 0), (PREC != 0)>(d, xd, cv.pd, lanes_d);
    }
    fb = fuse_list1(fgc, fgd, fb);

    void *plw = cv.planes;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const Fields f = {c[i].w, c[i].mu[0], c[i].mu[1], c[i].mu[2], c[i].v,
                          d[i].w, d[i].mu[0], d[i].v};
        if (kVariant == 0)
            store_fields<PREC, M>(plw, e0, tb, t, i, f);
        else
            store_fields<PREC, M, true, true>(plw, e0, tb, t, i, f, sr_weights(cv, p32, i));
    }
    cv.fusion[p] = (uint8_t)fb;
    return (fb & 1u) | ((uint32_t)fgc << 1) | ((uint32_t)fgd << 2);
}

// All 32 lanes of the warp call this for 32 consecutive padded pixels
// starting at a multiple of 32 (word index wi).
__device__ __forceinline__ void write_mask_words(const CamView &cv, int64_t wi, uint32_t bits) {
    const uint32_t F = __ballot_sync(0xffffffffu, bits & 1u);
    const bool lane0 = (threadIdx.x & 31u) == 0u;
    if (lane0)
        cv.mask[wi] = F;
    if (cv.fg_rgb) { // uniform: the whole warp takes it or not
        const uint32_t fc = __ballot_sync(0xffffffffu, bits & 2u);
        if (lane0)
            cv.fg_rgb[wi] = fc;
    }
    if (cv.fg_d) {
        const uint32_t fd = __ballot_sync(0xffffffffu, bits & 4u);
        if (lane0)
            cv.fg_d[wi] = fd;
    }
}

} // namespace gmmdev
