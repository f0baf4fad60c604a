// Staged tick kernel: persistent CTAs stream tiles of the state through
// shared memory with 1-D bulk copies (TMA engine) in a multi-stage pipeline.
//
// A state tile (256 pixels, all 8*M planes) is one contiguous block in HBM.
// Per tile one thread issues a single bulk copy of that block, one of the
// tile's List-1 bytes and, when the frame rows allow it, one each for the
// tile's RGB and depth bytes, into a stage buffer (an mbarrier counts the
// bytes); the whole CTA computes one pixel per thread out of shared memory;
// the same thread writes the stage back with two bulk stores. Loads for the
// next ST-1 tiles are in flight while a tile is computed, so the HBM traffic
// does not wait on the arithmetic, and the per-thread instruction stream
// holds no global address arithmetic.
//
// With the state in shared memory the re-ranking needs no sorting network:
// each component's stable rank comes from M(M-1)/2 key comparisons and the
// component is written straight to its rank slot. Thread t always touches
// element t of a plane, so every access, including the rank-addressed ones,
// is bank-conflict free.
#include <cuda_runtime.h>

#include <mutex>

#include "gmm_internal.h"
#include "gmm_tma.cuh"

using namespace gmmdev;

namespace {

template <int PREC, int TP> struct Smem;
template <int TP> struct Smem<0, TP> {
    static constexpr int kBytes = 4;
    static __device__ __forceinline__ float ldw(const uint8_t *st, int k, int t) {
        return reinterpret_cast<const float *>(st + k * TP * 4)[t];
    }
    static __device__ __forceinline__ float ldv(const uint8_t *st, int k, int t) {
        return reinterpret_cast<const float *>(st + k * TP * 4)[t];
    }
    static __device__ __forceinline__ void stw(uint8_t *st, int k, int t, float v) {
        reinterpret_cast<float *>(st + k * TP * 4)[t] = v;
    }
    static __device__ __forceinline__ void stv(uint8_t *st, int k, int t, float v) {
        reinterpret_cast<float *>(st + k * TP * 4)[t] = v;
    }
};
// FP16/BF16: plane k = 8 i + f is slot h16_slot(f) of group h16_group(f) of
// component i (the layout of gmm_device.cuh; TP pixels per tile).
template <int TP> struct Smem<1, TP> {
    static constexpr int kBytes = 2;
    static __device__ __forceinline__ int at(int k, int t) {
        const int f = k & 7;
        return ((2 * (k >> 3) + h16_group(f)) * TP + t) * 4 + h16_slot(f);
    }
    static __device__ __forceinline__ float ldw(const uint8_t *st, int k, int t) {
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(st)[at(k, t)]);
    }
    static __device__ __forceinline__ float ldv(const uint8_t *st, int k, int t) {
        return __half2float(reinterpret_cast<const __half *>(st)[at(k, t)]);
    }
    static __device__ __forceinline__ void stw(uint8_t *st, int k, int t, float v) {
        reinterpret_cast<__nv_bfloat16 *>(st)[at(k, t)] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ void stv(uint8_t *st, int k, int t, float v) {
        reinterpret_cast<__half *>(st)[at(k, t)] = __float2half_rn(fminf(v, 65504.0f));
    }
};

// One tick of one mixture (§III.A) for the pixel in column t of the stage.
// f0: plane field of the stream's weight (colour 0, depth 5). Same readings
// as mixture_step in gmm_device.cuh; the components are read in rank order
// and written back at their new ranks.
template <int M, int D, int PREC, int TP>
__device__ __forceinline__ int staged_mixture_step(uint8_t *st, int f0, int t,
                                                   const float (&x)[D], const StreamPrm &p) {
    using A = Smem<PREC, TP>;
    float w[M], v[M], mu[M][D];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int b = kFields * i + f0;
        w[i] = A::ldw(st, b, t);
#pragma unroll
        for (int c = 0; c < D; ++c)
            mu[i][c] = A::ldv(st, b + 1 + c, t);
        v[i] = A::ldv(st, b + 1 + D, t);
    }
    // Match: first component in rank order within k standard deviations.
    int j = -1;
    float d2j = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float df = x[c] - mu[i][c];
            d2 = fmaf(df, df, d2);
        }
        if (j < 0 && d2 < p.k2 * v[i]) {
            j = i;
            d2j = d2;
        }
    }
    const bool matched = j >= 0;
    const int jj = matched ? j : M - 1;
    float muj[D], vj = v[0];
#pragma unroll
    for (int c = 0; c < D; ++c)
        muj[c] = mu[0][c];
#pragma unroll
    for (int i = 1; i < M; ++i) {
        if (i == jj) {
            vj = v[i];
#pragma unroll
            for (int c = 0; c < D; ++c)
                muj[c] = mu[i][c];
        }
    }
    // Weights: decay, gain or replacement, renormalisation.
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float wi = __fmul_rn(w[i], p.oma);
        if (i == jj)
            wi = matched ? __fadd_rn(wi, p.alpha) : p.init_w;
        w[i] = wi;
        sum = __fadd_rn(sum, wi);
    }
    const float inv = __fdividef(1.0f, sum);
#pragma unroll
    for (int i = 0; i < M; ++i)
        w[i] *= inv;
    // The matched component moves toward the sample; a miss starts a new one.
    if (matched) {
        float orho;
        const float rho = match_rate<D>(p, d2j, vj, orho);
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            muj[c] = fmaf(orho, muj[c], rho * x[c]);
            const float df = x[c] - muj[c];
            d2 = fmaf(df, df, d2);
        }
        vj = fmaxf(p.v_min, fmaf(orho, vj, rho * var_sample<D>(p, d2)));
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c)
            muj[c] = x[c];
        vj = p.init_var;
    }
    // Ranks by rank_key (w / sqrt(v), ties by stored rank): a component goes
    // after every earlier one with a larger key.
    uint32_t key[M];
    int r[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        key[i] = rank_key(w[i], i == jj ? vj : v[i], i);
        r[i] = 0;
    }
#pragma unroll
    for (int i = 1; i < M; ++i) {
#pragma unroll
        for (int l = 0; l < i; ++l) {
            if (key[l] > key[i])
                ++r[i];
            else
                ++r[l];
        }
    }
    int rank_j = r[0];
#pragma unroll
    for (int i = 1; i < M; ++i)
        if (i == jj)
            rank_j = r[i];
    // Write every component at its rank, then the updated one over its slot.
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int b = kFields * r[i] + f0;
        A::stw(st, b, t, w[i]);
#pragma unroll
        for (int c = 0; c < D; ++c)
            A::stv(st, b + 1 + c, t, mu[i][c]);
        A::stv(st, b + 1 + D, t, v[i]);
    }
    {
        const int b = kFields * rank_j + f0;
#pragma unroll
        for (int c = 0; c < D; ++c)
            A::stv(st, b + 1 + c, t, muj[c]);
        A::stv(st, b + 1 + D, t, vj);
    }
    // Background set: running sum of the weights in rank order (FP32 values).
    float acc = 0.f;
    int B = M;
#pragma unroll
    for (int rr = 0; rr < M; ++rr) {
        float wr = 0.f;
#pragma unroll
        for (int i = 0; i < M; ++i)
            wr += (r[i] == rr) ? w[i] : 0.f;
        acc += wr;
        if (B == M && acc > p.T)
            B = rr + 1;
    }
    return (!matched || rank_j >= B) ? 1 : 0;
}

// One pixel (column t of the stage); returns fused | colour << 1 | depth << 2.
template <int M, int PREC>
__device__ __forceinline__ uint32_t staged_pixel(uint8_t *st, int t, const CamView &cv,
                                                 const float (&xc)[3], uint32_t draw) {
    using A = Smem<PREC, kTile>;
    uint8_t *fus = st + kFields * M * kTile * A::kBytes;
    uint32_t fb = fus[t];
    const int fgc = staged_mixture_step<M, 3, PREC, kTile>(st, F_WC, t, xc, cv.pc);
    int fgd;
    if (draw == 0u) {
        fgd = fgc; // no reading: depth model untouched, depth answer = colour
    } else if (!(fb & kDepthStarted)) {
        const float d0 = (float)draw, w0 = 1.0f / (float)M;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            A::stw(st, kFields * i + F_WD, t, w0);
            A::stv(st, kFields * i + F_MUD, t, d0);
            A::stv(st, kFields * i + F_VD, t, cv.pd.init_var);
        }
        fb |= kDepthStarted;
        fgd = 0;
    } else {
        const float xd[1] = {(float)draw};
        fgd = staged_mixture_step<M, 1, PREC, kTile>(st, F_WD, t, xd, cv.pd);
    }
    fb = fuse_list1(fgc, fgd, fb);
    fus[t] = (uint8_t)fb;
    return (fb & 1u) | ((uint32_t)fgc << 1) | ((uint32_t)fgd << 2);
}

// One CTA of kTile threads per state tile in flight. A stage holds one tile:
// its 8M planes (one contiguous block in HBM, moved by one bulk copy), its
// List-1 bytes and, when cv.flags has kStageInputs, its RGB and depth bytes.
template <int M, int PREC, int ST>
__global__ void __launch_bounds__(kTile) k_tick_staged(const CamView cv, int *status) {
    using A = Smem<PREC, kTile>;
    constexpr uint32_t STATE = kFields * M * kTile * A::kBytes; // one tile of planes
    constexpr uint32_t FUS = STATE;                            // List-1 bytes
    constexpr uint32_t RGB = FUS + kTile;                      // 3 bytes per pixel
    constexpr uint32_t DEP = RGB + 3 * kTile;                  // 2 bytes per pixel
    constexpr uint32_t STAGE = DEP + 2 * kTile;
    static_assert(STATE % 16 == 0 && STAGE % 16 == 0, "bulk copies need 16-byte granules");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[ST];

    const int tid = threadIdx.x;
    const int64_t n_tiles = cv.n_tiles;
    const bool stage_in = (cv.flags & kStageInputs) != 0;
    const uint8_t *gsrc = static_cast<const uint8_t *>(cv.planes);
    uint8_t *gdst = static_cast<uint8_t *>(cv.planes);
    uint32_t pending = 0; // thread 0: stages with a load in flight

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < ST; ++s)
            gmmtma::mbar_init(&full[s], 1);
        gmmtma::fence_mbar_init();
    }
    __syncthreads();

    auto issue_load = [&](int64_t tile, int s) {
        const int64_t p0 = tile * kTile;
        const uint32_t npx = (uint32_t)min((int64_t)kTile, cv.n_pad - p0);
        uint8_t *dst = smem + s * STAGE;
        gmmtma::mbar_arrive_expect_tx(&full[s], STATE + kTile + (stage_in ? 5u * npx : 0u));
        gmmtma::bulk_load(dst, gsrc + (size_t)tile * STATE, STATE, &full[s]);
        gmmtma::bulk_load(dst + FUS, cv.fusion + p0, kTile, &full[s]);
        if (stage_in) {
            gmmtma::bulk_load(dst + RGB, cv.rgb + 3 * p0, 3 * npx, &full[s]);
            gmmtma::bulk_load(dst + DEP, cv.depth + p0, 2 * npx, &full[s]);
        }
        pending |= 1u << s;
    };

    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            const int64_t tile = blockIdx.x + (int64_t)s * gridDim.x;
            if (tile < n_tiles)
                issue_load(tile, s);
        }
    }

    int j = 0;
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++j) {
        const int s = j % ST;
        const uint32_t parity = (uint32_t)(j / ST) & 1u;
        const int64_t p0 = tile * kTile;
        const uint32_t p = (uint32_t)(p0 + tid);
        const bool in = (int64_t)p < cv.n_pad;
        uint8_t *stg = smem + s * STAGE;
        // Row of the pixel; frame inputs come from the stage or, when they are
        // not staged, straight from HBM before the stage wait.
        uint32_t row = 0, x = 0;
        bool valid = false;
        float xc[3] = {0.f, 0.f, 0.f};
        uint32_t draw = 0u;
        if (in) {
            row = div_wpr(p >> 5, cv);
            x = p - row * (uint32_t)cv.w_pad;
            valid = x < (uint32_t)cv.W;
            if (valid && !stage_in) {
                const int64_t q = (int64_t)row * cv.W + x;
                xc[0] = (float)cv.rgb[3 * q];
                xc[1] = (float)cv.rgb[3 * q + 1];
                xc[2] = (float)cv.rgb[3 * q + 2];
                draw = cv.depth[q];
            }
        }
        const bool ok = gmmtma::mbar_wait(&full[s], parity);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0)
            pending &= ~(1u << s);
        uint32_t bits = 0u;
        if (valid) {
            if (stage_in) {
                xc[0] = (float)stg[RGB + 3 * tid];
                xc[1] = (float)stg[RGB + 3 * tid + 1];
                xc[2] = (float)stg[RGB + 3 * tid + 2];
                draw = reinterpret_cast<const uint16_t *>(stg + DEP)[tid];
            }
            bits = staged_pixel<M, PREC>(stg, tid, cv, xc, draw);
        }
        if (in) // whole warps: n_pad and kTile are multiples of 32
            write_mask_words(cv, p >> 5, bits);
        gmmtma::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            gmmtma::bulk_store(gdst + (size_t)tile * STATE, stg, STATE);
            gmmtma::bulk_store(cv.fusion + p0, stg + FUS, kTile);
            gmmtma::bulk_commit();
            const int64_t next = tile + (int64_t)ST * gridDim.x;
            if (next < n_tiles) {
                gmmtma::bulk_wait_read<0>(); // the stage is read out before refilling it
                issue_load(next, s);
            }
        }
    }
    if (tid == 0) {
        gmmtma::bulk_wait<0>();
        if (failed) {
            // A stage wait ran out: report it, and give the loads still in
            // flight a bounded chance to land before the CTA leaves.
            atomicOr(status, 1);
            int jj = j;
            for (int s = 0; s < ST; ++s, ++jj)
                if (pending & (1u << (jj % ST)))
                    gmmtma::mbar_wait(&full[jj % ST], (uint32_t)(jj / ST) & 1u);
        }
    }
}

// Launch set-up of one staged instance on one device: the dynamic shared
// memory limit is a per-device attribute of the function, and the resident
// CTA count follows from it, so both are set and queried once per device
// (under a lock: two threads may make their first call together). A failed
// set-up is not remembered; the next call tries again.
constexpr int kMaxDevices = 64;

template <int M, int PREC, int ST>
cudaError_t staged_ctas_per_sm(size_t smem, int *out) {
    static std::mutex mu;
    static int max_per_sm[kMaxDevices] = {}; // 0: not set up on that device yet
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (max_per_sm[dev] == 0) {
        e = cudaFuncSetAttribute(k_tick_staged<M, PREC, ST>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tick_staged<M, PREC, ST>, kTile,
                                                          smem);
        if (e != cudaSuccess)
            return e;
        if (n < 1)
            return cudaErrorInvalidConfiguration;
        max_per_sm[dev] = n;
    }
    *out = max_per_sm[dev];
    return cudaSuccess;
}

template <int M, int PREC, int ST>
cudaError_t launch_staged_t(const CamView &cv, int ctas_per_sm, int *status, cudaStream_t s) {
    constexpr int EB = PREC == 0 ? 4 : 2;
    constexpr size_t smem = (size_t)ST * (kFields * M * kTile * EB + 6 * kTile);
    int max_per_sm = 1;
    cudaError_t e = staged_ctas_per_sm<M, PREC, ST>(smem, &max_per_sm);
    if (e != cudaSuccess)
        return e;
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < max_per_sm) ? ctas_per_sm : max_per_sm;
    int64_t grid = (int64_t)gmmhost::num_sms() * per_sm;
    if (grid > cv.n_tiles)
        grid = cv.n_tiles;
    k_tick_staged<M, PREC, ST><<<(unsigned)grid, kTile, smem, s>>>(cv, status);
    return cudaGetLastError();
}

template <int PREC, int ST>
cudaError_t launch_staged_m(const CamView &cv, int ctas, int *status, cudaStream_t s) {
    switch (cv.M) {
    case 3: return launch_staged_t<3, PREC, ST>(cv, ctas, status, s);
    case 4: return launch_staged_t<4, PREC, ST>(cv, ctas, status, s);
    case 5: return launch_staged_t<5, PREC, ST>(cv, ctas, status, s);
    }
    return cudaErrorInvalidValue;
}

template <int ST>
cudaError_t launch_staged_p(const CamView &cv, int ctas, int *status, cudaStream_t s) {
    return cv.prec == 0 ? launch_staged_m<0, ST>(cv, ctas, status, s)
                        : launch_staged_m<1, ST>(cv, ctas, status, s);
}

} // namespace

namespace gmmhost {

// Self-test of the bounded wait: one thread waits on an mbarrier whose
// phase can never complete (it expects 16 bytes that no copy delivers). The
// wait must give up after limit_ns, set bit 0 of *status, record how long it
// waited, and the kernel must return normally.
__global__ void k_wait_selftest(int *status, unsigned long long *waited_ns,
                                unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0)
        return;
    gmmtma::mbar_init(&bar, 1);
    gmmtma::fence_mbar_init();
    gmmtma::mbar_arrive_expect_tx(&bar, 16);
    const uint64_t t0 = gmmtma::global_ns();
    const bool ok = gmmtma::mbar_wait(&bar, 0, limit_ns);
    *waited_ns = gmmtma::global_ns() - t0;
    if (!ok)
        atomicOr(status, 1);
    gmmtma::mbar_inval(&bar);
}

cudaError_t launch_wait_selftest(int *status, unsigned long long *waited_ns,
                                 unsigned long long limit_ns, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, waited_ns, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_tick_staged(const CamView &cv_in, int variant, int ctas_per_sm, int *status,
                               cudaStream_t s) {
    if (cv_in.n_pad == 0)
        return cudaSuccess;
    CamView cv = cv_in;
    // Frame bytes are staged with the state when every tile's slice of them
    // is contiguous and 16-byte aligned: unpadded rows and aligned bases.
    if (cv.W == cv.w_pad && reinterpret_cast<uintptr_t>(cv.rgb) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(cv.depth) % 16 == 0)
        cv.flags |= kStageInputs;
    switch (variant) {
    case 0: return launch_staged_p<2>(cv, ctas_per_sm, status, s);
    case 1: return launch_staged_p<3>(cv, ctas_per_sm, status, s);
    case 2: return launch_staged_p<4>(cv, ctas_per_sm, status, s);
    case 3: return launch_staged_p<5>(cv, ctas_per_sm, status, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace gmmhost
