// Multi-camera tick: one launch advances every camera of a pool that has a
// submitted frame (up to kPoolViews cameras per launch), with the per-pixel
// arithmetic of the single-camera kernel (gmm_device.cuh), in a persistent
// form (CTAs loop over tiles) or a flat one (one chunk per warp); and the
// per-device argument bank their launches share.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gmm_internal.h"

using namespace gmmdev;
using gmmhost::PoolArgs;

namespace {

// ------------------------------------------------------------ kernel
// CTAs take tiles of the implicit worklist (PoolArgs) from an atomic counter;
// the camera of a tile is found by binary search over tile_begin. The
// launch's PoolArgs sit in constant memory (uploaded before each launch), so
// the views are read from the constant bank where they are used and hold no
// registers across a pixel's arithmetic.
__constant__ PoolArgs c_pool;
template <int M, int PREC, int V>
__device__ __forceinline__ void pool_tile(const CamView &cv, int64_t p0, int64_t p1) {
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        // p1 - p0 is a multiple of 32 and blockDim too: warps stay whole.
        const uint32_t bits = process_pixel<M, PREC, true, V>(cv, p);
        write_mask_words(cv, p >> 5, bits);
    }
}

template <int M, int PREC, bool kAll>
__device__ __forceinline__ void pool_tile_v(const CamView &cv, int64_t p0, int64_t p1) {
    if (!kAll) {
        pool_tile<M, PREC, 0>(cv, p0, p1);
        return;
    }
    switch (gmmhost::view_variant(cv)) {
    case 0: pool_tile<M, PREC, 0>(cv, p0, p1); break;
    case 1: pool_tile<M, PREC, 1>(cv, p0, p1); break;
    default: pool_tile<M, PREC, 2>(cv, p0, p1); break;
    }
}

// Camera of tile t: the last job with tile_begin <= t (0 past the end).
__device__ __forceinline__ int tile_job(const PoolArgs &a, int64_t t) {
    int lo = 0, hi = a.n_jobs - 1;
    if (t < a.n_tiles) {
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.tile_begin[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
    }
    return lo;
}

// Bulk prefetch of [p, p + bytes) into L2 (a hint: nothing waits for it);
// p and bytes multiples of 16.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 bytes the prefetched next tiles of all CTAs may hold together (state
// and List-1 bytes): each CTA prefetches the first pixels of its next tile,
// as many whole 256-pixel state tiles as its share of this budget holds (at
// least one). Past about this much, prefetched lines are evicted before their
// loads arrive and the data crosses HBM twice.
constexpr int64_t kPrefetchBudget = 16ll << 20;

// Prefetch the state and List-1 bytes of the first pixels of tile t (camera
// job) into L2. The state is whole 256-pixel state tiles, one contiguous block
// of the camera's allocation (which holds every state tile up to n_tiles);
// the List-1 bytes start at a multiple of 32 and number a multiple of 32.
template <int PREC>
__device__ __forceinline__ void prefetch_tile(const PoolArgs &a, int64_t t, int job) {
    const CamView &v = a.views[job];
    const int64_t tile_bytes = (int64_t)kFields * v.M * kTile * (PREC == 0 ? 4 : 2);
    const int64_t share = kPrefetchBudget / gridDim.x / (tile_bytes + kTile);
    const int64_t q0 = (t - a.tile_begin[job]) * a.tile_pixels;
    const int64_t s0 = q0 / kTile;
    const int64_t q1 = min(min(q0 + (int64_t)a.tile_pixels, v.n_pad),
                           (s0 + max(share, (int64_t)1)) * kTile);
    const int64_t s1 = (q1 + kTile - 1) / kTile;
    prefetch_l2(static_cast<const char *>(v.planes) + s0 * tile_bytes,
                (uint32_t)((s1 - s0) * tile_bytes));
    prefetch_l2(v.fusion + q0, (uint32_t)(q1 - q0));
}

// Take the CTA's next tile from the counter into slot `slot` (thread 0),
// prefetching its first pixels' state when asked.
template <int PREC>
__device__ __forceinline__ void take_next(const PoolArgs &a, int64_t *s_tile, int *s_job,
                                          int slot, bool prefetch) {
    const int64_t tn = atomicAdd(a.counter, 1);
    const int jn = tile_job(a, tn);
    s_tile[slot] = tn;
    s_job[slot] = jn;
    if (prefetch && tn < a.n_tiles)
        prefetch_tile<PREC>(a, tn, jn);
}

// kAll: tiles may come from cameras that use the options or the
// augmentation alternative (launched only when such a camera is in the tick).
// Registers: 64 in both precisions (32 resident warps per SM; FP32 at 72,
// 28 warps, measured 0.8% slower on the 64-camera mix), except the FP32
// instance that also handles the options, which keeps room to avoid spills.
// FP32 state, the instance that also handles the options, and FP16/BF16
// pools that turned the prefetch off (kPF = false): thread 0 takes a tile
// from the counter and publishes it between two barriers. Otherwise, in
// FP16/BF16 state (kPrefetch): a CTA's current and next tile (and camera) sit
// in alternate slots; thread 0 takes the next tile at the end of the current
// one, or, for tiles of at most two pixels per thread while at least two
// waves of tiles remain beyond the current one, at its start, and then
// prefetches the next tile's first pixels' state into L2, so those loads
// find the data on chip (with FP16/BF16 state the bytes a warp keeps in
// flight in its registers do not cover HBM latency). Taken early near the
// end of the worklist, a CTA would hold two tiles while others run out of
// work; with more pixels per thread per tile, and with FP32 state
// (HBM-bound), prefetching measured slower. One barrier per tile; slot k ^ 1
// is written only after the barrier that ended the tile at whose start every
// thread last read it.
template <int PREC, bool kAll, bool kPF = true>
__global__ void __launch_bounds__(256, (PREC == 0 && kAll) ? 3 : 4) k_pool_tick() {
    constexpr bool kPrefetch = PREC != 0 && !kAll && kPF;
    const PoolArgs &a = c_pool;
    __shared__ int64_t s_tile[2];
    __shared__ int s_job[2];
    if (blockIdx.x == 0) // the next tick's counters (their last users have finished)
        for (int i = threadIdx.x; i < a.n_reset; i += blockDim.x)
            a.reset[i] = 0;
    if constexpr (!kPrefetch) {
        for (;;) { // take a tile, publish it, read it, barrier (slot 0 is rewritten)
            if (threadIdx.x == 0)
                take_next<PREC>(a, s_tile, s_job, 0, false);
            __syncthreads();
            const int64_t t = s_tile[0];
            const int job = s_job[0];
            __syncthreads();
            if (t >= a.n_tiles)
                return;
            const CamView &cv = a.views[job];
            const int64_t p0 = (t - a.tile_begin[job]) * a.tile_pixels;
            const int64_t p1 = min(p0 + (int64_t)a.tile_pixels, cv.n_pad);
            switch (cv.M) {
            case 3: pool_tile_v<3, PREC, kAll>(cv, p0, p1); break;
            case 4: pool_tile_v<4, PREC, kAll>(cv, p0, p1); break;
            default: pool_tile_v<5, PREC, kAll>(cv, p0, p1); break;
            }
        }
    }
    if (threadIdx.x == 0)
        take_next<PREC>(a, s_tile, s_job, 0, false);
    __syncthreads();
    for (int k = 0;; k ^= 1) {
        const int64_t t = s_tile[k];
        const int job = s_job[k];
        if (t >= a.n_tiles)
            return;
        const bool early = a.tile_pixels <= 2 * (int)blockDim.x &&
                           t + 2 * (int64_t)gridDim.x < a.n_tiles;
        if (early && threadIdx.x == 0)
            take_next<PREC>(a, s_tile, s_job, k ^ 1, true);
        const CamView &cv = a.views[job];
        const int64_t p0 = (t - a.tile_begin[job]) * a.tile_pixels;
        const int64_t p1 = min(p0 + (int64_t)a.tile_pixels, cv.n_pad);
        switch (cv.M) {
        case 3: pool_tile_v<3, PREC, kAll>(cv, p0, p1); break;
        case 4: pool_tile_v<4, PREC, kAll>(cv, p0, p1); break;
        default: pool_tile_v<5, PREC, kAll>(cv, p0, p1); break;
        }
        if (!early && threadIdx.x == 0)
            take_next<PREC>(a, s_tile, s_job, k ^ 1, false);
        __syncthreads();
    }
}

// Non-persistent form: every warp takes one chunk of the launch's implicit
// chunk list (tile_begin counts chunks here: 32 pixels in FP32, one per lane;
// 64 in FP16/BF16, two per lane with the second pixel's loads overlapping
// the first one's arithmetic, as in the single-camera kernels) and finds its
// camera by binary search. No counter and no loop: a CTA's slot frees as soon
// as its own warps finish, and no registers carry a loop across pixels.
template <int M, int PREC, int V>
__device__ __forceinline__ void flat_chunk(const CamView &cv, int64_t base) {
    const int lane = threadIdx.x & 31;
    if constexpr (PREC == 0) { // n_pad is a multiple of 32: the chunk is whole
        const int64_t p = base + lane;
        write_mask_words(cv, p >> 5, process_pixel<M, PREC, true, V>(cv, p));
    } else {
        uint32_t bits[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t p = base + 32 * u + lane;
            bits[u] = p < cv.n_pad ? process_pixel<M, PREC, true, V>(cv, p) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (base + 32 * u < cv.n_pad)
                write_mask_words(cv, (base >> 5) + u, bits[u]);
    }
}

template <int M, int PREC, bool kAll>
__device__ __forceinline__ void flat_chunk_v(const CamView &cv, int64_t base) {
    if (!kAll) {
        flat_chunk<M, PREC, 0>(cv, base);
        return;
    }
    switch (gmmhost::view_variant(cv)) {
    case 0: flat_chunk<M, PREC, 0>(cv, base); break;
    case 1: flat_chunk<M, PREC, 1>(cv, base); break;
    default: flat_chunk<M, PREC, 2>(cv, base); break;
    }
}

// MM: every camera of the launch has M = MM (the host groups the flat
// form's launches by M, so each runs a body specialised to its M), or 0
// (any M, switched per warp). FP32: no residency hint; FP16/BF16: 64
// registers, as in the other kernels.
template <int PREC, bool kAll, int MM>
__global__ void __launch_bounds__(256, PREC == 0 ? 1 : 4) k_pool_flat() {
    const PoolArgs &a = c_pool;
    if (blockIdx.x == 0) // the next tick's counters, as the persistent form does
        for (int i = threadIdx.x; i < a.n_reset; i += blockDim.x)
            a.reset[i] = 0;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= a.n_tiles)
        return;
    int lo = 0, hi = a.n_jobs - 1;
    while (lo < hi) { // last job with tile_begin <= c (uniform across the warp)
        const int mid = (lo + hi + 1) >> 1;
        if (a.tile_begin[mid] <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    const CamView &cv = a.views[lo];
    const int64_t base = (c - a.tile_begin[lo]) * a.tile_pixels;
    if (MM != 0) {
        flat_chunk_v<MM != 0 ? MM : 3, PREC, kAll>(cv, base);
        return;
    }
    switch (cv.M) {
    case 3: flat_chunk_v<3, PREC, kAll>(cv, base); break;
    case 4: flat_chunk_v<4, PREC, kAll>(cv, base); break;
    default: flat_chunk_v<5, PREC, kAll>(cv, base); break;
    }
}

template <int PREC, bool kAll>
void launch_flat(int m, int blocks, int threads, cudaStream_t s) {
    switch (m) {
    case 3: k_pool_flat<PREC, kAll, 3><<<blocks, threads, 0, s>>>(); break;
    case 4: k_pool_flat<PREC, kAll, 4><<<blocks, threads, 0, s>>>(); break;
    case 5: k_pool_flat<PREC, kAll, 5><<<blocks, threads, 0, s>>>(); break;
    default: k_pool_flat<PREC, kAll, 0><<<blocks, threads, 0, s>>>(); break;
    }
}

} // namespace

namespace gmmhost {

// The argument bank is one per device: launches of different pools (other
// streams, other threads) take turns through a lock and an event that
// orders each bank user after the previous one on the GPU.
namespace {
struct BankGuard {
    std::mutex mu;
    cudaEvent_t last = nullptr;
};
BankGuard g_bank[64];
} // namespace

cudaError_t pool_bank_acquire(int device, cudaStream_t s) {
    if (device < 0 || device >= 64)
        return cudaErrorInvalidDevice;
    BankGuard &g = g_bank[device];
    g.mu.lock();
    cudaError_t e = cudaSuccess;
    if (!g.last)
        e = cudaEventCreateWithFlags(&g.last, cudaEventDisableTiming);
    else
        e = cudaStreamWaitEvent(s, g.last, 0);
    if (e != cudaSuccess)
        g.mu.unlock();
    return e;
}

cudaError_t pool_bank_release(int device, cudaStream_t s) {
    BankGuard &g = g_bank[device];
    const cudaError_t e = cudaEventRecord(g.last, s);
    g.mu.unlock();
    return e;
}

cudaError_t launch_pool_tick_impl(const PoolArgs *args_host, int threads, int blocks, int prec,
                                  bool all_variants, bool flat, int m, bool prefetch,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemcpyToSymbolAsync(c_pool, args_host, sizeof(PoolArgs), 0,
                                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return e;
    if (flat) {
        if (prec == 0 && !all_variants)
            launch_flat<0, false>(m, blocks, threads, s);
        else if (prec == 0)
            launch_flat<0, true>(m, blocks, threads, s);
        else if (!all_variants)
            launch_flat<1, false>(m, blocks, threads, s);
        else
            launch_flat<1, true>(m, blocks, threads, s);
    } else if (prec == 0 && !all_variants)
        k_pool_tick<0, false><<<blocks, threads, 0, s>>>();
    else if (prec == 0)
        k_pool_tick<0, true><<<blocks, threads, 0, s>>>();
    else if (!all_variants && prefetch)
        k_pool_tick<1, false><<<blocks, threads, 0, s>>>();
    else if (!all_variants)
        k_pool_tick<1, false, false><<<blocks, threads, 0, s>>>();
    else
        k_pool_tick<1, true><<<blocks, threads, 0, s>>>();
    return cudaGetLastError();
}

int pool_max_ctas_per_sm(int prec, int threads) {
    int n = 0;
    cudaError_t e = prec == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pool_tick<0, false>, threads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pool_tick<1, false>, threads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

} // namespace gmmhost
