// Multi-camera persistent tick: one launch advances every camera of a pool
// that has a submitted frame (up to kPoolViews cameras per launch), with the
// per-pixel arithmetic of the single-camera kernel (gmm_device.cuh), and the
// per-device argument bank its launches share.
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

// kAll: tiles may come from cameras that use the options or the
// augmentation alternative (launched only when such a camera is in the tick).
template <int PREC, bool kAll>
__global__ void __launch_bounds__(256, PREC == 0 ? 3 : 4) k_pool_tick() {
    const PoolArgs &a = c_pool;
    __shared__ int64_t s_tile;
    __shared__ int s_job;
    if (blockIdx.x == 0) // the next tick's counters (their last users have finished)
        for (int i = threadIdx.x; i < a.n_reset; i += blockDim.x)
            a.reset[i] = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t t = atomicAdd(a.counter, 1);
            int lo = 0, hi = a.n_jobs - 1;
            if (t < a.n_tiles) {
                while (lo < hi) { // last job with tile_begin <= t
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.tile_begin[mid] <= t)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
            }
            s_tile = t;
            s_job = lo;
        }
        __syncthreads();
        const int64_t t = s_tile;
        const int job = s_job;
        __syncthreads(); // s_tile and s_job are rewritten next round
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
                                  bool all_variants, cudaStream_t s) {
    cudaError_t e = cudaMemcpyToSymbolAsync(c_pool, args_host, sizeof(PoolArgs), 0,
                                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return e;
    if (prec == 0 && !all_variants)
        k_pool_tick<0, false><<<blocks, threads, 0, s>>>();
    else if (prec == 0)
        k_pool_tick<0, true><<<blocks, threads, 0, s>>>();
    else if (!all_variants)
        k_pool_tick<1, false><<<blocks, threads, 0, s>>>();
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
