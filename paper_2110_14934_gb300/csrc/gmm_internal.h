// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmm_device.cuh"

namespace gmmhost {

// Single-camera tick: one thread per padded pixel. threads: block size (32,
// 64, 128 or 256).
cudaError_t launch_tick(const gmmdev::CamView &cv, int threads, cudaStream_t s);

// Block size of the direct tick kernel for gmm_set_kernel's variant: 0 the
// measured best for the storage precision (FP32: 128; FP16/BF16: 64, two
// warps of two pixels per thread), 1..4: 256, 128, 64, 32.
inline int direct_threads(int variant, int prec) {
    switch (variant) {
    case 1: return 256;
    case 2: return 128;
    case 3: return 64;
    case 4: return 32;
    default: return prec == 0 ? 128 : 64;
    }
}

// Staged single-camera tick (bulk-copy pipeline through shared memory).
// variant: pipeline depth (0..3: 2..5 stages of one 256-pixel tile);
// ctas_per_sm: 0 = as many as fit. status: device word that
// gets bit 0 set if a pipeline wait runs out. Not for first ticks.
cudaError_t launch_tick_staged(const gmmdev::CamView &cv, int variant, int ctas_per_sm,
                               int *status, cudaStream_t s);

// Bounded-wait self-test (see gmm_wait_selftest): *status gets bit 0 when
// the wait ran out; *waited_ns the time waited.
cudaError_t launch_wait_selftest(int *status, unsigned long long *waited_ns,
                                 unsigned long long limit_ns, cudaStream_t s);

// Byte mask -> bit-packed mask; confusion counts {TP, FP, FN, TN} of two
// bit-packed masks into out (zeroed first).
cudaError_t launch_pack(const uint8_t *in, uint32_t *out, int H, int W, cudaStream_t s);
cudaError_t launch_confusion(const uint32_t *pred, const uint32_t *truth, int H, int W,
                             unsigned long long *out, cudaStream_t s);

// List 1 alone over bit-packed inputs.
cudaError_t launch_fuse(const uint32_t *fg_rgb, const uint32_t *fg_d, uint8_t *fusion,
                        uint32_t *mask, int H, int W, cudaStream_t s);

// 3x3 opening of a bit-packed mask.
cudaError_t launch_morph_open3(const uint32_t *in, uint32_t *out, int H, int W,
                               cudaStream_t s);

// Multi-camera persistent tick. The worklist is implicit: job j covers tiles
// [tile_begin[j], tile_begin[j+1]) of camera views[j], tile_pixels pixels
// each (the last one of a camera ragged). A launch handles up to kPoolViews
// cameras (a tick with more is split into several launches); its PoolArgs
// are copied into the kernel's constant memory on the stream right before
// it. *counter must be zero at launch; the launch zeroes the n_reset
// counters at reset (the next tick's).
constexpr int kPoolViews = 128;
struct PoolArgs {
    gmmdev::CamView views[kPoolViews];
    int64_t tile_begin[kPoolViews + 1];
    int *counter;
    int *reset;
    int n_reset;
    int n_jobs;
    int tile_pixels;
    int64_t n_tiles;
};
static_assert(sizeof(PoolArgs) <= 32768, "one launch's arguments fit half the constant bank");

// Upload *args_host (page-locked for an asynchronous copy) to the kernel's
// constant memory and launch the pool kernel; all_variants: the instance
// that also handles the options and the augmentation alternative; flat: the
// non-persistent form (tile_begin and n_tiles count one chunk per warp:
// 32 pixels in FP32, 64 in FP16/BF16; blocks covers every chunk); m: the M
// every camera of the launch has (a kernel specialised to it), or 0;
// prefetch: the FP16/BF16 persistent instance that takes next tiles early
// and prefetches them into L2 (else the one that does not).
cudaError_t launch_pool_tick_impl(const PoolArgs *args_host, int threads, int blocks, int prec,
                                  bool all_variants, bool flat, int m, bool prefetch,
                                  cudaStream_t s);

// The constant-memory argument bank is shared by every pool on a device:
// enqueue uploads and launches between acquire (takes the device's lock and
// orders stream s after the bank's previous user) and release (records s as
// the last user, drops the lock). Not needed while capturing a graph.
cudaError_t pool_bank_acquire(int device, cudaStream_t s);
cudaError_t pool_bank_release(int device, cudaStream_t s);

// process_pixel variant a camera needs: 0 default, 1 learning-rate/variance
// options, 2 augmentation alternative.
__host__ __device__ inline int view_variant(const gmmdev::CamView &cv) {
    if (cv.flags & gmmdev::kModeAugmented)
        return 2;
    return ((cv.pc.flags | cv.pd.flags) || (cv.flags & gmmdev::kStochasticWeights)) ? 1 : 0;
}

int num_sms();

} // namespace gmmhost
