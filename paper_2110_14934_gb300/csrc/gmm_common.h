// Host helpers shared by the single-camera and the pool entry points.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "gmm.h"
#include "gmm_device.cuh"

namespace gmmlib {

extern thread_local std::string g_err;

int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t *sticky, cudaError_t e, const char *what);

// An NVTX range over the scope (one per host entry point that queues a
// tick), so profilers can group each tick's launches and copies; without a
// profiler attached it costs one predictable branch.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Makes `dev` current for the scope and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// Device layout of one camera's state (tiles of planes, see gmm_device.cuh).
struct Layout {
    int w_pad = 0, wpr = 0, elem = 4, planes_per_tile = 0;
    int64_t n_pad = 0, n_tiles = 0;
    size_t tile_bytes = 0, planes_bytes = 0, fusion_bytes = 0, total = 0;
};
Layout make_layout(int H, int W, int M, int prec);

std::string check_config(const gmm_config *c);
gmmdev::StreamPrm stream_prm(const gmm_config &c, bool depth);
gmmdev::CamView make_view(const gmm_config &c, const Layout &L, void *arena,
                          const uint8_t *rgb, const uint16_t *depth, uint32_t *mask,
                          uint32_t *fgr, uint32_t *fgd, int first, uint32_t tick);
bool device_accessible(const void *p);
std::string check_frame_ptrs(const uint8_t *rgb, const uint16_t *depth, uint32_t *mask,
                             uint32_t *fgr, uint32_t *fgd);
int state_get_common(const gmm_config &c, const Layout &L, const void *arena,
                     cudaStream_t stream, cudaError_t *sticky, int plane, int comp, float *dst,
                     size_t n);
int state_set_common(const gmm_config &c, const Layout &L, void *arena, cudaStream_t stream,
                     cudaError_t *sticky, int plane, int comp, const float *src, size_t n);
int wait_event(cudaEvent_t ev, int timeout_ms, cudaError_t *sticky, const char *what);

// A stream-ordered memory pool on `device` that keeps up to `keep_bytes` of
// freed memory mapped (the default pool returns it to the system at the next
// synchronisation, so cameras that join later would pay for mapping again).
cudaError_t make_retaining_pool(int device, uint64_t keep_bytes, cudaMemPool_t *out);
// Allocates `bytes` from the pool on stream s and frees it again, then waits:
// the pool keeps that memory mapped (up to its release threshold), so later
// allocations of up to that much take it without mapping new pages.
cudaError_t reserve_in_pool(cudaMemPool_t pool, size_t bytes, cudaStream_t s);

} // namespace gmmlib
