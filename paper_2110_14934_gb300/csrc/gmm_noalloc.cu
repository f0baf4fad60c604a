// Allocation-free variant of the tick followed by the 3x3 opening.
//
// The regular path (a handle created with morph_open = 1) keeps the fused
// mask before the opening in a buffer the handle allocates. Here that
// intermediate mask lives in a fixed array of device memory that is part of
// the library image, so a call performs no allocation of any kind: the model
// state, the frame and the output mask all come from the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gmm.h"
#include "gmm_common.h"
#include "gmm_internal.h"

using namespace gmmlib;

// Every device that loads the library holds this array until the process
// exits. All calls share it.
static __device__ __align__(256) uint32_t g_noalloc_mask[GMM_NOALLOC_MAX_MASK_WORDS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint32_t *g_scratch[kMaxDevices] = {};

// Device address of g_noalloc_mask for the current device. The array's name
// in host code is only a host-side stand-in, so the address must come from
// the runtime, once per device, with that device current.
int scratch_for_current_device(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(nullptr, e, "gmm_apply_open3_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_mask);
        if (e != cudaSuccess || !ptr)
            return cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "gmm_apply_open3_noalloc: cudaGetSymbolAddress");
        g_scratch[dev] = static_cast<uint32_t *>(ptr);
    }
    *out = g_scratch[dev];
    return GMM_OK;
}

} // namespace

extern "C" int gmm_apply_open3_noalloc(const gmm_config *cfg, void *state, int first,
                                       const uint8_t *rgb8, const uint16_t *depth16,
                                       uint32_t *mask_out, void *stream) {
    const std::string msg = check_config(cfg);
    if (!msg.empty())
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: " + msg);
    const int wpr = (cfg->W + 31) / 32;
    if ((int64_t)cfg->H * wpr > (int64_t)GMM_NOALLOC_MAX_MASK_WORDS)
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: H * ceil(W/32) exceeds "
                                "GMM_NOALLOC_MAX_MASK_WORDS (the fixed scratch size)");
    if (first != 0 && first != 1)
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: first must be 0 or 1");
    if (cfg->flags & GMM_FLAG_STOCHASTIC_WEIGHTS)
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: GMM_FLAG_STOCHASTIC_WEIGHTS needs a "
                                "tick count (use a handle)");
    if (!state || reinterpret_cast<uintptr_t>(state) % 16)
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: state must be non-NULL and 16-byte aligned");
    std::string p = check_frame_ptrs(rgb8, depth16, mask_out, nullptr, nullptr);
    if (p.empty() && !device_accessible(state))
        p = "state must be device-accessible";
    if (!p.empty())
        return fail(GMM_EINVAL, "gmm_apply_open3_noalloc: " + p);
    uint32_t *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != GMM_OK)
        return rc;
    const Layout L = make_layout(cfg->H, cfg->W, cfg->M, cfg->precision);
    const gmmdev::CamView v = make_view(*cfg, L, state, rgb8, depth16, scratch, nullptr,
                                        nullptr, first, 0u);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = gmmhost::launch_tick(v, gmmhost::direct_threads(0, cfg->precision), s);
    if (e == cudaSuccess)
        e = gmmhost::launch_morph_open3(scratch, mask_out, cfg->H, cfg->W, s);
    if (e != cudaSuccess)
        return cuda_fail(nullptr, e, "gmm_apply_open3_noalloc launch");
    return GMM_OK;
}
