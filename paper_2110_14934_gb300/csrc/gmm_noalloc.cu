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
// exits (under lazy module loading, from the first call on that device on).
// All calls share it.
static __device__ __align__(256) uint32_t g_noalloc_mask[GMM_NOALLOC_MAX_MASK_WORDS];

namespace {

// Context of the calling thread, through the driver API entry points the
// runtime hands out (no link against libcuda). A context id is unique for
// the life of the process: a context made after cudaDeviceReset, or a
// non-primary context a driver-API caller made current, gets a new one.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
std::once_flag g_entry_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

void load_entry_points() {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(fn);
}

// Id of the context current on this thread; false if there is none or the
// driver cannot say.
bool current_context_id(unsigned long long *id) {
    std::call_once(g_entry_once, load_entry_points);
    if (!g_ctx_get_current || !g_ctx_get_id)
        return false;
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx)
        return false;
    return g_ctx_get_id(ctx, id) == 0;
}

// Addresses of g_noalloc_mask already looked up, keyed by context id (the
// address belongs to one context: each context loads its own copy of the
// module that holds the array).
constexpr int kCacheSlots = 64;
std::mutex g_setup_mu;
unsigned long long g_ctx_ids[kCacheSlots] = {};
uint32_t *g_scratch[kCacheSlots] = {};
int g_next_slot = 0;

// Device address of g_noalloc_mask in the calling thread's current context.
// The array's name in host code is only a host-side stand-in, so the address
// comes from the runtime, once per context, with that context current. The
// lookup also makes the runtime set up the device's primary context when no
// context is current yet, so the id is taken after it.
int scratch_for_current_context(uint32_t **out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    unsigned long long id = 0;
    if (current_context_id(&id)) {
        for (int i = 0; i < kCacheSlots; ++i) {
            if (g_scratch[i] && g_ctx_ids[i] == id) {
                *out = g_scratch[i];
                return GMM_OK;
            }
        }
    }
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_mask);
    if (e != cudaSuccess || !ptr)
        return cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                         "gmm_apply_open3_noalloc: cudaGetSymbolAddress");
    *out = static_cast<uint32_t *>(ptr);
    if (current_context_id(&id)) {
        g_ctx_ids[g_next_slot] = id;
        g_scratch[g_next_slot] = *out;
        g_next_slot = (g_next_slot + 1) % kCacheSlots;
    }
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
    int rc = scratch_for_current_context(&scratch);
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
