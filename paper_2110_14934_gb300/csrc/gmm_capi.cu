// C ABI of the single-camera model: argument checks, device state ownership,
// launches, state transfer and the pipelined host-memory path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "gmm.h"
#include "gmm_common.h"
#include "gmm_internal.h"

using gmmdev::CamView;

namespace gmmlib {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t *sticky, cudaError_t e, const char *what) {
    if (sticky && *sticky == cudaSuccess)
        *sticky = e;
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return GMM_ECUDA;
}

DeviceGuard::DeviceGuard(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && dev >= 0) {
        cudaSetDevice(dev);
        prev = cur;
    }
}
DeviceGuard::~DeviceGuard() {
    if (prev >= 0)
        cudaSetDevice(prev);
}

Layout make_layout(int H, int W, int M, int prec) {
    Layout L;
    L.w_pad = ((W + 31) / 32) * 32;
    L.wpr = L.w_pad / 32;
    L.n_pad = (int64_t)H * L.w_pad;
    L.elem = prec == GMM_PREC_F32 ? 4 : 2;
    L.n_tiles = (L.n_pad + gmmdev::kTile - 1) / gmmdev::kTile;
    L.planes_per_tile = M * gmmdev::kFields;
    L.tile_bytes = (size_t)L.planes_per_tile * gmmdev::kTile * L.elem;
    L.planes_bytes = (size_t)L.n_tiles * L.tile_bytes;
    L.fusion_bytes = (size_t)L.n_tiles * gmmdev::kTile;
    L.total = L.planes_bytes + L.fusion_bytes;
    return L;
}

std::string check_config(const gmm_config *c) {
    if (!c)
        return "null configuration";
    if (c->H < 1 || c->W < 1)
        return "H and W must be >= 1";
    if ((int64_t)c->H * (((int64_t)c->W + 31) / 32) * 32 > (int64_t(1) << 30))
        return "frame too large (more than 2^30 padded pixels)";
    if (c->M < 3 || c->M > 5)
        return "M must be in [3, 5]";
    if (!(c->alpha > 0.f && c->alpha < 1.f))
        return "alpha must be in (0, 1)";
    if (!(c->match_k > 0.f) || !std::isfinite(c->match_k))
        return "match_k must be a finite value > 0";
    if (!(c->bg_T > 0.f && c->bg_T < 1.f))
        return "bg_T must be in (0, 1)";
    if (!(c->init_var > 0.f) || !std::isfinite(c->init_var))
        return "init_var must be a finite value > 0";
    if (!(c->init_w > 0.f && c->init_w < 1.f))
        return "init_w must be in (0, 1)";
    if (!(c->init_var_d > 0.f) || !std::isfinite(c->init_var_d))
        return "init_var_d must be a finite value > 0";
    if (!(c->v_min_c > 0.f) || !std::isfinite(c->v_min_c) || !(c->v_min_d > 0.f) ||
        !std::isfinite(c->v_min_d))
        return "variance floors must be finite values > 0";
    if (c->precision != GMM_PREC_F32 && c->precision != GMM_PREC_F16)
        return "precision must be GMM_PREC_F32 or GMM_PREC_F16";
    if (c->morph_open != 0 && c->morph_open != 1)
        return "morph_open must be 0 or 1";
    if (c->mode != GMM_MODE_FUSION && c->mode != GMM_MODE_AUGMENTED)
        return "mode must be GMM_MODE_FUSION or GMM_MODE_AUGMENTED";
    if (!(c->depth_scale > 0.f) || !std::isfinite(c->depth_scale))
        return "depth_scale must be a finite value > 0";
    if (c->flags & ~(GMM_FLAG_RHO_ETA | GMM_FLAG_VAR_PER_CHANNEL | GMM_FLAG_STOCHASTIC_WEIGHTS))
        return "flags: unknown bits";
    if ((c->flags & GMM_FLAG_STOCHASTIC_WEIGHTS) && c->precision != GMM_PREC_F16)
        return "GMM_FLAG_STOCHASTIC_WEIGHTS needs GMM_PREC_F16 state";
    return "";
}

gmmdev::StreamPrm stream_prm(const gmm_config &c, bool depth) {
    gmmdev::StreamPrm p;
    p.alpha = c.alpha;
    p.oma = 1.0f - c.alpha;
    p.k2 = c.match_k * c.match_k;
    p.T = c.bg_T;
    p.init_var = depth ? c.init_var_d : c.init_var;
    p.init_w = c.init_w;
    p.v_min = depth ? c.v_min_d : c.v_min_c;
    p.flags = c.flags & (gmmdev::kRhoEta | gmmdev::kVarPerChannel);
    return p;
}

CamView make_view(const gmm_config &c, const Layout &L, void *arena, const uint8_t *rgb,
                  const uint16_t *depth, uint32_t *mask, uint32_t *fgr, uint32_t *fgd,
                  int first, uint32_t tick) {
    CamView v;
    std::memset(&v, 0, sizeof(v));
    v.planes = arena;
    v.fusion = static_cast<uint8_t *>(arena) + L.planes_bytes;
    v.rgb = rgb;
    v.depth = depth;
    v.mask = mask;
    v.fg_rgb = fgr;
    v.fg_d = fgd;
    v.n_tiles = L.n_tiles;
    v.n_pad = L.n_pad;
    v.H = c.H;
    v.W = c.W;
    v.w_pad = L.w_pad;
    v.wpr = L.wpr;
    v.M = c.M;
    v.prec = c.precision;
    v.first = first;
    if (L.wpr > 1) {
        uint32_t l = 0;
        while ((1u << l) < (uint32_t)L.wpr)
            ++l; // l = ceil(log2(wpr)) >= 1
        v.wpr_mul = (uint32_t)(((1ull << (31 + l)) + (uint64_t)L.wpr - 1) / (uint64_t)L.wpr);
        v.wpr_shift = l - 1;
    }
    v.pc = stream_prm(c, false);
    v.pd = stream_prm(c, true);
    if (c.mode == GMM_MODE_AUGMENTED)
        v.flags |= gmmdev::kModeAugmented;
    if (c.flags & GMM_FLAG_STOCHASTIC_WEIGHTS)
        v.flags |= gmmdev::kStochasticWeights;
    v.depth_scale = c.depth_scale;
    v.tick = tick;
    return v;
}

bool device_accessible(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return true;
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

std::string check_frame_ptrs(const uint8_t *rgb, const uint16_t *depth, uint32_t *mask,
                             uint32_t *fgr, uint32_t *fgd) {
    if (!rgb || !depth || !mask)
        return "rgb8, depth16 and mask_out must not be NULL";
    if (reinterpret_cast<uintptr_t>(depth) % 2)
        return "depth16 must be 2-byte aligned";
    if (reinterpret_cast<uintptr_t>(mask) % 4 || reinterpret_cast<uintptr_t>(fgr) % 4 ||
        reinterpret_cast<uintptr_t>(fgd) % 4)
        return "mask pointers must be 4-byte aligned";
    if (!device_accessible(rgb) || !device_accessible(depth) || !device_accessible(mask) ||
        (fgr && !device_accessible(fgr)) || (fgd && !device_accessible(fgd)))
        return "frame and mask pointers must be device-accessible";
    return "";
}

// Host-side conversion of one plane between the device layout (padded rows,
// storage type) and row-major floats. src/dst hold the plane's value of
// padded pixel p at element p * stride + slot.
void plane_to_float(const void *src, int elem, bool weight, int stride, int slot,
                    const Layout &L, int H, int W, float *dst) {
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const int64_t p = ((int64_t)y * L.w_pad + x) * stride + slot;
            float v;
            if (elem == 4)
                v = static_cast<const float *>(src)[p];
            else if (weight)
                v = __bfloat162float(static_cast<const __nv_bfloat16 *>(src)[p]);
            else
                v = __half2float(static_cast<const __half *>(src)[p]);
            dst[(int64_t)y * W + x] = v;
        }
    }
}

// Writes the plane's values into dst (other slots untouched); padded pixels
// get 0.
void float_to_plane(const float *src, int elem, bool weight, int stride, int slot,
                    const Layout &L, int H, int W, void *dst) {
    for (int64_t q = 0; q < L.n_pad; ++q) {
        const int64_t y = q / L.w_pad, x = q % L.w_pad;
        const float v = (y < H && x < W) ? src[y * W + x] : 0.f;
        const int64_t p = q * stride + slot;
        if (elem == 4)
            static_cast<float *>(dst)[p] = v;
        else if (weight)
            static_cast<__nv_bfloat16 *>(dst)[p] = __float2bfloat16_rn(v);
        else
            static_cast<__half *>(dst)[p] = __float2half_rn(fminf(v, 65504.0f));
    }
}

// Where one plane lives: in every tile, a run of `run` bytes starting `off`
// bytes into the tile, holding its value of tile pixel t at element
// t * stride + slot (FP32: the plane itself; FP16/BF16: its group).
struct PlaneRun {
    size_t off, run;
    int stride, slot;
};
PlaneRun plane_run(const Layout &L, int comp, int plane) {
    PlaneRun r;
    if (L.elem == 4) {
        r.run = (size_t)gmmdev::kTile * 4;
        r.off = (size_t)gmmdev::tile_elem<0>(comp, plane, 0) * 4;
        r.stride = 1;
        r.slot = 0;
    } else {
        r.run = (size_t)gmmdev::kTile * 8;
        r.off = (size_t)gmmdev::tile_elem<1>(comp, plane, 0) / 4 * 8;
        r.stride = 4;
        r.slot = gmmdev::h16_slot(plane);
    }
    return r;
}

int state_get_common(const gmm_config &c, const Layout &L, const void *arena,
                     cudaStream_t stream, cudaError_t *sticky, int plane, int comp, float *dst,
                     size_t n) {
    if (!dst)
        return fail(GMM_EINVAL, "dst_host must not be NULL");
    if (n < (size_t)c.H * c.W)
        return fail(GMM_EINVAL, "n is smaller than H*W");
    if (plane < 0 || plane > GMM_PLANE_FUSION)
        return fail(GMM_EINVAL, "unknown plane");
    if (plane != GMM_PLANE_FUSION && (comp < 0 || comp >= c.M))
        return fail(GMM_EINVAL, "component out of range");
    if (plane == GMM_PLANE_FUSION) {
        std::vector<uint8_t> tmp((size_t)L.n_pad);
        const uint8_t *src = static_cast<const uint8_t *>(arena) + L.planes_bytes;
        cudaError_t e = cudaMemcpyAsync(tmp.data(), src, (size_t)L.n_pad, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess)
            return cuda_fail(sticky, e, "gmm_state_get");
        for (int y = 0; y < c.H; ++y)
            for (int x = 0; x < c.W; ++x)
                dst[(int64_t)y * c.W + x] = (float)tmp[(size_t)y * L.w_pad + x];
        return GMM_OK;
    }
    const bool weight = plane == GMM_PLANE_W_C || plane == GMM_PLANE_W_D;
    // The plane (or its group) is a run of bytes in every tile: a pitched copy.
    const PlaneRun r = plane_run(L, comp, plane);
    std::vector<uint8_t> tmp((size_t)L.n_tiles * r.run);
    const uint8_t *src = static_cast<const uint8_t *>(arena) + r.off;
    cudaError_t e = cudaMemcpy2DAsync(tmp.data(), r.run, src, L.tile_bytes, r.run,
                                      (size_t)L.n_tiles, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return cuda_fail(sticky, e, "gmm_state_get");
    plane_to_float(tmp.data(), L.elem, weight, r.stride, r.slot, L, c.H, c.W, dst);
    return GMM_OK;
}

int state_set_common(const gmm_config &c, const Layout &L, void *arena, cudaStream_t stream,
                     cudaError_t *sticky, int plane, int comp, const float *src, size_t n) {
    if (!src)
        return fail(GMM_EINVAL, "src_host must not be NULL");
    if (n < (size_t)c.H * c.W)
        return fail(GMM_EINVAL, "n is smaller than H*W");
    if (plane < 0 || plane > GMM_PLANE_FUSION)
        return fail(GMM_EINVAL, "unknown plane");
    if (plane != GMM_PLANE_FUSION && (comp < 0 || comp >= c.M))
        return fail(GMM_EINVAL, "component out of range");
    cudaError_t e;
    if (plane == GMM_PLANE_FUSION) {
        std::vector<uint8_t> tmp((size_t)L.n_pad, 0);
        for (int y = 0; y < c.H; ++y)
            for (int x = 0; x < c.W; ++x) {
                float v = src[(int64_t)y * c.W + x];
                v = v < 0.f ? 0.f : (v > 255.f ? 255.f : v);
                tmp[(size_t)y * L.w_pad + x] = (uint8_t)v;
            }
        uint8_t *dst = static_cast<uint8_t *>(arena) + L.planes_bytes;
        e = cudaMemcpyAsync(dst, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(stream);
    } else {
        const bool weight = plane == GMM_PLANE_W_C || plane == GMM_PLANE_W_D;
        const PlaneRun r = plane_run(L, comp, plane);
        std::vector<uint8_t> tmp((size_t)L.n_tiles * r.run, 0);
        uint8_t *dst = static_cast<uint8_t *>(arena) + r.off;
        e = cudaSuccess;
        if (r.stride > 1) // the group's other slots keep their values
            e = cudaMemcpy2DAsync(tmp.data(), r.run, dst, L.tile_bytes, r.run,
                                  (size_t)L.n_tiles, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) {
            float_to_plane(src, L.elem, weight, r.stride, r.slot, L, c.H, c.W, tmp.data());
            e = cudaMemcpy2DAsync(dst, L.tile_bytes, tmp.data(), r.run, r.run,
                                  (size_t)L.n_tiles, cudaMemcpyHostToDevice, stream);
        }
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(stream);
    }
    if (e != cudaSuccess)
        return cuda_fail(sticky, e, "gmm_state_set");
    return GMM_OK;
}

cudaError_t make_retaining_pool(int device, uint64_t keep_bytes, cudaMemPool_t *out) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaError_t e = cudaMemPoolCreate(out, &props);
    if (e == cudaSuccess)
        e = cudaMemPoolSetAttribute(*out, cudaMemPoolAttrReleaseThreshold, &keep_bytes);
    return e;
}

cudaError_t reserve_in_pool(cudaMemPool_t pool, size_t bytes, cudaStream_t s) {
    if (bytes == 0)
        return cudaSuccess;
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, s);
    if (e == cudaSuccess)
        e = cudaFreeAsync(p, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    return e != cudaSuccess ? e : es;
}

int wait_event(cudaEvent_t ev, int timeout_ms, cudaError_t *sticky, const char *what) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess)
            return GMM_OK;
        if (q != cudaErrorNotReady)
            return cuda_fail(sticky, q, what);
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (ms >= timeout_ms)
                return fail(GMM_ETIMEOUT, std::string(what) + ": wait timed out");
        }
        std::this_thread::yield();
    }
}

} // namespace gmmlib

using namespace gmmlib;

struct gmm_ctx {
    gmm_config cfg;
    Layout L;
    int device = 0;
    cudaStream_t stream = nullptr;
    void *arena = nullptr;
    uint32_t *morph_tmp = nullptr;
    int initialized = 0;
    cudaError_t sticky = cudaSuccess;
    // pipelined host path
    bool pipe_ready = false;
    cudaStream_t s_up = nullptr, s_down = nullptr;
    uint8_t *d_rgb[GMM_PIPE_DEPTH] = {};
    uint16_t *d_depth[GMM_PIPE_DEPTH] = {};
    uint32_t *d_mask[GMM_PIPE_DEPTH] = {};
    cudaEvent_t ev_up[GMM_PIPE_DEPTH] = {}, ev_comp[GMM_PIPE_DEPTH] = {},
                ev_down[GMM_PIPE_DEPTH] = {};
    long long slot_ticket[GMM_PIPE_DEPTH] = {-1, -1, -1};
    long long next_ticket = 0;
    long long done_upto = -1;
    // tick kernel selection and the staged kernel's wait-status word
    int kernel = GMM_KERNEL_DIRECT, variant = 0, ctas_per_sm = 0;
    int *d_status = nullptr;
    uint32_t ticks = 0; // ticks taken (seeds stochastic rounding)
};

static int launch_apply(gmm_ctx *h, const uint8_t *rgb, const uint16_t *depth, uint32_t *mask,
                        uint32_t *fgr, uint32_t *fgd) {
    uint32_t *tick_mask = h->cfg.morph_open ? h->morph_tmp : mask;
    CamView v = make_view(h->cfg, h->L, h->arena, rgb, depth, tick_mask, fgr, fgd,
                          h->initialized ? 0 : 1, h->ticks);
    cudaError_t e;
    if (h->initialized && h->kernel == GMM_KERNEL_STAGED && h->cfg.mode == GMM_MODE_FUSION &&
        !(h->cfg.flags & GMM_FLAG_STOCHASTIC_WEIGHTS))
        e = gmmhost::launch_tick_staged(v, h->variant, h->ctas_per_sm, h->d_status, h->stream);
    else
        e = gmmhost::launch_tick(
            v, gmmhost::direct_threads(h->kernel == GMM_KERNEL_DIRECT ? h->variant : 0,
                                       h->cfg.precision),
            h->stream);
    if (e == cudaSuccess && h->cfg.morph_open)
        e = gmmhost::launch_morph_open3(h->morph_tmp, mask, h->cfg.H, h->cfg.W, h->stream);
    if (e != cudaSuccess)
        return cuda_fail(&h->sticky, e, "gmm_apply launch");
    h->initialized = 1;
    h->ticks += 1;
    return GMM_OK;
}

extern "C" {

void gmm_config_init(gmm_config *cfg, int H, int W, int M, float alpha, float match_k,
                     float bg_T, float init_var, float init_w) {
    if (!cfg)
        return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->H = H;
    cfg->W = W;
    cfg->M = M;
    cfg->alpha = alpha;
    cfg->match_k = match_k;
    cfg->bg_T = bg_T;
    cfg->init_var = init_var;
    cfg->init_w = init_w;
    cfg->init_var_d = init_var;
    cfg->v_min_c = 1.0f;
    cfg->v_min_d = 1.0f;
    cfg->precision = GMM_PREC_F32;
    cfg->morph_open = 0;
    cfg->mode = GMM_MODE_FUSION;
    cfg->depth_scale = 255.0f / 4095.0f;
    cfg->flags = 0u;
}

int gmm_mask_words_per_row(int W) { return W < 1 ? 0 : (W + 31) / 32; }

size_t gmm_state_bytes(int H, int W, int M, int precision) {
    if (H < 1 || W < 1 || M < 3 || M > 5 || (precision != 0 && precision != 1))
        return 0;
    return make_layout(H, W, M, precision).total;
}

const char *gmm_last_error(void) { return g_err.c_str(); }

gmm_t *gmm_create_ex(const gmm_config *cfg) {
    const std::string msg = check_config(cfg);
    if (!msg.empty()) {
        fail(GMM_EINVAL, "gmm_create: " + msg);
        return nullptr;
    }
    gmm_ctx *h = new (std::nothrow) gmm_ctx();
    if (!h) {
        fail(GMM_ENOMEM, "gmm_create: host allocation failed");
        return nullptr;
    }
    h->cfg = *cfg;
    h->L = make_layout(cfg->H, cfg->W, cfg->M, cfg->precision);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaMalloc(&h->arena, h->L.total);
    if (e == cudaSuccess)
        e = cudaMemset(h->arena, 0, h->L.total);
    if (e == cudaSuccess && cfg->morph_open)
        e = cudaMalloc(&h->morph_tmp, (size_t)cfg->H * h->L.wpr * 4);
    if (e == cudaSuccess)
        e = cudaMalloc(&h->d_status, 256);
    if (e == cudaSuccess)
        e = cudaMemset(h->d_status, 0, 256);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        if (oom)
            fail(GMM_ENOMEM, std::string("gmm_create: ") + cudaGetErrorString(e));
        else
            cuda_fail(nullptr, e, "gmm_create");
        cudaGetLastError();
        if (h->arena)
            cudaFree(h->arena);
        if (h->morph_tmp)
            cudaFree(h->morph_tmp);
        if (h->d_status)
            cudaFree(h->d_status);
        delete h;
        return nullptr;
    }
    return h;
}

gmm_t *gmm_create(int H, int W, int M, float alpha, float match_k, float bg_T, float init_var,
                  float init_w) {
    gmm_config c;
    gmm_config_init(&c, H, W, M, alpha, match_k, bg_T, init_var, init_w);
    return gmm_create_ex(&c);
}

int gmm_set_stream(gmm_t *h, void *stream) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_set_stream: null handle");
    h->stream = static_cast<cudaStream_t>(stream);
    return GMM_OK;
}

int gmm_apply_ex(gmm_t *h, const uint8_t *rgb8, const uint16_t *depth16, uint32_t *mask_out,
                 uint32_t *fg_rgb_out, uint32_t *fg_d_out) {
    TraceRange tr("gmm_apply");
    if (!h)
        return fail(GMM_EINVAL, "gmm_apply: null handle");
    if (h->sticky != cudaSuccess)
        return fail(GMM_ECUDA, std::string("gmm_apply: earlier CUDA failure: ") +
                                   cudaGetErrorString(h->sticky));
    const std::string msg = check_frame_ptrs(rgb8, depth16, mask_out, fg_rgb_out, fg_d_out);
    if (!msg.empty())
        return fail(GMM_EINVAL, "gmm_apply: " + msg);
    DeviceGuard g(h->device);
    return launch_apply(h, rgb8, depth16, mask_out, fg_rgb_out, fg_d_out);
}

int gmm_apply(gmm_t *h, const uint8_t *rgb8, const uint16_t *depth16, uint32_t *mask_out) {
    return gmm_apply_ex(h, rgb8, depth16, mask_out, nullptr, nullptr);
}

static int ensure_pipe(gmm_ctx *h) {
    if (h->pipe_ready)
        return GMM_OK;
    const size_t N = (size_t)h->cfg.H * h->cfg.W;
    const size_t mask_bytes = (size_t)h->cfg.H * h->L.wpr * 4;
    cudaError_t e = cudaStreamCreateWithFlags(&h->s_up, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&h->s_down, cudaStreamNonBlocking);
    for (int s = 0; s < GMM_PIPE_DEPTH && e == cudaSuccess; ++s) {
        e = cudaMalloc(&h->d_rgb[s], N * 3);
        if (e == cudaSuccess)
            e = cudaMalloc(&h->d_depth[s], N * 2);
        if (e == cudaSuccess)
            e = cudaMalloc(&h->d_mask[s], mask_bytes);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&h->ev_up[s], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&h->ev_comp[s], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&h->ev_down[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(GMM_ENOMEM, "gmm pipeline: staging allocation failed");
        }
        return cuda_fail(&h->sticky, e, "gmm pipeline setup");
    }
    h->pipe_ready = true;
    return GMM_OK;
}

long long gmm_pipe_submit(gmm_t *h, const uint8_t *rgb8_host, const uint16_t *depth16_host,
                          uint32_t *mask_host) {
    TraceRange tr("gmm_pipe_submit");
    if (!h)
        return fail(GMM_EINVAL, "gmm_pipe_submit: null handle");
    if (h->sticky != cudaSuccess)
        return fail(GMM_ECUDA, std::string("gmm_pipe_submit: earlier CUDA failure: ") +
                                   cudaGetErrorString(h->sticky));
    if (!rgb8_host || !depth16_host || !mask_host)
        return fail(GMM_EINVAL, "gmm_pipe_submit: null buffer");
    DeviceGuard g(h->device);
    int rc = ensure_pipe(h);
    if (rc != GMM_OK)
        return rc;
    const long long t = h->next_ticket;
    const int s = (int)(t % GMM_PIPE_DEPTH);
    const size_t N = (size_t)h->cfg.H * h->cfg.W;
    const size_t mask_bytes = (size_t)h->cfg.H * h->L.wpr * 4;
    cudaError_t e = cudaSuccess;
    if (h->slot_ticket[s] >= 0) {
        // The slot's previous frame must be computed before its inputs are
        // overwritten, and downloaded before its mask buffer is rewritten.
        e = cudaStreamWaitEvent(h->s_up, h->ev_comp[s], 0);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(h->stream, h->ev_down[s], 0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_rgb[s], rgb8_host, N * 3, cudaMemcpyHostToDevice, h->s_up);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_depth[s], depth16_host, N * 2, cudaMemcpyHostToDevice, h->s_up);
    if (e == cudaSuccess)
        e = cudaEventRecord(h->ev_up[s], h->s_up);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(h->stream, h->ev_up[s], 0);
    if (e != cudaSuccess)
        return cuda_fail(&h->sticky, e, "gmm_pipe_submit upload");
    rc = launch_apply(h, h->d_rgb[s], h->d_depth[s], h->d_mask[s], nullptr, nullptr);
    if (rc != GMM_OK)
        return rc;
    e = cudaEventRecord(h->ev_comp[s], h->stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(h->s_down, h->ev_comp[s], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mask_host, h->d_mask[s], mask_bytes, cudaMemcpyDeviceToHost, h->s_down);
    if (e == cudaSuccess)
        e = cudaEventRecord(h->ev_down[s], h->s_down);
    if (e != cudaSuccess)
        return cuda_fail(&h->sticky, e, "gmm_pipe_submit download");
    h->slot_ticket[s] = t;
    h->next_ticket = t + 1;
    return t;
}

int gmm_pipe_wait(gmm_t *h, long long ticket, int timeout_ms) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_pipe_wait: null handle");
    if (ticket < 0 || ticket >= h->next_ticket)
        return fail(GMM_EINVAL, "gmm_pipe_wait: unknown ticket");
    if (ticket <= h->done_upto)
        return GMM_OK;
    DeviceGuard g(h->device);
    const int s = (int)(ticket % GMM_PIPE_DEPTH);
    // The slot holds this ticket or a later one; downloads complete in order.
    const int rc = wait_event(h->ev_down[s], timeout_ms, &h->sticky, "gmm_pipe_wait");
    if (rc == GMM_OK && h->slot_ticket[s] > h->done_upto)
        h->done_upto = h->slot_ticket[s];
    return rc;
}

int gmm_apply_host(gmm_t *h, const uint8_t *rgb8_host, const uint16_t *depth16_host,
                   uint32_t *mask_host) {
    const long long t = gmm_pipe_submit(h, rgb8_host, depth16_host, mask_host);
    if (t < 0)
        return (int)t;
    return gmm_pipe_wait(h, t, -1);
}

int gmm_state_get(const gmm_t *h, int plane, int component, float *dst_host, size_t n) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_state_get: null handle");
    DeviceGuard g(h->device);
    gmm_ctx *hm = const_cast<gmm_ctx *>(h);
    return state_get_common(h->cfg, h->L, h->arena, h->stream, &hm->sticky, plane, component,
                            dst_host, n);
}

int gmm_state_set(gmm_t *h, int plane, int component, const float *src_host, size_t n) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_state_set: null handle");
    DeviceGuard g(h->device);
    const int rc = state_set_common(h->cfg, h->L, h->arena, h->stream, &h->sticky, plane,
                                    component, src_host, n);
    if (rc == GMM_OK)
        h->initialized = 1;
    return rc;
}

int gmm_inject_cuda_error(gmm_t *h, int cuda_error) {
    if (!h || cuda_error == 0)
        return fail(GMM_EINVAL, "gmm_inject_cuda_error: null handle or zero error code");
    if (h->sticky == cudaSuccess)
        h->sticky = static_cast<cudaError_t>(cuda_error);
    return GMM_OK;
}

int gmm_reset(gmm_t *h) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_reset: null handle");
    h->initialized = 0;
    return GMM_OK;
}

int gmm_sync(gmm_t *h) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_sync: null handle");
    DeviceGuard g(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    int status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(&h->sticky, e, "gmm_sync");
    if (status != 0)
        return fail(GMM_ETIMEOUT, "gmm_sync: a staged-kernel pipeline wait ran out");
    return h->sticky == cudaSuccess ? GMM_OK : fail(GMM_ECUDA, "gmm_sync: earlier CUDA failure");
}

int gmm_wait_selftest(int timeout_ms, int *timed_out, double *waited_ms) {
    if (timeout_ms < 1 || timeout_ms > 2000 || !timed_out || !waited_ms)
        return fail(GMM_EINVAL, "gmm_wait_selftest: timeout_ms in [1, 2000] and outputs required");
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 16);
    if (e == cudaSuccess)
        e = cudaMemset(buf, 0, 16);
    int *status = static_cast<int *>(buf);
    unsigned long long *waited = reinterpret_cast<unsigned long long *>(static_cast<char *>(buf) + 8);
    if (e == cudaSuccess)
        e = gmmhost::launch_wait_selftest(status, waited, (unsigned long long)timeout_ms * 1000000ull,
                                          nullptr);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    int st = 0;
    unsigned long long ns = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(&ns, waited, sizeof(ns), cudaMemcpyDeviceToHost);
    if (buf)
        cudaFree(buf);
    if (e != cudaSuccess)
        return fail(GMM_ECUDA, std::string("gmm_wait_selftest: ") + cudaGetErrorString(e));
    *timed_out = st & 1;
    *waited_ms = (double)ns * 1e-6;
    return GMM_OK;
}

int gmm_set_kernel(gmm_t *h, int kind, int variant, int ctas_per_sm) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_set_kernel: null handle");
    if (kind != GMM_KERNEL_STAGED && kind != GMM_KERNEL_DIRECT)
        return fail(GMM_EINVAL, "gmm_set_kernel: unknown kernel kind");
    if (variant < 0 || variant > (kind == GMM_KERNEL_DIRECT ? 4 : 3))
        return fail(GMM_EINVAL, "gmm_set_kernel: variant must be in [0, 4] (direct) or [0, 3] "
                                "(staged)");
    if (ctas_per_sm < 0 || ctas_per_sm > 32)
        return fail(GMM_EINVAL, "gmm_set_kernel: ctas_per_sm must be in [0, 32]");
    h->kernel = kind;
    h->variant = variant;
    h->ctas_per_sm = ctas_per_sm;
    return GMM_OK;
}

int gmm_destroy(gmm_t *h) {
    if (!h)
        return fail(GMM_EINVAL, "gmm_destroy: null handle");
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->pipe_ready) {
        cudaStreamSynchronize(h->s_up);
        cudaStreamSynchronize(h->s_down);
        for (int s = 0; s < GMM_PIPE_DEPTH; ++s) {
            cudaFree(h->d_rgb[s]);
            cudaFree(h->d_depth[s]);
            cudaFree(h->d_mask[s]);
            cudaEventDestroy(h->ev_up[s]);
            cudaEventDestroy(h->ev_comp[s]);
            cudaEventDestroy(h->ev_down[s]);
        }
        cudaStreamDestroy(h->s_up);
        cudaStreamDestroy(h->s_down);
    }
    cudaFree(h->arena);
    if (h->morph_tmp)
        cudaFree(h->morph_tmp);
    if (h->d_status)
        cudaFree(h->d_status);
    delete h;
    return GMM_OK;
}

int gmm_fuse_masks(const uint32_t *fg_rgb, const uint32_t *fg_d, uint8_t *fusion,
                   uint32_t *mask_out, int H, int W, void *stream) {
    if (H < 1 || W < 1)
        return fail(GMM_EINVAL, "gmm_fuse_masks: H and W must be >= 1");
    if (!fg_rgb || !fg_d || !fusion || !mask_out)
        return fail(GMM_EINVAL, "gmm_fuse_masks: null pointer");
    if (reinterpret_cast<uintptr_t>(fg_rgb) % 4 || reinterpret_cast<uintptr_t>(fg_d) % 4 ||
        reinterpret_cast<uintptr_t>(mask_out) % 4)
        return fail(GMM_EINVAL, "gmm_fuse_masks: masks must be 4-byte aligned");
    if (!device_accessible(fg_rgb) || !device_accessible(fg_d) || !device_accessible(fusion) ||
        !device_accessible(mask_out))
        return fail(GMM_EINVAL, "gmm_fuse_masks: pointers must be device-accessible");
    const cudaError_t e = gmmhost::launch_fuse(fg_rgb, fg_d, fusion, mask_out, H, W,
                                               static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GMM_OK : cuda_fail(nullptr, e, "gmm_fuse_masks");
}

int gmm_pack_mask(const uint8_t *bytes, uint32_t *mask_out, int H, int W, void *stream) {
    if (H < 1 || W < 1)
        return fail(GMM_EINVAL, "gmm_pack_mask: H and W must be >= 1");
    if (!bytes || !mask_out || reinterpret_cast<uintptr_t>(mask_out) % 4)
        return fail(GMM_EINVAL, "gmm_pack_mask: null or misaligned pointer");
    if (!device_accessible(bytes) || !device_accessible(mask_out))
        return fail(GMM_EINVAL, "gmm_pack_mask: pointers must be device-accessible");
    const cudaError_t e = gmmhost::launch_pack(bytes, mask_out, H, W,
                                               static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GMM_OK : cuda_fail(nullptr, e, "gmm_pack_mask");
}

int gmm_mask_confusion(const uint32_t *pred, const uint32_t *truth, int H, int W,
                       unsigned long long *counts_out, void *stream) {
    if (H < 1 || W < 1)
        return fail(GMM_EINVAL, "gmm_mask_confusion: H and W must be >= 1");
    if (!pred || !truth || !counts_out || reinterpret_cast<uintptr_t>(pred) % 4 ||
        reinterpret_cast<uintptr_t>(truth) % 4 || reinterpret_cast<uintptr_t>(counts_out) % 8)
        return fail(GMM_EINVAL, "gmm_mask_confusion: null or misaligned pointer");
    if (!device_accessible(pred) || !device_accessible(truth) || !device_accessible(counts_out))
        return fail(GMM_EINVAL, "gmm_mask_confusion: pointers must be device-accessible");
    const cudaError_t e = gmmhost::launch_confusion(pred, truth, H, W, counts_out,
                                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GMM_OK : cuda_fail(nullptr, e, "gmm_mask_confusion");
}

int gmm_morph_open3(const uint32_t *mask_in, uint32_t *mask_out, int H, int W, void *stream) {
    if (H < 1 || W < 1)
        return fail(GMM_EINVAL, "gmm_morph_open3: H and W must be >= 1");
    if (!mask_in || !mask_out || mask_in == mask_out)
        return fail(GMM_EINVAL, "gmm_morph_open3: null or identical buffers");
    if (reinterpret_cast<uintptr_t>(mask_in) % 4 || reinterpret_cast<uintptr_t>(mask_out) % 4)
        return fail(GMM_EINVAL, "gmm_morph_open3: masks must be 4-byte aligned");
    if (!device_accessible(mask_in) || !device_accessible(mask_out))
        return fail(GMM_EINVAL, "gmm_morph_open3: pointers must be device-accessible");
    const cudaError_t e = gmmhost::launch_morph_open3(mask_in, mask_out, H, W,
                                                      static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GMM_OK : cuda_fail(nullptr, e, "gmm_morph_open3");
}

} // extern "C"
