// Multi-camera pool: resident per-camera models, one persistent launch per
// tick over every camera with a submitted frame, optional CUDA-graph replay
// of the tick, and an autotuner for the launch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "gmm.h"
#include "gmm_common.h"
#include "gmm_internal.h"

using gmmdev::CamView;
using namespace gmmlib;

namespace {

struct PoolCam {
    bool used = false;
    gmm_config cfg{};
    Layout L{};
    void *arena = nullptr;
    int initialized = 0;
    uint32_t ticks = 0; // ticks taken (seeds stochastic rounding)
    bool submitted = false;
    const uint8_t *rgb = nullptr;
    const uint16_t *depth = nullptr;
    uint32_t *mask = nullptr, *fgr = nullptr, *fgd = nullptr;
};

// What a captured graph depends on. The views and tile tables are read at
// replay from the page-locked staging buffer the graph was captured with.
struct GraphSig {
    int n_launch = -1, threads = 0;
    std::vector<int> blocks; // per launch
    std::vector<int> m; // per launch: the M its cameras share (flat form), else 0
    bool all_variants = false, flat = false, prefetch = true;
    bool operator==(const GraphSig &o) const {
        return n_launch == o.n_launch && threads == o.threads && blocks == o.blocks &&
               m == o.m && all_variants == o.all_variants && flat == o.flat &&
               prefetch == o.prefetch;
    }
};

constexpr int kStaging = 2; // page-locked argument buffers, used alternately

// ctas < 0: the flat (non-persistent) form; tile is then its chunk size.
struct Shape {
    int threads, ctas, tile;
};

int chunk_pixels(int prec) { return prec == 0 ? 32 : 64; }

// Online tuning: real ticks cycle through candidate launch shapes; a trial
// tick is timed on the pool's stream from its start to the start of the
// next tick (the tick period), so a shape is also charged for what its
// kernel delays in the work queued before the next tick (uploads of the next
// frames sharing HBM with it, in a pipeline). Two rounds: when every
// candidate has run its ticks, the kFinalists shapes with the lowest median
// periods run again with twice the ticks each, and the lowest median of
// that second round is kept (shapes a few percent apart are told apart
// without giving every candidate the longer run).
struct Trial {
    int cand = -1;
    cudaEvent_t a = nullptr, b = nullptr;
};
constexpr int kFinalists = 4;
struct Tuning {
    bool active = false;
    bool saved_graph = false;
    bool final_round = false;
    int per_shape = 0, issued = 0;
    std::vector<Shape> cands;
    Trial open;                 // the last trial tick, until the next tick starts
    std::vector<Trial> pending; // closed trials not yet read
    std::vector<std::vector<float>> ms;
};

} // namespace

namespace gmmhost {
int pool_max_ctas_per_sm(int prec, int threads);
}

struct gmm_pool {
    size_t budget = 0, used_bytes = 0;
    int prec = 0, max_cams = 0, device = 0;
    std::vector<PoolCam> cams;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr; // graph capture (the legacy stream cannot capture)
    cudaMemPool_t mempool = nullptr;   // cameras' state; keeps freed memory mapped
    cudaError_t sticky = cudaSuccess;
    int threads = 128, ctas_per_sm = 0, tile_pixels = 2048; // ctas_per_sm < 0: flat form
    // Tile counters, two sets of kmax (one per launch of a tick): a tick
    // uses set `parity` and its launches zero the other set for the next.
    int *d_counters = nullptr;
    int kmax = 1, parity = 0; // kmax: launches a tick may take
    std::vector<int> launch_m; // per launch: the M its cameras share (flat form), else 0
    // Launch arguments (kmax per tick) in page-locked memory, two buffers.
    gmmhost::PoolArgs *h_args[kStaging] = {};
    cudaEvent_t ev_staged[kStaging] = {};
    bool staged_used[kStaging] = {};
    int buf = 0;
    bool use_graph = false;
    bool prefetch = true; // FP16/BF16: next-tile L2 prefetch in the persistent form
    cudaGraphExec_t gexec[kStaging] = {};
    GraphSig gsig[kStaging];
    Tuning tune;
    int occupancy[9] = {};  // resident pool CTAs per SM, by block size / 32
    int sms = 0;
};

static void destroy_graphs(gmm_pool *p) {
    for (int b = 0; b < kStaging; ++b) {
        if (p->gexec[b])
            cudaGraphExecDestroy(p->gexec[b]);
        p->gexec[b] = nullptr;
        p->gsig[b] = GraphSig();
    }
}

// Resident CTAs per SM of the pool kernel for a block size (queried once per
// block size) times the SM count (queried once).
static int blocks_for(gmm_pool *p) {
    int &max_per_sm = p->occupancy[p->threads / 32];
    if (max_per_sm == 0)
        max_per_sm = gmmhost::pool_max_ctas_per_sm(p->prec, p->threads);
    if (p->sms == 0)
        p->sms = gmmhost::num_sms();
    int per_sm = p->ctas_per_sm;
    if (per_sm <= 0 || per_sm > max_per_sm)
        per_sm = max_per_sm;
    if (per_sm < 1)
        per_sm = 1;
    return p->sms * per_sm;
}

// Candidate launch shapes: block sizes, full or half residency, tile sizes
// of the persistent form. (The flat form is left to an explicit choice: it
// is the faster one for FP32 state with every input already in device
// memory, but host uploads that run beside it slow it far more than they
// slow the persistent form, and ticks timed without such uploads cannot
// tell.)
static std::vector<Shape> tuning_candidates(const gmm_pool *p) {
    std::vector<Shape> out;
    const int cand_threads[] = {64, 128, 256};
    const int cand_tiles[] = {256, 512, 1024, 2048, 8192};
    for (int t : cand_threads) {
        const int max_c = gmmhost::pool_max_ctas_per_sm(p->prec, t);
        const int cand_c[2] = {max_c, max_c > 1 ? max_c / 2 : 0};
        for (int c : cand_c)
            if (c >= 1)
                for (int tp : cand_tiles)
                    out.push_back({t, c, tp});
    }
    return out;
}

static float median(std::vector<float> v) {
    if (v.empty())
        return -1.f;
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
}

// Read the finished trials; when all are in, keep the best shape.
static int tuning_poll(gmm_pool *p, bool block) {
    Tuning &tu = p->tune;
    if (!tu.active)
        return GMM_OK;
    size_t k = 0;
    for (; k < tu.pending.size(); ++k) {
        Trial &tr = tu.pending[k];
        cudaError_t e = block ? cudaEventSynchronize(tr.b) : cudaEventQuery(tr.b);
        if (e == cudaErrorNotReady)
            break;
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, tr.a, tr.b);
        cudaEventDestroy(tr.a);
        cudaEventDestroy(tr.b);
        if (e != cudaSuccess) {
            tu.pending.erase(tu.pending.begin(), tu.pending.begin() + (long)k + 1);
            return cuda_fail(&p->sticky, e, "gmm_pool tuning");
        }
        tu.ms[tr.cand].push_back(ms);
    }
    tu.pending.erase(tu.pending.begin(), tu.pending.begin() + (long)k);
    const int total = (int)tu.cands.size() * tu.per_shape;
    if (tu.issued < total || tu.open.a || !tu.pending.empty())
        return GMM_OK;
    std::vector<std::pair<float, int>> order; // (median period, candidate); untimed last
    for (size_t c = 0; c < tu.cands.size(); ++c) {
        const float m = median(tu.ms[c]);
        order.push_back({m >= 0.f ? m : 3.4e38f, (int)c});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<float, int> &x, const std::pair<float, int> &y) {
                         return x.first < y.first;
                     });
    if (!tu.final_round && (int)tu.cands.size() > kFinalists) {
        std::vector<Shape> fin;
        for (int i = 0; i < kFinalists; ++i)
            fin.push_back(tu.cands[order[i].second]);
        tu.cands = fin;
        tu.ms.assign(fin.size(), {});
        tu.per_shape *= 2;
        tu.issued = 0;
        tu.final_round = true;
        return GMM_OK; // the next ticks run the finalists
    }
    const int best = order[0].second;
    p->threads = tu.cands[best].threads;
    p->ctas_per_sm = tu.cands[best].ctas;
    p->tile_pixels = tu.cands[best].tile;
    p->use_graph = tu.saved_graph;
    tu.active = false;
    return GMM_OK;
}

// Enqueue the tick's launches (argument upload + persistent kernel each)
// from staging buffer b.
static cudaError_t enqueue_body(gmm_pool *p, cudaStream_t s, int b, const GraphSig &sig) {
    cudaError_t e = cudaSuccess;
    for (int li = 0; li < sig.n_launch && e == cudaSuccess; ++li)
        e = gmmhost::launch_pool_tick_impl(&p->h_args[b][li], sig.threads, sig.blocks[li],
                                           p->prec, sig.all_variants, sig.flat, sig.m[li],
                                           sig.prefetch, s);
    return e;
}

// Launch the tick, directly or by replaying the graph captured for staging
// buffer b (captured again when its shape changed).
static cudaError_t launch_tick(gmm_pool *p, int b, int n_launch, bool all_variants) {
    GraphSig sig;
    sig.n_launch = n_launch;
    sig.threads = p->threads;
    sig.all_variants = all_variants;
    sig.flat = p->ctas_per_sm < 0;
    sig.prefetch = p->prefetch;
    const int warps = p->threads / 32;
    for (int li = 0; li < n_launch; ++li) { // flat: one warp per chunk
        sig.blocks.push_back(sig.flat ? (int)((p->h_args[b][li].n_tiles + warps - 1) / warps)
                                      : blocks_for(p));
        sig.m.push_back(p->launch_m[li]);
    }
    if (!p->use_graph) {
        cudaError_t e = gmmhost::pool_bank_acquire(p->device, p->stream);
        if (e != cudaSuccess)
            return e;
        e = enqueue_body(p, p->stream, b, sig);
        const cudaError_t er = gmmhost::pool_bank_release(p->device, p->stream);
        return e != cudaSuccess ? e : er;
    }
    cudaError_t e = cudaSuccess;
    if (!(p->gexec[b] && p->gsig[b] == sig)) {
        if (p->gexec[b])
            cudaGraphExecDestroy(p->gexec[b]);
        p->gexec[b] = nullptr;
        p->gsig[b] = GraphSig();
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t eb = enqueue_body(p, p->cap_stream, b, sig);
            e = cudaStreamEndCapture(p->cap_stream, &g);
            if (eb != cudaSuccess)
                e = eb;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&p->gexec[b], g, 0);
        if (g)
            cudaGraphDestroy(g);
        if (e == cudaSuccess)
            p->gsig[b] = sig;
    }
    if (e == cudaSuccess)
        e = gmmhost::pool_bank_acquire(p->device, p->stream);
    if (e == cudaSuccess) {
        e = cudaGraphLaunch(p->gexec[b], p->stream);
        const cudaError_t er = gmmhost::pool_bank_release(p->device, p->stream);
        if (e == cudaSuccess)
            e = er;
    }
    return e;
}

// One tick over the submitted cameras. clear: drop the submissions and mark
// the cameras initialised afterwards (false while autotuning).
static int pool_tick_impl(gmm_pool *p, bool clear) {
    int n_jobs = 0;
    for (const PoolCam &c : p->cams)
        n_jobs += (c.used && c.submitted) ? 1 : 0;
    if (n_jobs == 0)
        return GMM_OK;
    // An online-tuning trial sets its launch shape first: the tile tables
    // below depend on the tile size.
    Tuning &tu = p->tune;
    const bool trial = clear && tu.active && tu.issued < (int)tu.cands.size() * tu.per_shape;
    Trial tr{};
    if (trial) {
        // round-robin over the candidates, so drift in the frames spreads evenly
        tr.cand = tu.issued % (int)tu.cands.size();
        p->threads = tu.cands[tr.cand].threads;
        p->ctas_per_sm = tu.cands[tr.cand].ctas;
        p->tile_pixels = tu.cands[tr.cand].tile;
    }
    const int b = p->buf;
    if (p->staged_used[b]) {
        // The uploads that last read this staging buffer must have run.
        const int rc = wait_event(p->ev_staged[b], 60000, &p->sticky, "gmm_pool_tick staging");
        if (rc != GMM_OK)
            return rc;
    }
    // The launches' arguments: up to kPoolViews cameras each.
    // tiles, or in the flat form one chunk per warp
    const int unit = p->ctas_per_sm < 0 ? chunk_pixels(p->prec) : p->tile_pixels;
    int *cur = p->d_counters + p->parity * p->kmax;
    int *next = p->d_counters + (1 - p->parity) * p->kmax;
    int li = 0, j = 0;
    int64_t tiles = 0;
    bool all_variants = false; // some camera needs the options or the augmented mixture
    const bool flat = p->ctas_per_sm < 0;
    int group_m = 0; // flat form: the launch's cameras share M (a kernel per M)
    auto close_launch = [&]() {
        gmmhost::PoolArgs &a = p->h_args[b][li];
        p->launch_m[li] = group_m;
        a.tile_begin[j] = tiles;
        a.n_jobs = j;
        a.n_tiles = tiles;
        a.tile_pixels = unit;
        a.counter = cur + li;
        a.reset = next;
        a.n_reset = p->kmax;
        ++li;
        j = 0;
        tiles = 0;
    };
    const int groups[3] = {3, 4, 5};
    for (int gi = 0; gi < (flat ? 3 : 1); ++gi) {
        group_m = flat ? groups[gi] : 0;
        for (PoolCam &c : p->cams) {
            if (!(c.used && c.submitted) || (group_m && c.cfg.M != group_m))
                continue;
            gmmhost::PoolArgs &a = p->h_args[b][li];
            a.views[j] = make_view(c.cfg, c.L, c.arena, c.rgb, c.depth, c.mask, c.fgr, c.fgd,
                                   c.initialized ? 0 : 1, c.ticks);
            all_variants = all_variants || gmmhost::view_variant(a.views[j]) != 0;
            a.tile_begin[j] = tiles;
            tiles += (c.L.n_pad + unit - 1) / unit;
            if (++j == gmmhost::kPoolViews)
                close_launch();
        }
        if (j > 0)
            close_launch();
    }
    const int n_launch = li;
    cudaError_t e = cudaSuccess;
    if (clear && tu.active && tu.open.a) { // this tick's start ends the last trial's period
        e = cudaEventCreate(&tu.open.b);
        if (e == cudaSuccess)
            e = cudaEventRecord(tu.open.b, p->stream);
        if (e != cudaSuccess)
            return cuda_fail(&p->sticky, e, "gmm_pool_tick tuning");
        tu.pending.push_back(tu.open);
        tu.open = Trial();
    }
    if (trial) {
        e = cudaEventCreate(&tr.a);
        if (e == cudaSuccess)
            e = cudaEventRecord(tr.a, p->stream);
        if (e != cudaSuccess) {
            if (tr.a)
                cudaEventDestroy(tr.a);
            return cuda_fail(&p->sticky, e, "gmm_pool_tick tuning");
        }
        tu.open = tr;
        ++tu.issued;
    }
    e = launch_tick(p, b, n_launch, all_variants);
    if (e == cudaSuccess)
        e = cudaEventRecord(p->ev_staged[b], p->stream);
    if (e != cudaSuccess)
        return cuda_fail(&p->sticky, e, "gmm_pool_tick");
    p->staged_used[b] = true;
    p->buf = (b + 1) % kStaging;
    p->parity ^= 1;
    if (clear) {
        for (PoolCam &c : p->cams) {
            if (c.used && c.submitted) {
                c.initialized = 1;
                c.ticks += 1;
                c.submitted = false;
            }
        }
    }
    return tuning_poll(p, false);
}

static bool valid_cam(const gmm_pool *p, int cam) {
    return p && cam >= 0 && cam < (int)p->cams.size() && p->cams[cam].used;
}

extern "C" {

gmm_pool_t *gmm_pool_create(size_t budget_bytes, int precision, int max_cams) {
    if (precision != GMM_PREC_F32 && precision != GMM_PREC_F16) {
        fail(GMM_EINVAL, "gmm_pool_create: bad precision");
        return nullptr;
    }
    if (max_cams < 1 || max_cams > 65536) {
        fail(GMM_EINVAL, "gmm_pool_create: max_cams must be in [1, 65536]");
        return nullptr;
    }
    gmm_pool *p = new (std::nothrow) gmm_pool();
    if (!p) {
        fail(GMM_ENOMEM, "gmm_pool_create: host allocation failed");
        return nullptr;
    }
    p->budget = budget_bytes;
    p->prec = precision;
    p->max_cams = max_cams;
    p->cams.resize((size_t)max_cams);
    // one launch per kPoolViews cameras, plus one per M group in the flat form
    p->kmax = (max_cams + gmmhost::kPoolViews - 1) / gmmhost::kPoolViews + 2;
    p->launch_m.assign((size_t)p->kmax, 0);
    cudaError_t e = cudaGetDevice(&p->device);
    for (int b = 0; b < kStaging && e == cudaSuccess; ++b) {
        e = cudaMallocHost(&p->h_args[b], sizeof(gmmhost::PoolArgs) * (size_t)p->kmax);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&p->ev_staged[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&p->d_counters, sizeof(int) * 2 * (size_t)p->kmax);
    if (e == cudaSuccess)
        e = cudaMemset(p->d_counters, 0, sizeof(int) * 2 * (size_t)p->kmax);
    if (e == cudaSuccess)
        e = make_retaining_pool(p->device, budget_bytes ? (uint64_t)budget_bytes : UINT64_MAX,
                                &p->mempool);
    if (e != cudaSuccess) {
        fail(e == cudaErrorMemoryAllocation ? GMM_ENOMEM : GMM_ECUDA,
             std::string("gmm_pool_create: ") + cudaGetErrorString(e));
        cudaGetLastError();
        gmm_pool_destroy(p);
        return nullptr;
    }
    return p;
}

int gmm_pool_admit(gmm_pool_t *p, const gmm_config *cfg) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_admit: null pool");
    const std::string msg = check_config(cfg);
    if (!msg.empty())
        return fail(GMM_EINVAL, "gmm_pool_admit: " + msg);
    if (cfg->precision != p->prec)
        return fail(GMM_EINVAL, "gmm_pool_admit: precision differs from the pool's");
    if (cfg->morph_open)
        return fail(GMM_EINVAL, "gmm_pool_admit: morph_open is not supported in a pool");
    const Layout L = make_layout(cfg->H, cfg->W, cfg->M, cfg->precision);
    if (p->budget && p->used_bytes + L.total > p->budget)
        return fail(GMM_EBUDGET, "gmm_pool_admit: state budget exhausted");
    int slot = -1;
    for (int i = 0; i < (int)p->cams.size(); ++i)
        if (!p->cams[i].used) {
            slot = i;
            break;
        }
    if (slot < 0)
        return fail(GMM_ENOMEM, "gmm_pool_admit: every slot is taken");
    DeviceGuard g(p->device);
    void *arena = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&arena, L.total, p->mempool, p->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(arena, 0, L.total, p->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (arena)
            cudaFreeAsync(arena, p->stream);
        return fail(e == cudaErrorMemoryAllocation ? GMM_ENOMEM : GMM_ECUDA,
                    std::string("gmm_pool_admit: ") + cudaGetErrorString(e));
    }
    PoolCam &c = p->cams[slot];
    c = PoolCam();
    c.used = true;
    c.cfg = *cfg;
    c.L = L;
    c.arena = arena;
    p->used_bytes += L.total;
    return slot;
}

int gmm_pool_reserve(gmm_pool_t *p, size_t bytes) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_reserve: null pool");
    if (p->budget && bytes > p->budget)
        bytes = p->budget;
    DeviceGuard g(p->device);
    const cudaError_t e = reserve_in_pool(p->mempool, bytes, p->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? GMM_ENOMEM : GMM_ECUDA,
                    std::string("gmm_pool_reserve: ") + cudaGetErrorString(e));
    }
    return GMM_OK;
}

int gmm_pool_release(gmm_pool_t *p, int cam) {
    if (!valid_cam(p, cam))
        return fail(GMM_EINVAL, "gmm_pool_release: unknown camera");
    DeviceGuard g(p->device);
    PoolCam &c = p->cams[cam];
    // Stream-ordered free: queued ticks that use the state run first.
    const cudaError_t e = cudaFreeAsync(c.arena, p->stream);
    p->used_bytes -= c.L.total;
    c = PoolCam();
    if (e != cudaSuccess)
        return cuda_fail(&p->sticky, e, "gmm_pool_release");
    return GMM_OK;
}

int gmm_pool_submit(gmm_pool_t *p, int cam, const uint8_t *rgb8, const uint16_t *depth16,
                    uint32_t *mask_out, uint32_t *fg_rgb_out, uint32_t *fg_d_out) {
    if (!valid_cam(p, cam))
        return fail(GMM_EINVAL, "gmm_pool_submit: unknown camera");
    const std::string msg = check_frame_ptrs(rgb8, depth16, mask_out, fg_rgb_out, fg_d_out);
    if (!msg.empty())
        return fail(GMM_EINVAL, "gmm_pool_submit: " + msg);
    PoolCam &c = p->cams[cam];
    c.submitted = true;
    c.rgb = rgb8;
    c.depth = depth16;
    c.mask = mask_out;
    c.fgr = fg_rgb_out;
    c.fgd = fg_d_out;
    return GMM_OK;
}

int gmm_pool_submit_many(gmm_pool_t *p, int n, const int *cams, const uint8_t *const *rgb8,
                         const uint16_t *const *depth16, uint32_t *const *mask_out) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_submit_many: null pool");
    if (n < 0 || (n > 0 && (!cams || !rgb8 || !depth16 || !mask_out)))
        return fail(GMM_EINVAL, "gmm_pool_submit_many: bad arrays");
    for (int i = 0; i < n; ++i) {
        const int rc = gmm_pool_submit(p, cams[i], rgb8[i], depth16[i], mask_out[i], nullptr,
                                       nullptr);
        if (rc != GMM_OK)
            return rc;
    }
    return GMM_OK;
}

int gmm_pool_inject_cuda_error(gmm_pool_t *p, int cuda_error) {
    if (!p || cuda_error == 0)
        return fail(GMM_EINVAL, "gmm_pool_inject_cuda_error: null pool or zero error code");
    if (p->sticky == cudaSuccess)
        p->sticky = static_cast<cudaError_t>(cuda_error);
    return GMM_OK;
}

int gmm_pool_tick(gmm_pool_t *p) {
    TraceRange tr("gmm_pool_tick");
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_tick: null pool");
    if (p->sticky != cudaSuccess)
        return fail(GMM_ECUDA, std::string("gmm_pool_tick: earlier CUDA failure: ") +
                                   cudaGetErrorString(p->sticky));
    DeviceGuard g(p->device);
    return pool_tick_impl(p, true);
}

int gmm_pool_set_stream(gmm_pool_t *p, void *cuda_stream) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_set_stream: null pool");
    if (p->stream != static_cast<cudaStream_t>(cuda_stream))
        destroy_graphs(p);
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    return GMM_OK;
}

int gmm_pool_set_launch(gmm_pool_t *p, int threads, int ctas_per_sm, int tile_pixels) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_set_launch: null pool");
    const int t = threads ? threads : p->threads;
    const int c = ctas_per_sm ? ctas_per_sm : p->ctas_per_sm;
    // leaving the flat form without a tile size: the default tile
    const int tp = tile_pixels ? tile_pixels : (c >= 0 && p->ctas_per_sm < 0) ? 2048 : p->tile_pixels;
    if (t < 64 || t > 256 || t % 32)
        return fail(GMM_EINVAL, "gmm_pool_set_launch: threads must be 64..256, a multiple of 32");
    if (c < -1 || c > 32)
        return fail(GMM_EINVAL, "gmm_pool_set_launch: ctas_per_sm must be in [-1, 32]");
    if (c >= 0 && (tp < t || tp % t || tp > (1 << 24)))
        return fail(GMM_EINVAL, "gmm_pool_set_launch: tile_pixels must be a multiple of threads");
    p->threads = t;
    p->ctas_per_sm = c;
    p->tile_pixels = tp;
    return GMM_OK;
}

int gmm_pool_set_prefetch(gmm_pool_t *p, int enable) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_set_prefetch: null pool");
    p->prefetch = enable != 0; // picks the kernel instance from the next tick
    return GMM_OK;
}

int gmm_pool_use_graph(gmm_pool_t *p, int enable) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_use_graph: null pool");
    if (p->tune.active) { // applies once online tuning has finished
        p->tune.saved_graph = enable != 0;
        return GMM_OK;
    }
    p->use_graph = enable != 0;
    if (!p->use_graph)
        destroy_graphs(p);
    return GMM_OK;
}

int gmm_pool_autotune_online(gmm_pool_t *p, int ticks_per_shape) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_autotune_online: null pool");
    if (ticks_per_shape < 1 || ticks_per_shape > 1000)
        return fail(GMM_EINVAL, "gmm_pool_autotune_online: ticks_per_shape must be in [1, 1000]");
    DeviceGuard g(p->device);
    const int rc = tuning_poll(p, true); // finish an earlier run first
    if (rc != GMM_OK)
        return rc;
    Tuning &tu = p->tune;
    if (tu.open.a) { // an unfinished run's last trial: no tick will end it now
        cudaEventDestroy(tu.open.a);
        tu.open = Trial();
    }
    tu.cands = tuning_candidates(p);
    tu.ms.assign(tu.cands.size(), {});
    tu.per_shape = ticks_per_shape;
    tu.issued = 0;
    tu.final_round = false;
    tu.saved_graph = p->use_graph;
    p->use_graph = false; // each trial tick launches directly
    tu.active = true;
    return GMM_OK;
}

int gmm_pool_tuning(gmm_pool_t *p, int *threads, int *ctas_per_sm, int *tile_pixels) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_tuning: null pool");
    DeviceGuard g(p->device);
    const int rc = tuning_poll(p, false);
    if (rc != GMM_OK)
        return rc;
    if (threads)
        *threads = p->threads;
    if (ctas_per_sm)
        *ctas_per_sm = p->ctas_per_sm;
    if (tile_pixels)
        *tile_pixels = p->tile_pixels;
    return p->tune.active ? 1 : 0;
}

int gmm_pool_autotune(gmm_pool_t *p, int iters, int *threads_out, int *ctas_out,
                      int *tile_out) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_autotune: null pool");
    if (iters < 1)
        return fail(GMM_EINVAL, "gmm_pool_autotune: iters must be >= 1");
    if (p->sticky != cudaSuccess)
        return fail(GMM_ECUDA, "gmm_pool_autotune: earlier CUDA failure");
    bool any = false;
    size_t snap_bytes = 0;
    for (const PoolCam &c : p->cams)
        if (c.used && c.submitted) {
            any = true;
            snap_bytes += c.L.total;
        }
    if (!any)
        return fail(GMM_EINVAL, "gmm_pool_autotune: no camera has a submitted frame");
    DeviceGuard g(p->device);
    // Snapshot every submitted camera's state so the trials leave no trace.
    uint8_t *snap = nullptr;
    cudaError_t e = cudaMalloc(&snap, snap_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GMM_ENOMEM, "gmm_pool_autotune: no room for the state snapshot");
    }
    std::vector<int> init_saved(p->cams.size());
    size_t off = 0;
    for (size_t i = 0; i < p->cams.size() && e == cudaSuccess; ++i) {
        PoolCam &c = p->cams[i];
        init_saved[i] = c.initialized;
        if (c.used && c.submitted) {
            e = cudaMemcpyAsync(snap + off, c.arena, c.L.total, cudaMemcpyDeviceToDevice, p->stream);
            off += c.L.total;
        }
    }
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess)
        e = cudaEventCreate(&t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t1);
    const int saved_t = p->threads, saved_c = p->ctas_per_sm, saved_tp = p->tile_pixels;
    const bool saved_graph = p->use_graph;
    p->use_graph = false;
    int best_t = saved_t, best_c = saved_c, best_tp = saved_tp;
    float best_ms = -1.f;
    const std::vector<Shape> cands = tuning_candidates(p);
    int rc = GMM_OK;
    // Two passes over the candidates (the best time of each counts), so a
    // transient slowdown during one trial does not decide the shape.
    for (int pass = 0; pass < 2; ++pass) {
        for (const Shape &sh : cands) {
            if (e != cudaSuccess || rc != GMM_OK)
                break;
            p->threads = sh.threads;
            p->ctas_per_sm = sh.ctas;
            p->tile_pixels = sh.tile;
            rc = pool_tick_impl(p, false); // warm-up of this shape
            if (rc != GMM_OK)
                break;
            e = cudaEventRecord(t0, p->stream);
            for (int k = 0; k < iters && rc == GMM_OK; ++k)
                rc = pool_tick_impl(p, false);
            if (e == cudaSuccess)
                e = cudaEventRecord(t1, p->stream);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && rc == GMM_OK && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best_t = sh.threads;
                best_c = sh.ctas;
                best_tp = sh.tile;
            }
            for (PoolCam &cam : p->cams)
                if (cam.used && cam.submitted)
                    cam.initialized = 1; // later trials update, as real ticks would
        }
    }
    // Restore the snapshot and the initialisation flags.
    off = 0;
    for (size_t i = 0; i < p->cams.size(); ++i) {
        PoolCam &c = p->cams[i];
        c.initialized = init_saved[i];
        if (c.used && c.submitted) {
            const cudaError_t er = cudaMemcpyAsync(c.arena, snap + off, c.L.total,
                                                   cudaMemcpyDeviceToDevice, p->stream);
            if (e == cudaSuccess)
                e = er;
            off += c.L.total;
        }
    }
    const cudaError_t es = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess)
        e = es;
    cudaFree(snap);
    if (t0)
        cudaEventDestroy(t0);
    if (t1)
        cudaEventDestroy(t1);
    p->use_graph = saved_graph;
    if (e != cudaSuccess)
        return cuda_fail(&p->sticky, e, "gmm_pool_autotune");
    if (rc != GMM_OK)
        return rc;
    p->threads = best_t;
    p->ctas_per_sm = best_c;
    p->tile_pixels = best_tp;
    destroy_graphs(p);
    if (threads_out)
        *threads_out = best_t;
    if (ctas_out)
        *ctas_out = best_c;
    if (tile_out)
        *tile_out = best_tp;
    return GMM_OK;
}

int gmm_pool_state_get(const gmm_pool_t *p, int cam, int plane, int component,
                       float *dst_host, size_t n) {
    if (!valid_cam(p, cam))
        return fail(GMM_EINVAL, "gmm_pool_state_get: unknown camera");
    DeviceGuard g(p->device);
    gmm_pool *pm = const_cast<gmm_pool *>(p);
    const PoolCam &c = p->cams[cam];
    return state_get_common(c.cfg, c.L, c.arena, p->stream, &pm->sticky, plane, component,
                            dst_host, n);
}

size_t gmm_pool_state_used(const gmm_pool_t *p) { return p ? p->used_bytes : 0; }

int gmm_pool_sync(gmm_pool_t *p) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_sync: null pool");
    DeviceGuard g(p->device);
    const cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess)
        return cuda_fail(&p->sticky, e, "gmm_pool_sync");
    return p->sticky == cudaSuccess ? GMM_OK : fail(GMM_ECUDA, "gmm_pool_sync: earlier CUDA failure");
}

int gmm_pool_destroy(gmm_pool_t *p) {
    if (!p)
        return fail(GMM_EINVAL, "gmm_pool_destroy: null pool");
    DeviceGuard g(p->device);
    cudaStreamSynchronize(p->stream);
    destroy_graphs(p);
    for (Trial &tr : p->tune.pending) {
        cudaEventDestroy(tr.a);
        cudaEventDestroy(tr.b);
    }
    p->tune.pending.clear();
    if (p->tune.open.a)
        cudaEventDestroy(p->tune.open.a);
    p->tune.open = Trial();
    for (PoolCam &c : p->cams)
        if (c.used && c.arena)
            cudaFreeAsync(c.arena, p->stream);
    cudaStreamSynchronize(p->stream);
    if (p->mempool)
        cudaMemPoolDestroy(p->mempool);
    if (p->d_counters)
        cudaFree(p->d_counters);
    if (p->cap_stream)
        cudaStreamDestroy(p->cap_stream);
    for (int b = 0; b < kStaging; ++b) {
        if (p->h_args[b])
            cudaFreeHost(p->h_args[b]);
        if (p->ev_staged[b])
            cudaEventDestroy(p->ev_staged[b]);
    }
    delete p;
    return GMM_OK;
}

} // extern "C"
