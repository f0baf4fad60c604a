// Serving engine: continuous batching of frames from many cameras over the
// multi-camera pool. Client threads admit cameras and push frames that live
// in page-locked host memory; one engine thread forms ticks, launches the
// pooled kernel and stamps latencies. By default the pooled kernel reads
// the frames and writes the masks in that host memory directly (over the
// coherent host link: no copies, no staging buffers); in the copy mode the
// engine uploads the frames into per-camera device buffers and downloads the
// masks, on separate streams so the copies of one tick overlap the compute
// of its neighbours.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "gmm.h"
#include "gmm_common.h"

using namespace gmmlib;

namespace {

double clock_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct Frame {
    long long ticket;
    const uint8_t *rgb;
    const uint16_t *depth;
    uint32_t *mask;
    double t_arrival;
    double t_pushed = 0.0;  // gmm_server_push queued it
    double t_batched = 0.0; // the engine took it into a tick
};

struct SrvCam {
    bool used = false;
    int pool_id = -1;
    gmm_config cfg{};
    size_t rgb_bytes = 0, dep_bytes = 0, mask_bytes = 0, mem_bytes = 0;
    uint8_t *d_buf = nullptr; // upload buffers + device mask, one frame in flight
    std::deque<Frame> queue;
    bool in_flight = false;
};

constexpr size_t kMaxRecords = size_t(1) << 20; // latencies and traces kept

struct TickRec {
    cudaEvent_t done = nullptr;
    double t_submitted = 0.0; // copies and launch queued
    std::vector<std::pair<int, Frame>> jobs;
};

} // namespace

struct gmm_server {
    int device = 0, prec = 0, queue_depth = 1;
    std::atomic<int> transfer{GMM_SERVE_ZERO_COPY}; // fixed once a camera has been admitted
    size_t budget = 0, used = 0;
    gmm_pool_t *pool = nullptr;
    std::vector<SrvCam> cams;
    cudaStream_t s_up = nullptr, s_comp = nullptr, s_down = nullptr;
    cudaEvent_t ev_up = nullptr, ev_comp = nullptr, ev_alloc = nullptr;
    cudaMemPool_t mempool = nullptr; // staging buffers; keeps freed memory mapped
    std::mutex mu;      // queues, tickets, counters, slots
    std::mutex pool_mu; // every call into the pool and stream-ordered allocation
    std::condition_variable cv_work, cv_done;
    std::thread engine;
    std::atomic<bool> stop{false}, abort_now{false};
    std::atomic<double> max_gap_ms{0.0}; // longest gap between engine loop passes
    // Per-ticket and per-frame records grow in chunks (no reallocation
    // copies a growing array while the lock that pushes need is held) and
    // stay bounded on a long-running server: ticket states before the first
    // one not yet done are dropped (done_base counts them), and only the
    // most recent kMaxRecords latencies and traces are kept.
    std::deque<signed char> done; // tickets done_base..: 0 pending, 1 done, -1 failed
    long long done_base = 0, next_ticket = 0;
    std::deque<float> lat_ms;
    std::deque<gmm_server_trace> traces; // parallel to lat_ms
    gmm_server_stats st{};
    cudaError_t sticky = cudaSuccess;
    // engine thread only
    std::deque<TickRec> inflight;
    std::vector<cudaEvent_t> ev_pool;
};

// State of a ticket (caller holds s->mu): tickets before done_base are done.
static int ticket_state(const gmm_server *s, long long ticket) {
    return ticket < s->done_base ? 1 : s->done[(size_t)(ticket - s->done_base)];
}

static void finish_tick(gmm_server *s, TickRec &t, bool ok) {
    const double tnow = clock_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &j : t.jobs) {
            SrvCam &c = s->cams[j.first];
            c.in_flight = false;
            if (ok) {
                s->lat_ms.push_back((float)((tnow - j.second.t_arrival) * 1e3));
                s->traces.push_back(gmm_server_trace{j.second.ticket, j.first, (int)t.jobs.size(),
                                                     j.second.t_arrival, j.second.t_pushed,
                                                     j.second.t_batched, t.t_submitted, tnow});
                s->done[(size_t)(j.second.ticket - s->done_base)] = 1;
                s->st.completed += 1;
                s->st.pixels += (long long)c.cfg.H * c.cfg.W;
            } else {
                s->done[(size_t)(j.second.ticket - s->done_base)] = -1;
            }
        }
        while (!s->done.empty() && s->done.front() == 1) {
            s->done.pop_front();
            ++s->done_base;
        }
        while (s->lat_ms.size() > kMaxRecords) {
            s->lat_ms.pop_front();
            s->traces.pop_front();
        }
    }
    s->ev_pool.push_back(t.done);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Retire finished ticks, oldest first. block: wait (bounded) for the oldest.
static void harvest(gmm_server *s, bool block) {
    while (!s->inflight.empty()) {
        TickRec &t = s->inflight.front();
        cudaError_t q = cudaEventQuery(t.done);
        if (q == cudaErrorNotReady && block) {
            const int rc = wait_event(t.done, 60000, &s->sticky, "gmm server tick");
            q = rc == GMM_OK ? cudaSuccess : cudaErrorLaunchTimeout;
        }
        if (q == cudaErrorNotReady)
            return;
        if (q != cudaSuccess && s->sticky == cudaSuccess)
            s->sticky = q;
        finish_tick(s, t, q == cudaSuccess);
        s->inflight.pop_front();
        block = false;
    }
}

static cudaError_t enqueue_tick(gmm_server *s, TickRec &t) {
    TraceRange tr("gmm_server tick");
    cudaError_t e = cudaSuccess;
    if (s->transfer == GMM_SERVE_ZERO_COPY) {
        // the kernel reads the frames and writes the masks in host memory
        {
            std::lock_guard<std::mutex> lk(s->pool_mu);
            for (auto &j : t.jobs) {
                SrvCam &c = s->cams[j.first];
                if (gmm_pool_submit(s->pool, c.pool_id, j.second.rgb, j.second.depth,
                                    j.second.mask, nullptr, nullptr) != GMM_OK)
                    return cudaErrorInvalidValue;
            }
            if (gmm_pool_tick(s->pool) != GMM_OK)
                return cudaErrorLaunchFailure;
        }
        return cudaEventRecord(t.done, s->s_comp);
    }
    for (auto &j : t.jobs) {
        SrvCam &c = s->cams[j.first];
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.d_buf, j.second.rgb, c.rgb_bytes, cudaMemcpyHostToDevice, s->s_up);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.d_buf + align256(c.rgb_bytes), j.second.depth, c.dep_bytes,
                                cudaMemcpyHostToDevice, s->s_up);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(s->ev_up, s->s_up);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s->s_comp, s->ev_up, 0);
    if (e != cudaSuccess)
        return e;
    {
        std::lock_guard<std::mutex> lk(s->pool_mu);
        for (auto &j : t.jobs) {
            SrvCam &c = s->cams[j.first];
            uint8_t *rgb = c.d_buf;
            uint16_t *dep = reinterpret_cast<uint16_t *>(c.d_buf + align256(c.rgb_bytes));
            uint32_t *msk = reinterpret_cast<uint32_t *>(c.d_buf + align256(c.rgb_bytes) +
                                                         align256(c.dep_bytes));
            if (gmm_pool_submit(s->pool, c.pool_id, rgb, dep, msk, nullptr, nullptr) != GMM_OK)
                return cudaErrorInvalidValue;
        }
        if (gmm_pool_tick(s->pool) != GMM_OK)
            return cudaErrorLaunchFailure;
    }
    e = cudaEventRecord(s->ev_comp, s->s_comp);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s->s_down, s->ev_comp, 0);
    for (auto &j : t.jobs) {
        SrvCam &c = s->cams[j.first];
        const uint8_t *msk = c.d_buf + align256(c.rgb_bytes) + align256(c.dep_bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(j.second.mask, msk, c.mask_bytes, cudaMemcpyDeviceToHost, s->s_down);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(t.done, s->s_down);
    return e;
}

static void engine_main(gmm_server *s) {
    cudaSetDevice(s->device);
    double last_pass = clock_s();
    for (;;) {
        const double now = clock_s();
        if ((now - last_pass) * 1e3 > s->max_gap_ms.load(std::memory_order_relaxed))
            s->max_gap_ms.store((now - last_pass) * 1e3, std::memory_order_relaxed);
        last_pass = now;
        harvest(s, false);
        TickRec t;
        bool quit = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const double tb = clock_s();
            for (size_t i = 0; i < s->cams.size(); ++i) {
                SrvCam &c = s->cams[i];
                if (c.used && !c.in_flight && !c.queue.empty()) {
                    t.jobs.emplace_back((int)i, c.queue.front());
                    t.jobs.back().second.t_batched = tb;
                    c.queue.pop_front();
                    c.in_flight = true;
                }
            }
            if (t.jobs.empty()) {
                bool queued = false;
                for (auto &c : s->cams)
                    queued = queued || (c.used && !c.queue.empty());
                if ((s->stop && !queued && s->inflight.empty()) || s->abort_now)
                    quit = true;
                else // a push wakes the engine at once; otherwise poll completions
                    s->cv_work.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 200 : 20));
            }
        }
        if (quit)
            break;
        if (t.jobs.empty())
            continue;
        if (s->ev_pool.empty()) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                finish_tick(s, t, false);
                continue;
            }
            s->ev_pool.push_back(ev);
        }
        t.done = s->ev_pool.back();
        s->ev_pool.pop_back();
        const cudaError_t e = s->sticky == cudaSuccess ? enqueue_tick(s, t) : s->sticky;
        if (e != cudaSuccess) {
            if (s->sticky == cudaSuccess)
                s->sticky = e;
            finish_tick(s, t, false);
            continue;
        }
        t.t_submitted = clock_s();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.ticks += 1;
        }
        s->inflight.push_back(std::move(t));
    }
    while (!s->inflight.empty())
        harvest(s, true);
}

extern "C" {

double gmm_server_now(void) { return clock_s(); }

// Launch shape of the engine's pool. FP16/BF16 state in the zero-copy mode:
// 256-thread CTAs (as many as fit) over 512-pixel tiles, whose CTAs prefetch
// their next tile (the pool tuner's choice on the 64-camera mix; it also
// splits small ticks into more tiles). Measured on the 256-camera schedule:
// p50 0.114 -> 0.106 ms, p99 0.26 -> 0.21 ms, the genlocked rig's p50
// 0.68 -> 0.47 ms. Otherwise the pool's default (128 threads, 2048-pixel
// tiles, no early take): the copy mode uploads frames beside the running
// tick, and its latency tail grew with the other shape.
static void set_pool_shape(gmm_server *s) {
    if (s->prec == GMM_PREC_F16 && s->transfer == GMM_SERVE_ZERO_COPY)
        gmm_pool_set_launch(s->pool, 256, 0, 512);
    else
        gmm_pool_set_launch(s->pool, 128, 0, 2048);
}

gmm_server_t *gmm_server_create(size_t budget_bytes, int precision, int max_cams, int queue_depth) {
    if (precision != GMM_PREC_F32 && precision != GMM_PREC_F16) {
        fail(GMM_EINVAL, "gmm_server_create: bad precision");
        return nullptr;
    }
    if (max_cams < 1 || max_cams > 65536 || queue_depth < 1 || queue_depth > 1024) {
        fail(GMM_EINVAL, "gmm_server_create: max_cams in [1, 65536], queue_depth in [1, 1024]");
        return nullptr;
    }
    gmm_server *s = new (std::nothrow) gmm_server();
    if (!s) {
        fail(GMM_ENOMEM, "gmm_server_create: host allocation failed");
        return nullptr;
    }
    s->prec = precision;
    s->budget = budget_bytes;
    s->queue_depth = queue_depth;
    s->cams.resize((size_t)max_cams);
    s->st.budget_bytes = budget_bytes;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&s->s_up, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&s->s_down, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s->ev_up, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s->ev_comp, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s->ev_alloc, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = make_retaining_pool(s->device, budget_bytes ? (uint64_t)budget_bytes : UINT64_MAX,
                                &s->mempool);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "gmm_server_create");
        gmm_server_destroy(s, 0);
        return nullptr;
    }
    s->pool = gmm_pool_create(0, precision, max_cams);
    if (!s->pool) {
        gmm_server_destroy(s, 0);
        return nullptr;
    }
    gmm_pool_set_stream(s->pool, s->s_comp);
    set_pool_shape(s);
    s->engine = std::thread(engine_main, s);
    return s;
}

int gmm_server_set_transfer(gmm_server_t *s, int mode) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_set_transfer: null server");
    if (mode != GMM_SERVE_ZERO_COPY && mode != GMM_SERVE_COPY)
        return fail(GMM_EINVAL, "gmm_server_set_transfer: unknown mode");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->st.admitted > 0)
        return fail(GMM_EINVAL, "gmm_server_set_transfer: set it before the first admission");
    s->transfer = mode;
    set_pool_shape(s);
    return GMM_OK;
}

int gmm_server_admit(gmm_server_t *s, const gmm_config *cfg) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_admit: null server");
    const std::string msg = check_config(cfg);
    if (!msg.empty())
        return fail(GMM_EINVAL, "gmm_server_admit: " + msg);
    if (cfg->precision != s->prec || cfg->morph_open)
        return fail(GMM_EINVAL, "gmm_server_admit: precision must match the server; no opening");
    const size_t wpr = (size_t)(cfg->W + 31) / 32;
    const size_t rgb = (size_t)cfg->H * cfg->W * 3, dep = (size_t)cfg->H * cfg->W * 2;
    const size_t msk = (size_t)cfg->H * wpr * 4;
    const size_t staging =
        s->transfer == GMM_SERVE_COPY ? align256(rgb) + align256(dep) + align256(msk) : 0;
    const size_t bytes = gmm_state_bytes(cfg->H, cfg->W, cfg->M, cfg->precision) + staging;
    int slot = -1;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->budget && s->used + bytes > s->budget) {
            s->st.rejected += 1;
            return fail(GMM_EBUDGET, "gmm_server_admit: memory budget exhausted");
        }
        for (size_t i = 0; i < s->cams.size(); ++i)
            if (!s->cams[i].used && s->cams[i].pool_id < 0) {
                slot = (int)i;
                break;
            }
        if (slot < 0) {
            s->st.rejected += 1;
            return fail(GMM_ENOMEM, "gmm_server_admit: every slot is taken");
        }
        s->cams[slot].pool_id = -2; // reserved
        s->used += bytes;
    }
    DeviceGuard g(s->device);
    int pid;
    uint8_t *buf = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->pool_mu);
        pid = gmm_pool_admit(s->pool, cfg);
        cudaError_t e = cudaSuccess;
        if (pid >= 0 && staging > 0) {
            e = cudaMallocFromPoolAsync(&buf, staging, s->mempool, s->s_comp);
            if (e == cudaSuccess)
                e = cudaEventRecord(s->ev_alloc, s->s_comp);
            if (e == cudaSuccess) // uploads may only start once the buffer exists
                e = cudaStreamWaitEvent(s->s_up, s->ev_alloc, 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                gmm_pool_release(s->pool, pid);
                pid = e == cudaErrorMemoryAllocation ? GMM_ENOMEM : GMM_ECUDA;
                fail(pid, std::string("gmm_server_admit: ") + cudaGetErrorString(e));
            }
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    SrvCam &c = s->cams[slot];
    if (pid < 0) {
        c = SrvCam();
        s->used -= bytes;
        s->st.rejected += 1;
        return pid;
    }
    c = SrvCam();
    c.used = true;
    c.pool_id = pid;
    c.cfg = *cfg;
    c.rgb_bytes = rgb;
    c.dep_bytes = dep;
    c.mask_bytes = msk;
    c.mem_bytes = bytes;
    c.d_buf = buf;
    s->st.admitted += 1;
    s->st.live_cams += 1;
    s->st.used_bytes = s->used;
    return slot;
}

int gmm_server_reserve(gmm_server_t *s, size_t state_bytes, size_t staging_bytes) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_reserve: null server");
    DeviceGuard g(s->device);
    std::lock_guard<std::mutex> plk(s->pool_mu);
    const int rc = gmm_pool_reserve(s->pool, state_bytes);
    if (rc != GMM_OK)
        return rc;
    const cudaError_t e = reserve_in_pool(s->mempool, staging_bytes, s->s_comp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? GMM_ENOMEM : GMM_ECUDA,
                    std::string("gmm_server_reserve: ") + cudaGetErrorString(e));
    }
    return GMM_OK;
}

int gmm_server_release(gmm_server_t *s, int cam, int timeout_ms) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_release: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    if (cam < 0 || cam >= (int)s->cams.size() || !s->cams[cam].used)
        return fail(GMM_EINVAL, "gmm_server_release: unknown camera");
    auto idle = [&] { return s->cams[cam].queue.empty() && !s->cams[cam].in_flight; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, idle);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
        return fail(GMM_ETIMEOUT, "gmm_server_release: frames still pending");
    SrvCam c = s->cams[cam];
    s->cams[cam].used = false; // no new ticks pick it up
    lk.unlock();
    DeviceGuard g(s->device);
    cudaError_t e;
    {
        std::lock_guard<std::mutex> plk(s->pool_mu);
        gmm_pool_release(s->pool, c.pool_id);
        e = c.d_buf ? cudaFreeAsync(c.d_buf, s->s_comp) // after any queued use on the stream
                    : cudaSuccess;
    }
    lk.lock();
    s->cams[cam] = SrvCam();
    s->used -= c.mem_bytes;
    s->st.released += 1;
    s->st.live_cams -= 1;
    s->st.used_bytes = s->used;
    if (e != cudaSuccess)
        return cuda_fail(&s->sticky, e, "gmm_server_release");
    return GMM_OK;
}

long long gmm_server_push(gmm_server_t *s, int cam, const uint8_t *rgb8_host,
                          const uint16_t *depth16_host, uint32_t *mask_host, double t_arrival) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_push: null server");
    if (!rgb8_host || !depth16_host || !mask_host)
        return fail(GMM_EINVAL, "gmm_server_push: null buffer");
    if (s->transfer == GMM_SERVE_ZERO_COPY) { // the kernel will read and write them itself
        const std::string msg = check_frame_ptrs(rgb8_host, depth16_host, mask_host, nullptr,
                                                 nullptr);
        if (!msg.empty())
            return fail(GMM_EINVAL, "gmm_server_push (zero-copy mode: page-locked host memory the "
                                    "device can reach, or GMM_SERVE_COPY): " + msg);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->sticky != cudaSuccess)
        return fail(GMM_ECUDA, std::string("gmm_server_push: earlier CUDA failure: ") +
                                   cudaGetErrorString(s->sticky));
    if (cam < 0 || cam >= (int)s->cams.size() || !s->cams[cam].used)
        return fail(GMM_EINVAL, "gmm_server_push: unknown camera");
    SrvCam &c = s->cams[cam];
    if ((int)c.queue.size() >= s->queue_depth) {
        s->st.dropped += 1;
        return fail(GMM_EBUDGET, "gmm_server_push: camera queue full, frame dropped");
    }
    const long long t = s->next_ticket++;
    s->done.push_back(0);
    c.queue.push_back(Frame{t, rgb8_host, depth16_host, mask_host, t_arrival, clock_s()});
    s->st.pushed += 1;
    s->cv_work.notify_one();
    return t;
}

int gmm_server_done(gmm_server_t *s, long long ticket) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_done: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket < 0 || ticket >= s->next_ticket)
        return fail(GMM_EINVAL, "gmm_server_done: unknown ticket");
    const int d = ticket_state(s, ticket);
    return d < 0 ? fail(GMM_ECUDA, "gmm_server_done: the frame's tick failed") : d;
}

int gmm_server_wait(gmm_server_t *s, long long ticket, int timeout_ms) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket < 0 || ticket >= s->next_ticket)
        return fail(GMM_EINVAL, "gmm_server_wait: unknown ticket");
    auto ready = [&] { return ticket_state(s, ticket) != 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(GMM_ETIMEOUT, "gmm_server_wait: timed out");
    return ticket_state(s, ticket) > 0 ? GMM_OK
                                       : fail(GMM_ECUDA, "gmm_server_wait: the frame's tick failed");
}

int gmm_server_stats_get(gmm_server_t *s, gmm_server_stats *out) {
    if (!s || !out)
        return fail(GMM_EINVAL, "gmm_server_stats_get: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->max_engine_gap_ms = s->max_gap_ms.load(std::memory_order_relaxed);
    return GMM_OK;
}

size_t gmm_server_latencies(gmm_server_t *s, float *ms_out, size_t n) {
    if (!s)
        return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t k = n < s->lat_ms.size() ? n : s->lat_ms.size();
    if (ms_out && k)
        std::copy(s->lat_ms.begin(), s->lat_ms.begin() + (std::ptrdiff_t)k, ms_out);
    return s->lat_ms.size();
}

size_t gmm_server_traces(gmm_server_t *s, gmm_server_trace *out, size_t n) {
    if (!s)
        return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t k = n < s->traces.size() ? n : s->traces.size();
    if (out && k)
        std::copy(s->traces.begin(), s->traces.begin() + (std::ptrdiff_t)k, out);
    return s->traces.size();
}

int gmm_server_destroy(gmm_server_t *s, int timeout_ms) {
    if (!s)
        return fail(GMM_EINVAL, "gmm_server_destroy: null server");
    int rc = GMM_OK;
    if (s->engine.joinable()) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->stop = true;
            s->cv_work.notify_all();
            if (timeout_ms >= 0) {
                auto drained = [&] {
                    for (auto &c : s->cams)
                        if (c.used && (!c.queue.empty() || c.in_flight))
                            return false;
                    return true;
                };
                if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), drained)) {
                    s->abort_now = true; // stop forming ticks; in-flight ones still finish
                    rc = fail(GMM_ETIMEOUT, "gmm_server_destroy: frames were still queued");
                }
            }
        }
        s->cv_work.notify_all();
        s->engine.join();
    }
    DeviceGuard g(s->device);
    for (auto &c : s->cams)
        if (c.d_buf)
            cudaFreeAsync(c.d_buf, s->s_comp); // after any queued use on the stream
    if (s->s_comp)
        cudaStreamSynchronize(s->s_comp);
    if (s->mempool)
        cudaMemPoolDestroy(s->mempool);
    if (s->pool)
        gmm_pool_destroy(s->pool);
    for (cudaEvent_t ev : s->ev_pool)
        cudaEventDestroy(ev);
    for (cudaEvent_t ev : {s->ev_up, s->ev_comp, s->ev_alloc})
        if (ev)
            cudaEventDestroy(ev);
    for (cudaStream_t st : {s->s_up, s->s_comp, s->s_down})
        if (st)
            cudaStreamDestroy(st);
    delete s;
    return rc;
}

} // extern "C"
