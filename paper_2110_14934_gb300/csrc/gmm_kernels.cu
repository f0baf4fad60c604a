// Kernels: single-camera tick, List 1 alone, the 3x3 opening of a
// bit-packed mask, mask packing and confusion counts. (The multi-camera tick
// is in gmm_pool_kernel.cu.)
//
// The tick is HBM-bound: per pixel it reads and writes the whole mixture
// state (64*M bytes in FP32, 32*M in FP16/BF16) plus 5 bytes of frame, the
// List-1 byte and 1/8 byte of mask. There is no dense contraction, so there
// is no tensor-core work; the design goal is full-line coalesced traffic
// with enough bytes in flight per SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gmm_internal.h"

using namespace gmmdev;
using gmmhost::PoolArgs;

namespace {

// ------------------------------------------------------------ single camera
// Programmatic dependent launch between consecutive ticks on a stream: a
// tick waits for the kernel before it to complete (and its writes to be
// visible) before it reads anything, then lets the next tick be scheduled,
// so the next tick's CTAs take the SMs this tick's last CTAs leave idle
// instead of waiting for a full launch. (Both are no-ops when the kernel was
// not launched as a dependent.)
__device__ __forceinline__ void dependent_launch_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// FP32 state: one thread per padded pixel (n_pad is a multiple of 32: whole
// warps leave).
template <int M, int PREC, int V>
__device__ __forceinline__ void tick_body(const CamView &cv) {
    dependent_launch_prologue();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= cv.n_pad)
        return;
    const uint32_t bits = process_pixel<M, PREC, PREC != 0, V>(cv, p);
    write_mask_words(cv, p >> 5, bits);
}

// FP16/BF16 state: two pixels per thread, each warp a 64-pixel chunk (lane
// t takes pixels t and t + 32, so both halves stay coalesced); the second
// pixel's loads overlap the first one's arithmetic. A half chunk past n_pad
// is skipped by the whole warp.
template <int M, int PREC, int V>
__device__ __forceinline__ void tick_body2(const CamView &cv) {
    dependent_launch_prologue();
    const int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 64;
    if (base >= cv.n_pad)
        return;
    const int lane = threadIdx.x & 31;
    uint32_t bits[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t p = base + 32 * u + lane;
        bits[u] = p < cv.n_pad ? process_pixel<M, PREC, PREC != 0, V>(cv, p) : 0u;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (base + 32 * u < cv.n_pad)
            write_mask_words(cv, (base >> 5) + u, bits[u]);
}

// FP32 state: HBM-bound; the register allocation without a residency hint
// (64 registers) measured fastest. FP16/BF16 state: issue bound; at least
// 1024 threads per SM. V: process_pixel's variant (the options are separate
// instantiations, so the default kernels carry none of them). Small CTAs
// measured faster than 256 threads: a CTA's slot frees as soon as its own
// warps finish. A persistent grid-stride form measured slower (its loop
// costs registers: 66 in FP32, i.e. 3 CTAs of 256 per SM).
template <int M, int V>
__global__ void __launch_bounds__(256) k_tick_f32(const CamView cv) { tick_body<M, 0, V>(cv); }
template <int M, int V>
__global__ void __launch_bounds__(256, 4) k_tick_f16(const CamView cv) { tick_body2<M, 1, V>(cv); }

template <int M, int PREC, int V>
cudaError_t launch_tick_v(const CamView &cv, int threads, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (PREC == 0) {
        cfg.gridDim = dim3((unsigned)((cv.n_pad + threads - 1) / threads));
        return cudaLaunchKernelEx(&cfg, k_tick_f32<M, V>, cv);
    }
    const int64_t chunks = (cv.n_pad + 63) / 64; // one per warp
    const int warps = threads / 32;
    cfg.gridDim = dim3((unsigned)((chunks + warps - 1) / warps));
    return cudaLaunchKernelEx(&cfg, k_tick_f16<M, V>, cv);
}

template <int M, int PREC>
cudaError_t launch_tick_t(const CamView &cv, int threads, cudaStream_t s) {
    switch (gmmhost::view_variant(cv)) {
    case 0: return launch_tick_v<M, PREC, 0>(cv, threads, s);
    case 1: return launch_tick_v<M, PREC, 1>(cv, threads, s);
    default: return launch_tick_v<M, PREC, 2>(cv, threads, s);
    }
}

// ------------------------------------------------------------ List 1 alone
__global__ void __launch_bounds__(256) k_fuse(const uint32_t *fg_rgb, const uint32_t *fg_d,
                                              uint8_t *fusion, uint32_t *mask, int H, int W,
                                              int wpr) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_pad = (int64_t)H * wpr * 32;
    if (p >= n_pad)
        return;
    const int64_t wi = p >> 5;
    const int64_t row = wi / wpr;
    const int x = (int)(p - row * wpr * 32);
    const int lane = (int)(p & 31);
    uint32_t F = 0u;
    if (x < W) {
        const int fc = (int)((fg_rgb[wi] >> lane) & 1u);
        const int fd = (int)((fg_d[wi] >> lane) & 1u);
        const int64_t q = row * W + x;
        const uint32_t fb = fuse_list1(fc, fd, fusion[q]);
        fusion[q] = (uint8_t)fb;
        F = fb & 1u;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, F);
    if (lane == 0)
        mask[wi] = word;
}

// ------------------------------------------------------------ 3x3 opening
// A CTA of 32 x 8 threads produces an 8-row x 32-word tile. It stages the
// input tile with a 2-row and 2-word halo in shared memory, erodes (AND of
// the 3x3 neighbourhood, outside = 0) into a 1-row/1-word halo, then dilates
// (OR) into the output. Bit i of a word is pixel 32*word + i, so the left
// neighbour of bit i is bit i-1 (x << 1) and bit 0 takes bit 31 of the word
// on the left.
constexpr int kMR = 8, kMW = 32;

__device__ __forceinline__ uint32_t row_valid_bits(int w, int wpr, int W) {
    if (w < 0 || w >= wpr)
        return 0u;
    const int rem = W - 32 * w;
    return rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
}

__global__ void __launch_bounds__(kMR * kMW) k_morph_open3(const uint32_t *in, uint32_t *out,
                                                          int H, int W, int wpr) {
    __shared__ uint32_t s_in[kMR + 4][kMW + 4];  // rows r0-2.., words w0-2..
    __shared__ uint32_t s_h[kMR + 4][kMW + 2];   // horizontal erosion, words w0-1..
    __shared__ uint32_t s_e[kMR + 2][kMW + 2];   // erosion, rows r0-1.., words w0-1..
    __shared__ uint32_t s_hd[kMR + 2][kMW];      // horizontal dilation, words w0..
    dependent_launch_prologue(); // the mask it reads is complete; the next tick may be scheduled
    const int r0 = blockIdx.y * kMR, w0 = blockIdx.x * kMW;
    const int tid = threadIdx.y * kMW + threadIdx.x, nt = kMR * kMW;

    for (int i = tid; i < (kMR + 4) * (kMW + 4); i += nt) {
        const int rr = i / (kMW + 4), ww = i % (kMW + 4);
        const int r = r0 - 2 + rr, w = w0 - 2 + ww;
        uint32_t v = 0u;
        if (r >= 0 && r < H && w >= 0 && w < wpr)
            v = in[(int64_t)r * wpr + w] & row_valid_bits(w, wpr, W);
        s_in[rr][ww] = v;
    }
    __syncthreads();
    for (int i = tid; i < (kMR + 4) * (kMW + 2); i += nt) {
        const int rr = i / (kMW + 2), ww = i % (kMW + 2);
        const uint32_t m = s_in[rr][ww + 1], l = s_in[rr][ww], r = s_in[rr][ww + 2];
        s_h[rr][ww] = m & ((m << 1) | (l >> 31)) & ((m >> 1) | (r << 31));
    }
    __syncthreads();
    for (int i = tid; i < (kMR + 2) * (kMW + 2); i += nt) {
        const int rr = i / (kMW + 2), ww = i % (kMW + 2);
        const int r = r0 - 1 + rr, w = w0 - 1 + ww;
        uint32_t e = s_h[rr][ww] & s_h[rr + 1][ww] & s_h[rr + 2][ww];
        if (r < 0 || r >= H)
            e = 0u;
        s_e[rr][ww] = e & row_valid_bits(w, wpr, W);
    }
    __syncthreads();
    for (int i = tid; i < (kMR + 2) * kMW; i += nt) {
        const int rr = i / kMW, ww = i % kMW;
        const uint32_t m = s_e[rr][ww + 1], l = s_e[rr][ww], r = s_e[rr][ww + 2];
        s_hd[rr][ww] = m | (m << 1) | (l >> 31) | (m >> 1) | (r << 31);
    }
    __syncthreads();
    const int r = r0 + threadIdx.y, w = w0 + threadIdx.x;
    if (r < H && w < wpr) {
        const int rr = threadIdx.y + 1;
        const uint32_t o = s_hd[rr - 1][threadIdx.x] | s_hd[rr][threadIdx.x] | s_hd[rr + 1][threadIdx.x];
        out[(int64_t)r * wpr + w] = o & row_valid_bits(w, wpr, W);
    }
}

// ------------------------------------------------------------ mask metrics
// Byte mask (H*W, non-zero = 1) to the bit-packed layout: one thread per
// padded pixel, one ballot per word.
__global__ void __launch_bounds__(256) k_pack(const uint8_t *in, uint32_t *out, int H, int W,
                                              int wpr) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)H * wpr * 32)
        return;
    const int64_t row = (p >> 5) / wpr;
    const int x = (int)(p - row * wpr * 32);
    const uint32_t b = (x < W && in[row * W + x] != 0) ? 1u : 0u;
    const uint32_t word = __ballot_sync(0xffffffffu, b);
    if ((p & 31) == 0)
        out[p >> 5] = word;
}

// Confusion counts of a predicted mask against a truth mask (both
// bit-packed, bits beyond W ignored): out = {TP, FP, FN, TN}, accumulated.
__global__ void __launch_bounds__(256) k_confusion(const uint32_t *pred, const uint32_t *truth,
                                                   int H, int W, int wpr,
                                                   unsigned long long *out) {
    unsigned long long c[4] = {0, 0, 0, 0}; // TP, FP, FN, TN
    const int64_t n_words = (int64_t)H * wpr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_words;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(i % wpr);
        const int rem = W - 32 * col;
        const uint32_t valid = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
        const uint32_t p = pred[i], t = truth[i];
        c[0] += __popc(p & t & valid);
        c[1] += __popc(p & ~t & valid);
        c[2] += __popc(~p & t & valid);
        c[3] += __popc(~p & ~t & valid);
    }
    __shared__ unsigned long long s[4][8]; // blockDim.x = 256: 8 warps
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int off = 16; off > 0; off >>= 1)
            c[k] += __shfl_xor_sync(0xffffffffu, c[k], off);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k)
            s[k][threadIdx.x >> 5] = c[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long v = 0;
        for (int w = 0; w < 8; ++w)
            v += s[threadIdx.x][w];
        atomicAdd(&out[threadIdx.x], v);
    }
}

} // namespace

namespace gmmhost {

cudaError_t launch_tick(const CamView &cv, int threads, cudaStream_t s) {
    if (cv.n_pad == 0)
        return cudaSuccess;
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256)
        return cudaErrorInvalidValue;
    if (cv.prec == 0) {
        switch (cv.M) {
        case 3: return launch_tick_t<3, 0>(cv, threads, s);
        case 4: return launch_tick_t<4, 0>(cv, threads, s);
        case 5: return launch_tick_t<5, 0>(cv, threads, s);
        }
    } else {
        switch (cv.M) {
        case 3: return launch_tick_t<3, 1>(cv, threads, s);
        case 4: return launch_tick_t<4, 1>(cv, threads, s);
        case 5: return launch_tick_t<5, 1>(cv, threads, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fuse(const uint32_t *fg_rgb, const uint32_t *fg_d, uint8_t *fusion,
                        uint32_t *mask, int H, int W, cudaStream_t s) {
    const int wpr = (W + 31) / 32;
    const int64_t n_pad = (int64_t)H * wpr * 32;
    if (n_pad == 0)
        return cudaSuccess;
    k_fuse<<<(unsigned)((n_pad + 255) / 256), 256, 0, s>>>(fg_rgb, fg_d, fusion, mask, H, W, wpr);
    return cudaGetLastError();
}

cudaError_t launch_morph_open3(const uint32_t *in, uint32_t *out, int H, int W, cudaStream_t s) {
    const int wpr = (W + 31) / 32;
    // a programmatic dependent of the kernel before it, like the ticks
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3((unsigned)((wpr + kMW - 1) / kMW), (unsigned)((H + kMR - 1) / kMR));
    cfg.blockDim = dim3(kMW, kMR);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_morph_open3, in, out, H, W, wpr);
}

cudaError_t launch_pack(const uint8_t *in, uint32_t *out, int H, int W, cudaStream_t s) {
    const int wpr = (W + 31) / 32;
    const int64_t n = (int64_t)H * wpr * 32;
    if (n == 0)
        return cudaSuccess;
    k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, H, W, wpr);
    return cudaGetLastError();
}

cudaError_t launch_confusion(const uint32_t *pred, const uint32_t *truth, int H, int W,
                             unsigned long long *out, cudaStream_t s) {
    const int wpr = (W + 31) / 32;
    const int64_t n_words = (int64_t)H * wpr;
    cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || n_words == 0)
        return e;
    int64_t blocks = (n_words + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap)
        blocks = cap;
    k_confusion<<<(unsigned)blocks, 256, 0, s>>>(pred, truth, H, W, wpr, out);
    return cudaGetLastError();
}

int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n;
}

} // namespace gmmhost
