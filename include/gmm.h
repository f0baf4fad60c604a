/*
 * gmm.h - C ABI of the GB300 library for per-pixel Gaussian-mixture
 * background subtraction of RGB-D frames with counter-based fusion
 * ("GPU based GMM segmentation of Kinect data", Amamra, Mouats, Aouf).
 *
 * Method (§III): every pixel keeps two independent mixtures of M Gaussians
 * (3 <= M <= 5, §III.A), one on the colour image (3-channel mean, isotropic
 * variance) and one on the depth map (§III.B, "separated" modalities). Each
 * new frame is matched against the components in rank order, the matched
 * component is updated (or the weakest one replaced on a miss), the
 * components are re-ranked by w / sigma, and a pixel is foreground for a
 * stream when it does not fit that stream's background set (the best ranked
 * components whose weights sum above T). The two binary foregrounds are then
 * fused per pixel with List 1 (§III.C), using a fused label and a counter in
 * [-3, 3] kept per pixel.
 *
 * Model readings where the paper is silent (it defers the update equations
 * to Stauffer and Grimson): learning rate rho = alpha; colour variance is one
 * scalar tracking the squared distance summed over channels; rank key
 * w / sqrt(v), stable; a miss replaces the last-ranked component with
 * {mu = x, v = init_var, w = init_w}; weights are renormalised every tick;
 * B = shortest rank prefix with summed weight > T; variances are floored at
 * v_min; the first frame initialises every component on the sample with
 * w = 1/M and yields foreground 0; a zero depth reading is invalid (depth
 * model untouched, depth foreground := colour foreground) and the depth model
 * of a pixel starts at its first valid reading; List 1 is applied literally,
 * label and counter starting at 0. The registration of depth into the colour
 * frame (§III.C) is the identity: inputs are given on one pixel grid.
 *
 * Conventions
 *  - Every int return is a status (GMM_OK or a negative GMM_E* code).
 *    gmm_last_error() gives a thread-local message for the last failure.
 *  - Pointers documented as "device" must be device-accessible (device
 *    allocations, managed or mapped pinned memory); plain pageable host
 *    pointers are rejected with GMM_EINVAL instead of being dereferenced.
 *  - The library owns all model state (allocated at create, freed at
 *    destroy). The caller owns frames and masks and must keep them valid
 *    until the handle's stream has passed the call's work.
 *  - Frame layout: rgb8 is H*W*3 bytes, interleaved R,G,B, row-major, row
 *    stride W*3. depth16 is H*W uint16 millimetres, row stride W, 0 = no
 *    reading, 2-byte aligned.
 *  - Mask layout (bit-packed): H rows of gmm_mask_words_per_row(W) =
 *    ceil(W/32) uint32 words, 4-byte aligned; bit i of word c of row y is
 *    pixel x = 32*c + i (least significant bit first); bits for x >= W are 0.
 *  - A CUDA failure is sticky on the handle: later calls return GMM_ECUDA.
 *  - Threads: a handle or a pool is used by one thread at a time (calls on
 *    different handles and pools may run concurrently, and pools on one
 *    device share their launch-argument bank safely); the gmm_server_*
 *    calls other than gmm_server_destroy may be made from any thread.
 *    Device work is ordered on the object's stream.
 */
#ifndef GMM_H
#define GMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define GMM_OK 0
#define GMM_EINVAL (-1)   /* bad argument; nothing was launched */
#define GMM_ENOMEM (-2)   /* device or host allocation failed */
#define GMM_ECUDA (-3)    /* a CUDA call failed (sticky on the handle) */
#define GMM_EBUDGET (-4)  /* admission would exceed the pool's state budget */
#define GMM_ETIMEOUT (-5) /* a bounded wait ran out */

/* ------------------------------------------------------------ state planes */
/* Per component i (rank order, 0 = best ranked) the state has 8 planes:
 * colour weight, mean R, G, B, variance; depth weight, mean, variance.
 * GMM_PLANE_FUSION is the per-pixel List-1 byte: bit 0 fused label, bits
 * 1-3 counter + 3, bit 4 depth model started. */
#define GMM_PLANE_W_C 0
#define GMM_PLANE_MU_R 1
#define GMM_PLANE_MU_G 2
#define GMM_PLANE_MU_B 3
#define GMM_PLANE_V_C 4
#define GMM_PLANE_W_D 5
#define GMM_PLANE_MU_D 6
#define GMM_PLANE_V_D 7
#define GMM_PLANE_FUSION 8
#define GMM_NUM_PLANES 8

/* State storage precision. Arithmetic is FP32 in both. */
#define GMM_PREC_F32 0 /* every plane float32 */
#define GMM_PREC_F16 1 /* means and variances float16, weights bfloat16 */

typedef struct gmm_ctx gmm_t;

/* Model configuration. gmm_config_init fills the defaults below; edit the
 * fields, then call gmm_create_ex. */
typedef struct gmm_config {
    int H, W;          /* frame size in pixels, >= 1 */
    int M;             /* components per pixel and stream, 3..5 (§III.A) */
    float alpha;       /* learning rate, 0 < alpha < 1 */
    float match_k;     /* match within k standard deviations, > 0 */
    float bg_T;        /* background weight fraction T, 0 < T < 1 */
    float init_var;    /* variance of a new colour component (levels^2), > 0 */
    float init_w;      /* weight of a replacing component, 0 < init_w < 1 */
    float init_var_d;  /* variance of a new depth component (mm^2), > 0; default init_var */
    float v_min_c;     /* colour variance floor, > 0; default 1 */
    float v_min_d;     /* depth variance floor, > 0; default 1 */
    int precision;     /* GMM_PREC_F32 (default) or GMM_PREC_F16 */
    int morph_open;    /* 1: mask_out gets a 3x3 opening of the fused mask */
    int mode;          /* GMM_MODE_FUSION (default) or GMM_MODE_AUGMENTED */
    float depth_scale; /* GMM_MODE_AUGMENTED: depth (mm) multiplier, > 0;
                          default 255/4095 (the 12-bit range onto the byte range) */
    unsigned int flags; /* GMM_FLAG_* for both streams; default 0 */
} gmm_config;

/* Model structure (§III.B). GMM_MODE_FUSION: a colour mixture (D = 3) and a
 * depth mixture (D = 1) per pixel, fused by List 1 (§III.C). Depth 0 is "no
 * reading": the depth mixture is left untouched and its answer is the colour
 * answer; the depth mixture starts at the first non-zero reading.
 * GMM_MODE_AUGMENTED: the alternative §III.B sets aside, one mixture per
 * pixel over (R, G, B, depth_scale * depth) with the colour parameters
 * (init_var, v_min_c); a zero reading takes the best-ranked component's depth
 * mean (0 on the first frame). Its foreground is the mask; fg_rgb and fg_d
 * outputs, if given, receive the same bits. State: w, mu_R, mu_G, mu_B and
 * v in the colour planes, the depth-channel mean in GMM_PLANE_MU_D; planes
 * W_D and V_D are zero. */
#define GMM_MODE_FUSION 0
#define GMM_MODE_AUGMENTED 1

/* Readings of §III.A the paper leaves open (defaults: neither). The match
 * test d^2 < k^2 v and the rank key w / sqrt(v) are the same under all.
 * GMM_FLAG_RHO_ETA: the matched component's mean and variance move with
 * rho = alpha * N(x; mu, sigma^2 I) (Stauffer-Grimson's second learning
 * rate), evaluated with the parameters before the update and capped at 1;
 * default rho = alpha.
 * GMM_FLAG_VAR_PER_CHANNEL: v tracks the squared distance divided by D (the
 * per-channel variance sigma^2, so the match test is the Mahalanobis test);
 * default: v tracks the summed squared distance and sigma^2 = v / D. */
#define GMM_FLAG_RHO_ETA 1u
#define GMM_FLAG_VAR_PER_CHANNEL 2u
/* Storage option, GMM_PREC_F16 only (not part of the method): the bfloat16
 * weights are stored with stochastic rounding (round up with probability
 * equal to the dropped fraction; random bits from a counter-based hash of
 * the model's tick count, the pixel and the component), so a weight's
 * expected stored value equals its FP32 value instead of stalling when an
 * update is below half a bfloat16 step. Not available to
 * gmm_apply_open3_noalloc, which has no tick count. */
#define GMM_FLAG_STOCHASTIC_WEIGHTS 4u

/* Fill *cfg with the given model parameters and the defaults above. */
void gmm_config_init(gmm_config *cfg, int H, int W, int M, float alpha,
                     float match_k, float bg_T, float init_var, float init_w);

/* Create a model for H x W frames (§III.A: M Gaussians per pixel, weights
 * positive and summing to one; §III.B: one mixture per modality). FP32
 * state, defaults of gmm_config_init. Allocates the state in device memory
 * of the current CUDA device. Returns NULL on error (GMM_EINVAL for
 * out-of-range parameters, GMM_ENOMEM, GMM_ECUDA); see gmm_last_error(). */
gmm_t *gmm_create(int H, int W, int M, float alpha, float match_k, float bg_T,
                  float init_var, float init_w);

/* As gmm_create, from a full configuration. */
gmm_t *gmm_create_ex(const gmm_config *cfg);

/* Stream for all later work of the handle (a cudaStream_t; NULL = legacy
 * default stream). The caller keeps the stream alive. */
int gmm_set_stream(gmm_t *h, void *cuda_stream);

/* Failure-path test hook (no counterpart in the paper): records cuda_error
 * (a nonzero cudaError_t value) as the handle's sticky CUDA failure, exactly
 * as a failing CUDA call on the handle would, so that the error path can be
 * exercised without a GPU fault. Every later call that would launch work or
 * copy returns GMM_ECUDA; the handle can only be destroyed. GMM_EINVAL for a
 * NULL handle or a zero code. */
int gmm_inject_cuda_error(gmm_t *h, int cuda_error);

/* Self-test of the bounded device wait the staged kernel relies on (no
 * counterpart in the paper). Launches one thread that waits on a barrier
 * that nothing completes, with the same time-bounded wait; the wait must run
 * out after timeout_ms (1..2000), the kernel records it and returns, and the
 * context stays usable. On GMM_OK, *timed_out = 1 if the device reported the
 * timeout and *waited_ms the time it waited. Synchronous on the current
 * device; allocates 16 bytes of device memory for the results. GMM_EINVAL
 * for out-of-range arguments, GMM_ECUDA if a CUDA call fails. */
int gmm_wait_selftest(int timeout_ms, int *timed_out, double *waited_ms);

/* Tick kernel of the handle (§IV: the per-pixel GPU pass). Both compute the
 * same arithmetic bit for bit. GMM_KERNEL_DIRECT (default): one thread per
 * pixel, coalesced loads and stores straight from and to HBM (always used
 * for the initialising tick; FP16/BF16 state: two pixels per thread);
 * variant picks the CTA size (0, the default: the measured best for the
 * precision, 128 threads for FP32 and 64 for FP16/BF16; 1..4: 256, 128, 64,
 * 32 threads), ctas_per_sm is ignored.
 * GMM_KERNEL_STAGED: persistent CTAs stream tiles of the state through
 * shared memory with bulk copies in a multi-stage pipeline; variant picks
 * the depth (0..3: 2..5 stages of one 256-pixel tile each), ctas_per_sm the
 * residency (0 = as many as fit); the augmentation mode always uses the
 * direct kernel. A staged pipeline wait that runs out is reported by
 * gmm_sync as GMM_ETIMEOUT. */
#define GMM_KERNEL_STAGED 0
#define GMM_KERNEL_DIRECT 1
int gmm_set_kernel(gmm_t *h, int kind, int variant, int ctas_per_sm);

/* One tick (§III.A-C, §IV): both mixtures and the List-1 fusion for one
 * RGB-D frame, in one fused kernel. rgb8, depth16: device, read-only.
 * mask_out: device, receives the fused foreground (bit-packed, see top), or
 * its 3x3 opening when the handle was created with morph_open = 1. Any of
 * the three may instead be page-locked host memory mapped into the device's
 * address space (cudaHostAlloc or cudaHostRegister under unified
 * addressing): the kernel then reads the frame or writes the mask there
 * directly over the host link, with no separate copy (zero-copy).
 * Asynchronous on the handle's stream. The first call after create (or
 * gmm_reset) initialises the models from this frame. The direct tick (and
 * the opening) is launched as a programmatic dependent of the kernel before
 * it on the stream: it may be scheduled while that kernel's last CTAs run,
 * but reads nothing until that kernel has completed and its writes are
 * visible, so stream order holds as for any launch. */
int gmm_apply(gmm_t *h, const uint8_t *rgb8, const uint16_t *depth16,
              uint32_t *mask_out);

/* As gmm_apply, and also writes the per-stream foregrounds (colour and
 * depth, before fusion; bit-packed like mask_out) where the pointers are
 * not NULL (§V.A compares the colour, depth and fused answers). */
int gmm_apply_ex(gmm_t *h, const uint8_t *rgb8, const uint16_t *depth16,
                 uint32_t *mask_out, uint32_t *fg_rgb_out, uint32_t *fg_d_out);

/* One tick from host memory (§IV, Fig. 4(a): frames cross the bus each
 * tick). rgb8_host, depth16_host: host, read; mask_host: host, written.
 * Copies the frame in, runs gmm_apply, copies the mask out, and returns when
 * the mask is in host memory. Staging buffers are owned by the handle and
 * allocated on first use. Page-locked host buffers give overlapped copies. */
int gmm_apply_host(gmm_t *h, const uint8_t *rgb8_host,
                   const uint16_t *depth16_host, uint32_t *mask_host);

/* Pipelined host path (§IV, Fig. 4(a)): queue frame i's upload, compute and
 * mask download and return at once; up to GMM_PIPE_DEPTH frames may be in
 * flight, so the upload of frame i+1 and the download of frame i-1 overlap
 * the compute of frame i. The host buffers must stay valid (and the mask
 * unread) until gmm_pipe_wait returns for that frame; page-locked buffers
 * are required for overlap. Returns a ticket >= 0, or a negative status. */
#define GMM_PIPE_DEPTH 3
long long gmm_pipe_submit(gmm_t *h, const uint8_t *rgb8_host,
                          const uint16_t *depth16_host, uint32_t *mask_host);

/* Wait (bounded by timeout_ms; < 0 = no bound) until ticket's mask is in
 * host memory. GMM_ETIMEOUT if the bound ran out. */
int gmm_pipe_wait(gmm_t *h, long long ticket, int timeout_ms);

/* Copy one state plane to host memory, converted to float, row-major H*W
 * (dst_host: host, n >= H*W). plane: GMM_PLANE_*; component: rank 0..M-1
 * (ignored for GMM_PLANE_FUSION, whose bytes are returned as exact floats).
 * Synchronous: waits for the handle's stream. */
int gmm_state_get(const gmm_t *h, int plane, int component, float *dst_host,
                  size_t n);

/* Load one state plane from host floats (converted to the storage
 * precision; GMM_PLANE_FUSION takes byte values 0..255). Marks the model as
 * initialised, so the next tick updates instead of restarting. For tests,
 * checkpoint restore and migration. Synchronous. */
int gmm_state_set(gmm_t *h, int plane, int component, const float *src_host,
                  size_t n);

/* The next tick re-initialises every model from its frame. */
int gmm_reset(gmm_t *h);

/* Wait for the handle's stream. */
int gmm_sync(gmm_t *h);

/* Free the state and staging buffers. Waits for outstanding work. */
int gmm_destroy(gmm_t *h);

/* Thread-local message of the last failed call on this thread. */
const char *gmm_last_error(void);

/* Words per mask row (ceil(W/32)) and device bytes of one model's state. */
int gmm_mask_words_per_row(int W);
size_t gmm_state_bytes(int H, int W, int M, int precision);

/* ---------------------------------------------------- standalone operators */
/* List 1 (§III.C) alone: fuse two bit-packed binary foregrounds (device,
 * mask layout) with the per-pixel fusion bytes (device, H*W, updated in
 * place; only bits 0-3 are used and changed) into mask_out (device).
 * Asynchronous on `stream`. */
int gmm_fuse_masks(const uint32_t *fg_rgb, const uint32_t *fg_d,
                   uint8_t *fusion, uint32_t *mask_out, int H, int W,
                   void *stream);

/* 3x3 morphological opening (erosion then dilation, 3x3 square, pixels
 * outside the image are 0) of a bit-packed mask. Not in the paper: an
 * optional clean-up of the fused output. mask_in, mask_out: device, must not
 * overlap. Asynchronous on `stream`. */
int gmm_morph_open3(const uint32_t *mask_in, uint32_t *mask_out, int H, int W,
                    void *stream);

/* Pack a byte mask (device, H*W bytes row-major, non-zero = foreground) into
 * the bit-packed mask layout (device). Asynchronous on `stream`. */
int gmm_pack_mask(const uint8_t *bytes, uint32_t *mask_out, int H, int W,
                  void *stream);

/* Confusion counts of a predicted mask against a ground-truth mask (both
 * bit-packed, device), the quantities of the paper's evaluation (§V.A):
 * recall R = TP/(TP+FN) (Eq. 1), precision P = TP/(TP+FP) (Eq. 2), F1 =
 * 2PR/(P+R) (Eq. 3). counts_out: device, 4 unsigned 64-bit values
 * {TP, FP, FN, TN}, overwritten. Asynchronous on `stream`. */
int gmm_mask_confusion(const uint32_t *pred, const uint32_t *truth, int H, int W,
                       unsigned long long *counts_out, void *stream);

/* ------------------------------------------------- allocation-free variant */
/* The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory, such as a host application that
 * reserves all of the GPU's memory at start-up and hands out pieces of it,
 * a real-time loop that may not stall on the allocator, or code that runs
 * where allocation calls are not allowed. It performs one tick followed by
 * the 3x3 opening (what gmm_apply does for a handle created with
 * morph_open = 1) without any handle and without calling cudaMalloc,
 * cudaFree or any allocating routine.
 *
 * The caller provides the model state: `state` is device memory of
 * gmm_state_bytes(H, W, M, precision) bytes, 16-byte aligned. Pixels are
 * numbered p = y*Wp + x with Wp = ceil(W/32)*32 and grouped in tiles of 256
 * pixels of 8*M*256 elements each (i the rank, f a GMM_PLANE_* field).
 * GMM_PREC_F32: float32; field f of component i at pixel p is element
 * ((p/256)*8*M + 8*i + f)*256 + p%256. GMM_PREC_F16: 2-byte elements
 * (bfloat16 weights, float16 means and variances); per component and pixel
 * two groups of four slots, group 0 = {W_C, W_D, MU_R, MU_G}, group 1 =
 * {MU_B, V_C, MU_D, V_D}; field f of component i at pixel p is element
 * (p/256)*8*M*256 + ((2*i + group)*256 + p%256)*4 + slot.
 * The ceil(H*Wp/256) tiles are followed by one List-1 byte per tiled pixel. The state
 * persists between calls; first = 1 initialises it from this frame (it
 * need not be cleared beforehand), first = 0 updates it. cfg gives the
 * model parameters (its morph_open field is ignored). rgb8, depth16 and
 * mask_out are as for gmm_apply; mask_out receives the opened mask.
 * Asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).
 *
 * The fused mask before the opening is kept in one fixed array of device
 * memory inside the library, GMM_NOALLOC_MAX_MASK_WORDS words (1 MiB), that
 * every GPU loading the library holds until the process exits. Frames with
 * H*ceil(W/32) above that limit (more than 8,388,608 pixels, e.g. 4096 x
 * 2048) are rejected with GMM_EINVAL. All calls share the array: calls that
 * can overlap on the GPU (different streams, or other threads) race on it
 * and must be serialised by the caller. The first call in each CUDA context
 * (per device, and again after cudaDeviceReset or in another context the
 * caller made current) looks up the array's device address; under lazy
 * module loading, the CUDA default, that first call also loads the module
 * that holds the array, which needs its 1 MiB of free device memory and can
 * fail with GMM_ECUDA when the application has already taken the rest.
 * Make one warm-up call per device at start-up, before reserving the GPU's
 * memory and before any stream capture; later calls allocate nothing. */
#define GMM_NOALLOC_MAX_MASK_WORDS (1 << 18)
int gmm_apply_open3_noalloc(const gmm_config *cfg, void *state, int first,
                            const uint8_t *rgb8, const uint16_t *depth16,
                            uint32_t *mask_out, void *stream);

/* ------------------------------------------------------ multi-camera pool */
/* Many cameras (the paper's future work, §VI: several RGB-D sensors), each
 * with its own resident model, advanced together: one persistent kernel
 * launch per tick walks a tile worklist over every camera that has a frame
 * submitted. All cameras of a pool share its storage precision. */
typedef struct gmm_pool gmm_pool_t;

/* budget_bytes: cap on the summed state of admitted cameras (0 = no cap).
 * max_cams: slot count (>= 1). Allocation of a camera's state happens at
 * admission. */
gmm_pool_t *gmm_pool_create(size_t budget_bytes, int precision, int max_cams);

/* Admit a camera (cfg->precision must equal the pool's). Returns its slot
 * id >= 0, GMM_EBUDGET if its state would exceed the budget, GMM_EINVAL,
 * GMM_ENOMEM (also when every slot is taken). */
int gmm_pool_admit(gmm_pool_t *p, const gmm_config *cfg);

/* Free a camera's slot and state. Waits for the pool's stream first. */
int gmm_pool_release(gmm_pool_t *p, int cam);

/* Queue camera cam's next frame for the next gmm_pool_tick (device
 * pointers, layouts as gmm_apply; fg pointers may be NULL). A second submit
 * for the same camera before the tick replaces the first. */
int gmm_pool_submit(gmm_pool_t *p, int cam, const uint8_t *rgb8,
                    const uint16_t *depth16, uint32_t *mask_out,
                    uint32_t *fg_rgb_out, uint32_t *fg_d_out);

/* n submissions in one call: entry i is (cams[i], rgb8[i], depth16[i],
 * mask_out[i]) as for gmm_pool_submit (no per-stream masks). Host arrays of
 * n entries each; the pointers they hold are device pointers. Stops at the
 * first bad entry and returns its status (earlier entries stay submitted). */
int gmm_pool_submit_many(gmm_pool_t *p, int n, const int *cams,
                         const uint8_t *const *rgb8, const uint16_t *const *depth16,
                         uint32_t *const *mask_out);

/* Advance every submitted camera by one frame in one launch (asynchronous
 * on the pool's stream), then clear the submissions. */
int gmm_pool_tick(gmm_pool_t *p);

/* As gmm_inject_cuda_error, for a pool: later ticks return GMM_ECUDA. */
int gmm_pool_inject_cuda_error(gmm_pool_t *p, int cuda_error);

int gmm_pool_set_stream(gmm_pool_t *p, void *cuda_stream);

/* Launch shape of the pooled kernel: threads per block (64..256, a
 * multiple of 32); CTAs per SM of the persistent form (>= 1; its CTAs loop
 * over tiles of tile_pixels pixels, a multiple of the block size), or -1
 * for the flat form (a grid over the launch's pixels in which every warp
 * takes one chunk of 32 pixels, FP32, or 64, FP16/BF16, and exits;
 * tile_pixels is then unused). 0 keeps the current value (initially: 128
 * threads, as many persistent CTAs as fit, 2048-pixel tiles). */
int gmm_pool_set_launch(gmm_pool_t *p, int threads, int ctas_per_sm,
                        int tile_pixels);

/* Next-tile prefetch of the FP16/BF16 persistent form (enable = 1, the
 * default; 0 turns it off). With a launch shape whose tiles hold at most two
 * pixels per thread, a CTA takes its next tile when the current one starts
 * (except in the last two waves of a tick's tiles) and prefetches that
 * tile's first pixels' state into L2. Measured on the 64-camera mix: 94-95%
 * of the HBM copy bandwidth instead of 90-91% with the frames in device
 * memory, and no loss with frames read over the host link; but when frames
 * are uploaded on a copy stream beside each tick, the uploads slow down
 * (end to end 29 against 36-40 Gpixel-frames/s) and the online tuner's
 * trial ticks do not show it, so such pipelines should turn it off. It
 * changes no result (bit for bit the same either way) and does nothing for
 * FP32 pools. Applies from the next tick. GMM_EINVAL on a null pool. */
int gmm_pool_set_prefetch(gmm_pool_t *p, int enable);

/* Time each candidate launch shape on the current submissions (the state is
 * snapshotted and restored around the trials, so the models do not move)
 * and keep the fastest. Requires a submitted tick; leaves it submitted.
 * Writes the chosen shape to *threads, *ctas_per_sm, *tile_pixels when not
 * NULL. Synchronous. */
int gmm_pool_autotune(gmm_pool_t *p, int iters, int *threads,
                      int *ctas_per_sm, int *tile_pixels);

/* Online tuning of the launch shape on real ticks: the next
 * ticks_per_shape x (number of candidates) calls of gmm_pool_tick each run
 * one candidate shape (block size 64/128/256; the persistent form at full or
 * half residency with tiles of 256/512/1024/2048/8192 pixels; round-robin, CUDA
 * graphs off meanwhile; the flat form is chosen only explicitly). Each such tick is timed on the
 * pool's stream from its start to the start of the next tick (the tick
 * period, so whatever the tick's kernel delays among the work queued before
 * the next tick, such as uploads of the next frames, counts against its
 * shape). Once every trial has completed, the 4 shapes with the lowest median
 * periods run a second round of 2 x ticks_per_shape ticks each (ticks
 * between the rounds, until the first round's timings are read, keep the
 * last trial's shape), and the one with the lowest median period in that
 * round is kept and graph use restored. The ticks do their
 * normal work, so nothing is snapshotted. gmm_pool_set_launch during tuning
 * is overridden. */
int gmm_pool_autotune_online(gmm_pool_t *p, int ticks_per_shape);

/* Polls online tuning (non-blocking). Returns 1 while it is still running,
 * 0 when done (or never started), < 0 on error; writes the current shape to
 * the non-NULL outputs. */
int gmm_pool_tuning(gmm_pool_t *p, int *threads, int *ctas_per_sm, int *tile_pixels);

/* Run the pool's tick as a CUDA graph (enable = 1): the graph of the tick's
 * launches is built once and replayed every tick, its kernel nodes updated
 * with the tick's cameras; it is rebuilt when the number of launches (one
 * per 128 cameras), the launch shape or the kernel instance changes. */
int gmm_pool_use_graph(gmm_pool_t *p, int enable);

/* As gmm_state_get, for camera cam. */
int gmm_pool_state_get(const gmm_pool_t *p, int cam, int plane, int component,
                       float *dst_host, size_t n);

/* Summed state bytes of admitted cameras, and the budget. */
size_t gmm_pool_state_used(const gmm_pool_t *p);

/* Map `bytes` of device memory into the pool's allocator up front (at most
 * the budget): allocated and freed once, it stays reserved, so later
 * admissions take their state without mapping new device memory (mapping
 * can stall every thread of the process). Synchronous on the pool's stream;
 * counts nothing against the budget. GMM_ENOMEM if the device cannot
 * supply it, GMM_ECUDA on another CUDA failure (not sticky). */
int gmm_pool_reserve(gmm_pool_t *p, size_t bytes);

/* Wait for every tick queued on the pool's stream. GMM_ECUDA if a CUDA
 * failure is sticky on the pool. */
int gmm_pool_sync(gmm_pool_t *p);

/* Wait for the pool's stream, then free every camera's state, the pool's
 * buffers and the pool itself (p is invalid afterwards). */
int gmm_pool_destroy(gmm_pool_t *p);

/* ---------------------------------------------------------------- serving */
/* Frames from many cameras arriving in host memory at their own pace (the
 * paper's per-sensor frame stream, §IV, Fig. 4(a), for several sensors as in
 * §VI), served with continuous batching: an engine thread repeatedly forms a
 * tick from every camera that has a queued frame and no frame in flight,
 * advances those frames together with one pooled launch, and records each
 * frame's latency from its arrival time to its mask being in host memory.
 * Frames that arrive while a tick is on the GPU join a later tick, which is
 * queued behind it at once. Each camera's model stays resident in device
 * memory between its frames.
 *
 * Transfer modes (gmm_server_set_transfer):
 *   GMM_SERVE_ZERO_COPY (default): the pooled kernel reads each frame and
 *     writes each mask in the caller's page-locked host memory directly,
 *     over the coherent host link; no copies and no per-camera device
 *     buffers.
 *   GMM_SERVE_COPY: the engine uploads each frame into a per-camera device
 *     buffer and downloads the mask (Fig. 4(a)'s three-stage pipeline), the
 *     uploads, compute and downloads of consecutive ticks overlapping on
 *     separate streams. */
#define GMM_SERVE_ZERO_COPY 0
#define GMM_SERVE_COPY 1
typedef struct gmm_server gmm_server_t;

typedef struct gmm_server_stats {
    long long pushed, completed, dropped; /* frames */
    long long admitted, rejected, released; /* camera sessions */
    long long ticks;                      /* pooled launches */
    long long pixels;                     /* pixels of completed frames */
    int live_cams;
    size_t budget_bytes, used_bytes;      /* state (+ staging, copy mode) of admitted cameras */
    double max_engine_gap_ms;             /* longest time between two passes of the
                                             engine's loop (a pass waits at most
                                             0.2 ms for work; a longer gap means the
                                             thread was blocked, in a CUDA call or a
                                             lock, or not scheduled) */
} gmm_server_stats;

/* budget_bytes caps the device memory of admitted cameras (state, plus in
 * the copy mode the per-camera upload and mask buffers; 0 = no cap).
 * max_cams: slots.
 * queue_depth: frames a camera may have waiting (>= 1). Starts the engine
 * thread on the current device. NULL on error. */
gmm_server_t *gmm_server_create(size_t budget_bytes, int precision, int max_cams,
                                int queue_depth);

/* Choose the transfer mode (GMM_SERVE_ZERO_COPY or GMM_SERVE_COPY) before the
 * first admission; GMM_EINVAL afterwards or for another value. */
int gmm_server_set_transfer(gmm_server_t *s, int mode);

/* Admit a camera (cfg->precision must equal the server's). Returns its id,
 * or GMM_EBUDGET when its memory would exceed the budget (the admission is
 * rejected and counted), or another negative status. */
int gmm_server_admit(gmm_server_t *s, const gmm_config *cfg);

/* As gmm_pool_reserve for the server: state_bytes for camera state,
 * staging_bytes for the per-camera upload and mask buffers of the copy mode
 * (0 in the zero-copy mode); same statuses.
 * May be called from any thread; synchronous: it waits for the work queued
 * on the engine's compute stream, so call it before the frames flow. */
int gmm_server_reserve(gmm_server_t *s, size_t state_bytes, size_t staging_bytes);

/* End a camera's session: waits (up to timeout_ms; < 0 = no bound) until
 * its queued frames are done, then frees its slot and memory. */
int gmm_server_release(gmm_server_t *s, int cam, int timeout_ms);

/* Queue one frame. rgb8_host, depth16_host: host memory, page-locked (in
 * the zero-copy mode the device must be able to reach it, else GMM_EINVAL;
 * in the copy mode page-locked memory lets the uploads overlap), read when
 * the frame's tick runs; mask_host: host, receives the fused mask. All three
 * must stay valid and unmodified until the frame is done. t_arrival: arrival
 * time on the gmm_server_now() clock. Returns a ticket >= 0, or GMM_EBUDGET if
 * the camera's queue is full (the frame is dropped and counted), or another
 * negative status. */
long long gmm_server_push(gmm_server_t *s, int cam, const uint8_t *rgb8_host,
                          const uint16_t *depth16_host, uint32_t *mask_host,
                          double t_arrival);

/* 1 if the ticket's mask is in host memory, 0 if not yet, < 0 on error. */
int gmm_server_done(gmm_server_t *s, long long ticket);

/* Wait (up to timeout_ms; < 0 = no bound) for a ticket. GMM_ETIMEOUT if the
 * bound ran out. */
int gmm_server_wait(gmm_server_t *s, long long ticket, int timeout_ms);

/* Counters, and the per-frame latencies in milliseconds (arrival to mask in
 * host memory, in completion order; the most recent 1,048,576 frames are
 * kept): copies up to n, returns how many are kept. */
int gmm_server_stats_get(gmm_server_t *s, gmm_server_stats *out);
size_t gmm_server_latencies(gmm_server_t *s, float *ms_out, size_t n);

/* Where a completed frame's latency went, on the gmm_server_now() clock
 * (seconds): t_arrival as given to gmm_server_push; t_pushed when that call
 * queued it; t_batched when the engine took the frame into a tick;
 * t_submitted when that tick's launch (and copies, in the copy mode) were
 * queued on the device; t_done when the engine saw the tick complete, its
 * masks in host memory (the latency's end). cam: the server's camera id;
 * tick_frames: frames in the same tick. */
typedef struct gmm_server_trace {
    long long ticket;
    int cam, tick_frames;
    double t_arrival, t_pushed, t_batched, t_submitted, t_done;
} gmm_server_trace;

/* Copies up to n records, in completion order (the records of
 * gmm_server_latencies, the same frames), into out; returns how many are
 * kept. */
size_t gmm_server_traces(gmm_server_t *s, gmm_server_trace *out, size_t n);

/* Seconds on the engine's monotonic clock (the clock of t_arrival). */
double gmm_server_now(void);

/* Stops the engine after the queued frames are done (waits up to
 * timeout_ms), frees everything. */
int gmm_server_destroy(gmm_server_t *s, int timeout_ms);

#ifdef __cplusplus
}
#endif

#endif /* GMM_H */
