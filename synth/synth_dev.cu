// Device side of the seeded synthetic RGB-D scene (see synth_core.h): the same
// per-pixel function as the host build, one thread per pixel, so frames can be
// produced directly in device memory outside any timed region.
#include <cuda_runtime.h>
#include <stdint.h>

#include "synth_core.h"

static __global__ void synth_frames_kernel(const synth_scene s, int f0, int nf,
                                           uint8_t *rgb, uint16_t *depth,
                                           uint8_t *gt)
{
    const int64_t N = (int64_t)s.H * s.W;
    const int64_t total = N * nf;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int f = (int)(i / N);
        int64_t p = i - (int64_t)f * N;
        int32_t y = (int32_t)(p / s.W), x = (int32_t)(p - (int64_t)y * s.W);
        uint8_t c[3], g;
        uint16_t d;
        synth_pixel(&s, f0 + f, x, y, c, &d, &g);
        rgb[3 * i] = c[0];
        rgb[3 * i + 1] = c[1];
        rgb[3 * i + 2] = c[2];
        depth[i] = d;
        if (gt)
            gt[i] = g;
    }
}

// Frames f0 .. f0+nf-1 into device buffers laid out like synth_frames_host.
// Asynchronous on `stream`; returns a cudaError_t value (0 = success).
extern "C" int synth_frames_device(const synth_scene *s, int f0, int nf,
                                   uint8_t *rgb, uint16_t *depth, uint8_t *gt,
                                   void *stream)
{
    if (!s || !rgb || !depth || nf < 0 || f0 < 0)
        return (int)cudaErrorInvalidValue;
    const int64_t total = (int64_t)s->H * s->W * nf;
    if (total == 0)
        return 0;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64)
        blocks = 152 * 64;
    synth_frames_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(*s, f0, nf, rgb, depth, gt);
    return (int)cudaGetLastError();
}
