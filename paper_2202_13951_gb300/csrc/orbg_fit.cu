/*
 * orbg_fit.cu -- per-block piece-wise linear fitting and quantisation of the
 * ordered reliability curve on the device (Sec. III-E, Eq. Q, Eq. quant).
 *
 * One warp per received block, blocks taken in a grid-stride loop.  The
 * block's reliabilities |LLR| are staged in the warp's shared memory and
 * sorted ascending by a bitonic network over 256 slots (unused slots hold
 * +inf and sort last), which gives the ordered curve L_1 <= ... <= L_n of
 * Sec. III-A.  Lane 0 then places the anchors and quantises the segments
 * (orbg_fit.cuh).  The work per block is O(n log^2 n) compares and
 * O(lines * n) double operations: small beside one decode.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/orbg.h"
#include "orbg_fit.cuh"
#include "orbg_internal.h"

namespace {

constexpr int kWarps = 8;           /* warps per CTA */
constexpr int kSlots = 256;         /* sorted slots per block: n <= 256 */
static_assert(ORBG_FIT_WORDS == ORBG_FIT_STRIDE, "model record size");

__global__ void __launch_bounds__(kWarps * 32) orbg_fit_kernel(const float *__restrict__ llr,
                                                              int64_t B, int n, int lines,
                                                              int divisible,
                                                              int32_t *__restrict__ models)
{
    __shared__ float sm[kWarps][kSlots];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *s = sm[warp];
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t b = (int64_t)blockIdx.x * kWarps + warp; b < B; b += nwarps) {
        const float *x = llr + b * (int64_t)n;
        bool nan = false;
        for (int i = lane; i < kSlots; i += 32) {
            const float v = i < n ? x[i] : INFINITY;
            nan |= isnan(v);
            s[i] = fabsf(v);
        }
        nan = __any_sync(0xFFFFFFFFu, nan);
        int32_t *out = models + b * (int64_t)ORBG_FIT_STRIDE;
        if (nan) {
            for (int i = lane; i < ORBG_FIT_STRIDE; i += 32)
                out[i] = 0; /* m = 0 marks a NaN block */
            __syncwarp();
            continue;
        }
        __syncwarp();
        /* bitonic sort, ascending: each stage's 128 pairs, four per lane */
        for (int k = 2; k <= kSlots; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < kSlots / 2; t += 32)
                    orbg_fit::bitonic_step(s, k, j, t);
                __syncwarp();
            }
        }
        if (lane == 0) {
            int32_t res[ORBG_FIT_STRIDE];
            for (int i = 0; i < ORBG_FIT_STRIDE; i++)
                res[i] = 0;
            orbg_fit::fit_sorted(s, n, lines, divisible, res);
            for (int i = 0; i < ORBG_FIT_STRIDE; i++)
                out[i] = res[i];
        }
        __syncwarp();
    }
}

/* J_0 of a one-line record, as the fitted decoder groups blocks: NaN
 * blocks (m = 0) join J_0 = 0, and J_0 is held within [-1, top]. */
__device__ __forceinline__ int32_t line_j0(const int32_t *rec, int32_t top)
{
    const int32_t j0 = rec[0] == 0 ? 0 : rec[8];
    return j0 < -1 ? -1 : j0 > top ? top : j0;
}

__global__ void orbg_fit_mark_kernel(const int32_t *__restrict__ models, int64_t B, int32_t top,
                                     uint8_t *__restrict__ present)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x)
        present[line_j0(models + b * (int64_t)ORBG_FIT_STRIDE, top) + 1] = 1;
}

__global__ void orbg_fit_map_kernel(const int32_t *__restrict__ models, int64_t B, int32_t top,
                                    const int32_t *__restrict__ lut, int32_t *__restrict__ cid)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x)
        cid[b] = lut[line_j0(models + b * (int64_t)ORBG_FIT_STRIDE, top) + 1];
}

/* SMs of the current device (the grids below are grid-stride loops, so
 * any count gives the same result; 1 if the query fails) */
int64_t device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
        return 1;
    return sms;
}

unsigned grid_for(int64_t B, int threads)
{
    const int64_t g = (B + threads - 1) / threads, top = device_sms() * 8;
    return (unsigned)(g < top ? (g > 0 ? g : 1) : top);
}

bool device_accessible(const void *p)
{
    const cudaError_t pending = cudaPeekAtLastError(); /* left for the caller */
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        if (pending == cudaSuccess)
            cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

int orbg_fit_launch(const float *llr, int64_t B, int n, int lines, int divisible,
                    int32_t *models, void *stream)
{
    const int64_t ctas = (B + kWarps - 1) / kWarps, top = device_sms() * 16;
    const unsigned grid = (unsigned)(ctas < top ? ctas : top);
    orbg_fit_kernel<<<grid, kWarps * 32, 0, (cudaStream_t)stream>>>(llr, B, n, lines,
                                                                    divisible ? 1 : 0, models);
    return (int)cudaGetLastError();
}

extern "C" ORBG_API int orbg_fit_models(const float *llr, int64_t B, int n, int lines,
                                        int divisible, int32_t *models, void *cuda_stream)
{
    if (B < 0 || n < 1 || n > ORBG_MAX_N || lines < 1 || lines > ORBG_FIT_SEG)
        return ORBG_EINVAL;
    if (B == 0)
        return ORBG_OK;
    if (!llr || !models || !device_accessible(llr) || !device_accessible(models))
        return ORBG_EINVAL;
    const int e = orbg_fit_launch(llr, B, n, lines, divisible, models, cuda_stream);
    return e == 0 ? ORBG_OK : orbg_note_cuda_error(e);
}

int orbg_fit_mark_lines(const int32_t *models, int64_t B, int32_t top, uint8_t *present,
                        void *stream)
{
    orbg_fit_mark_kernel<<<grid_for(B, 256), 256, 0, (cudaStream_t)stream>>>(models, B, top,
                                                                             present);
    return (int)cudaGetLastError();
}

int orbg_fit_map_lines(const int32_t *models, int64_t B, int32_t top, const int32_t *lut,
                       int32_t *cid, void *stream)
{
    orbg_fit_map_kernel<<<grid_for(B, 256), 256, 0, (cudaStream_t)stream>>>(models, B, top, lut,
                                                                            cid);
    return (int)cudaGetLastError();
}
