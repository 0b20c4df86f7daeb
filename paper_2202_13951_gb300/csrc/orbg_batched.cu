/*
 * orbg_batched.cu -- the batched form: a persistent launch whose warps pull
 * blocks, possibly of different codes, from an atomic work queue.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_decode_block.cuh"

using namespace orbg_dev;

namespace {

template <int KMAX, int WMAX>
__global__ void __launch_bounds__(512) orbg_batched_kernel(
    const OrbgDeviceCode *__restrict__ codes, int ncodes, const int32_t *__restrict__ code_id,
    const int64_t *__restrict__ llr_off, const float *__restrict__ llr, int64_t B, uint32_t cap,
    uint8_t *__restrict__ cw, const int64_t *__restrict__ cw_off, uint32_t *__restrict__ q,
    uint8_t *__restrict__ ab, unsigned long long *__restrict__ counter, uint32_t wstride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    unsigned char *wsm = smem + warp * wstride;
    const int64_t n0 = codes[0].n;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0)
            b = atomicAdd(counter, 1ull);
        b = __shfl_sync(FULL_MASK, b, 0);
        if ((int64_t)b >= B)
            break;
        int cid = code_id ? code_id[b] : 0;
        if (cid < 0 || cid >= ncodes) {
            if (lane == 0) {
                q[b] = 0u;
                ab[b] = 2;
            }
            continue;
        }
        const OrbgDeviceCode code = codes[cid];
        const int64_t lo = llr_off ? llr_off[b] : (int64_t)b * n0;
        const int64_t co = cw_off ? cw_off[b] : (int64_t)b * n0;
        decode_any<KMAX, WMAX>(code, llr + lo, cw + co, q + b, ab + b, cap, wsm, lane);
    }
}

}  // namespace

namespace {

template <int KMAX, int WMAX>
cudaError_t launch_batched_t(const OrbgDeviceCode *d_codes, int ncodes, int n_max, int w32_max,
                             const int32_t *code_id, const int64_t *llr_off, const float *llr,
                             int64_t B, uint32_t cap, uint8_t *cw, const int64_t *cw_off,
                             uint32_t *q, uint8_t *ab, unsigned long long *counter,
                             int warps_per_cta, int ctas_per_sm, cudaStream_t st)
{
    auto kern = orbg_batched_kernel<KMAX, WMAX>;
    int wpc = warps_per_cta > 0 ? warps_per_cta : 8;
    uint32_t wstride = warp_smem_bytes(n_max, w32_max);
    size_t smem = (size_t)wstride * wpc;
    cudaError_t e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int per_sm = ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ;
    int64_t grid = (int64_t)sms * per_sm;
    int64_t need = (B + wpc - 1) / wpc;
    if (grid > need) grid = need > 0 ? need : 1;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st)) != cudaSuccess)
        return e;
    kern<<<(unsigned)grid, wpc * 32, smem, st>>>(d_codes, ncodes, code_id, llr_off, llr, B, cap,
                                                 cw, cw_off, q, ab, counter, wstride);
    return cudaGetLastError();
}

}  // namespace

int orbg_launch_batched(const OrbgDeviceCode *d_codes, int ncodes, int n_max, int w32_max,
                        const int32_t *code_id, const int64_t *llr_off, const float *llr,
                        int64_t B, uint32_t cap, uint8_t *cw, const int64_t *cw_off,
                        uint32_t *q, uint8_t *ab, unsigned long long *counter,
                        int warps_per_cta, int ctas_per_sm, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
#define ORBG_B(KM, WM)                                                                       \
    return (int)launch_batched_t<KM, WM>(d_codes, ncodes, n_max, w32_max, code_id, llr_off, \
                                         llr, B, cap, cw, cw_off, q, ab, counter,            \
                                         warps_per_cta, ctas_per_sm, st);
#define ORBG_BW(KM)                 \
    if (w32_max <= 1) { ORBG_B(KM, 1) } \
    else if (w32_max <= 2) { ORBG_B(KM, 2) } \
    else { ORBG_B(KM, 4) }
    if (n_max <= 32) {
        ORBG_BW(1)
    } else if (n_max <= 64) {
        ORBG_BW(2)
    } else if (n_max <= 128) {
        ORBG_BW(4)
    } else {
        ORBG_BW(8)
    }
#undef ORBG_BW
#undef ORBG_B
}
