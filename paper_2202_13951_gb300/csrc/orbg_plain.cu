/*
 * orbg_plain.cu -- the plain form: one launch, one warp per block in a static
 * grid (Algorithm 1 per block; see orbg_decode_block.cuh).
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_decode_block.cuh"

using namespace orbg_dev;

namespace {

template <int K, int W>
__global__ void __launch_bounds__(256) orbg_plain_kernel(OrbgDeviceCode code,
                                                         const float *__restrict__ llr,
                                                         int64_t B, uint32_t cap,
                                                         uint8_t *__restrict__ cw,
                                                         uint32_t *__restrict__ q,
                                                         uint8_t *__restrict__ ab,
                                                         uint32_t wstride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= B)
        return; /* whole warp */
    const int64_t off = b * (int64_t)code.n;
    decode_block_warp<K, W, false, false, true, (K >= 8)>(code, llr + off, cw + off, q + b,
                                                          ab + b, cap, cap, smem + warp * wstride,
                                                          lane, nullptr, nullptr, 0ull);
}

template <int K, int W>
cudaError_t launch_plain_t(const OrbgDeviceCode &code, const float *llr, int64_t B, uint32_t cap,
                           uint8_t *cw, uint32_t *q, uint8_t *ab, cudaStream_t st)
{
    const int wpc = 8;
    uint32_t wstride = block_smem_bytes(code.n, W);
    size_t smem = (size_t)wstride * wpc;
    int64_t grid = (B + wpc - 1) / wpc;
    if (grid > 0x7FFFFFFF)
        return cudaErrorInvalidValue;
    orbg_plain_kernel<K, W><<<(unsigned)grid, wpc * 32, smem, st>>>(code, llr, B, cap, cw, q, ab,
                                                                      wstride);
    return cudaGetLastError();
}

}  // namespace

int orbg_launch_plain(const OrbgDeviceCode &code, const float *llr, int64_t B, uint32_t cap,
                      uint8_t *cw, uint32_t *q, uint8_t *ab, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int n = code.n, w = code.w32;
#define ORBG_PLAIN(KK)                                                            \
    return (int)(w == 1 ? launch_plain_t<KK, 1>(code, llr, B, cap, cw, q, ab, st) \
                 : w == 2 ? launch_plain_t<KK, 2>(code, llr, B, cap, cw, q, ab, st) \
                          : launch_plain_t<KK, 4>(code, llr, B, cap, cw, q, ab, st));
    if (n <= 32) {
        ORBG_PLAIN(1)
    } else if (n <= 64) {
        ORBG_PLAIN(2)
    } else if (n <= 128) {
        ORBG_PLAIN(4)
    } else {
        ORBG_PLAIN(8)
    }
#undef ORBG_PLAIN
}

