/*
 * orbg_heavy.cuh -- phase 2 of the batched form: every CTA takes one block
 * left open by phase 1 at a time and searches it with all its warps
 * (decode_block_cta in orbg_decode_block.cuh).  Included by the
 * orbg_batched_k*.cu translation units; ONE as in orbg_batched.cuh.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_decode_block.cuh"

namespace orbg_batched_impl {

using namespace orbg_dev;

/* resident 512-thread phase-2 CTAs per SM the register allocation is sized for */
#ifndef ORBG_PHASE2_MIN_CTAS
#define ORBG_PHASE2_MIN_CTAS 2
#endif

template <int KMAX, int WMAX, bool ONE, bool STRIDE>
__global__ void __launch_bounds__(512, ORBG_PHASE2_MIN_CTAS) orbg_heavy_kernel(
    const OrbgDeviceCode *__restrict__ codes, int ncodes, const int32_t *__restrict__ code_id,
    const int64_t *__restrict__ llr_off, const float *__restrict__ llr, uint32_t cap,
    uint8_t *__restrict__ cw, const int64_t *__restrict__ cw_off, uint32_t *__restrict__ q,
    uint8_t *__restrict__ ab, unsigned long long *__restrict__ counters,
    const unsigned long long *__restrict__ heavy, const unsigned char *__restrict__ hand,
    uint32_t bstride, const __grid_constant__ OrbgDeviceCode code0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_block, s_slot;
    __shared__ uint32_t s_best;
    __shared__ uint4 s_s0;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int64_t n0 = ONE ? code0.n : codes[0].n;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long nheavy = *((volatile unsigned long long *)&counters[1]);
            const unsigned long long slot = atomicAdd(&counters[2], 1ull);
            /* block | tested-below << 32 | handover record << 63 */
            /* code sets take the list from its end: its phase-1 launches run
             * by decoder variant, shortest codes first, so the longest codes'
             * blocks, which search longest, list last and start first here */
            const unsigned long long r = ONE ? slot : nheavy - 1ull - slot;
            s_block = slot < nheavy ? heavy[r] : ~0ull;
            s_slot = r;
        }
        __syncthreads();
        const unsigned long long bb = s_block;
        if (bb == ~0ull)
            break; /* uniform: every thread read the same s_block */
        const int64_t b = (int64_t)(bb & 0xFFFFFFFFull);
        const uint32_t from = (uint32_t)((bb >> 32) & 0x7FFFFFFFull);
        const unsigned char *rec = (bb >> 63) ? hand + s_slot * ORBG_HANDOVER_BYTES : nullptr;
        const int64_t lo = llr_off ? llr_off[b] : b * n0;
        const int64_t co = cw_off ? cw_off[b] : b * n0;
        if (ONE) {
            decode_block_cta<KMAX, WMAX, STRIDE>(code0, llr + lo, cw + co, q + b, ab + b, cap, smem,
                                         reinterpret_cast<uint16_t *>(smem + bstride), &s_best,
                                         reinterpret_cast<typename Syn<WMAX>::T *>(&s_s0), from,
                                         warp, lane, nwarps, rec);
            continue;
        }
        const int cid = code_id ? code_id[b] : 0; /* checked in phase 1 */
        const OrbgDeviceCode code = codes[cid];
#define ORBG_CALL_CTA(KK, WW)                                                               \
    decode_block_cta<KK, WW, STRIDE>(code, llr + lo, cw + co, q + b, ab + b, cap, smem,              \
                             reinterpret_cast<uint16_t *>(smem + bstride), &s_best,          \
                             reinterpret_cast<typename Syn<WW>::T *>(&s_s0), from, warp, lane,  \
                             nwarps, rec)
        ORBG_DISPATCH(KMAX, WMAX, ORBG_CALL_CTA);
#undef ORBG_CALL_CTA
    }
    (void)ncodes;
}

template <int KMAX, int WMAX, bool ONE, bool STRIDE>
cudaError_t launch_heavy_k(const OrbgBatchedArgs &a, unsigned long long *counters,
                           const unsigned long long *heavy, const unsigned char *hand)
{
    auto k2 = orbg_heavy_kernel<KMAX, WMAX, ONE, STRIDE>;
    const int hw = a.heavy_warps > 0 ? a.heavy_warps : 16;
    const uint32_t bstride = block_smem_bytes(a.n_max, a.w32_max);
    const size_t smem = (size_t)bstride + triple_table_bytes(a.ntrip_max);
    int grid = 0;
    int rc = orbg_grid_for((const void *)k2, hw * 32, smem, 0, &grid);
    if (rc != 0)
        return (cudaError_t)rc;
    OrbgDeviceCode c0{};
    if (ONE)
        c0 = *a.code0;
    k2<<<grid, hw * 32, smem, (cudaStream_t)a.stream>>>(a.d_codes, a.ncodes, a.code_id,
                                                        a.llr_off, a.llr, a.cap, a.cw, a.cw_off,
                                                        a.q, a.ab, counters, heavy, hand, bstride,
                                                        c0);
    return cudaGetLastError();
}

/* One code: strided runs always handled (no cost measured there); code
 * sets: the kernel with them only where a code has them. */
template <int KMAX, int WMAX, bool ONE>
cudaError_t launch_heavy_t(const OrbgBatchedArgs &a, unsigned long long *counters,
                           const unsigned long long *heavy, const unsigned char *hand)
{
    if constexpr (ONE)
        return launch_heavy_k<KMAX, WMAX, true, true>(a, counters, heavy, hand);
    else
        return a.has_stride ? launch_heavy_k<KMAX, WMAX, false, true>(a, counters, heavy, hand)
                            : launch_heavy_k<KMAX, WMAX, false, false>(a, counters, heavy, hand);
}

}  // namespace orbg_batched_impl
