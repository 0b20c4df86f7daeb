/*
 * orbg_batched.cu -- the batched form: two persistent launches over blocks
 * that may belong to different codes.
 *
 * Phase 1 (orbg_batched_kernel): each warp pulls `grab` blocks at a time
 * from an atomic work queue and decodes each with decode_block_warp, giving
 * it a query budget.  Most blocks finish inside the budget (at high SNR
 * query 1 already decodes).  A block still open when its warp reaches the
 * budget is appended to a heavy list.
 * Phase 2 (orbg_heavy_kernel, orbg_heavy.cu): each CTA pulls heavy blocks
 * one at a time and decodes each with all its warps (decode_block_cta), so a
 * block that needs up to 1e6 queries is searched by a whole SM instead of a
 * single warp.
 * Both phases compute the exact first hit of the same query order, so the
 * result equals the plain form's block for block.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_pipeline.h>

#include "orbg_decode_block.cuh"

using namespace orbg_dev;

namespace {

constexpr int kCounters = ORBG_BATCHED_COUNTERS;

/* resident phase-1 CTAs per SM the register allocation is sized for */
#ifndef ORBG_PHASE1_MIN_CTAS
#define ORBG_PHASE1_MIN_CTAS 3
#endif

template <int KMAX, int WMAX>
__global__ void __launch_bounds__(256, ORBG_PHASE1_MIN_CTAS) orbg_batched_kernel(
    const OrbgDeviceCode *__restrict__ codes, int ncodes, const int32_t *__restrict__ code_id,
    const int64_t *__restrict__ llr_off, const float *__restrict__ llr, int64_t B, uint32_t cap,
    uint32_t budget, uint8_t *__restrict__ cw, const int64_t *__restrict__ cw_off,
    uint32_t *__restrict__ q, uint8_t *__restrict__ ab, unsigned long long *__restrict__ counters,
    unsigned long long *__restrict__ heavy, uint32_t bstride, uint32_t x3w_bytes, int grab)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    unsigned char *bsm = smem + warp * bstride;
    /* two LLR slots per warp: the block being decoded and the next one,
     * copied in asynchronously while the current one is decoded */
    constexpr int kSlot = 32 * KMAX;
    float *ring = reinterpret_cast<float *>(smem + nwarps * bstride) + warp * 2 * kSlot;
    /* the warp's own triple table (sums <= ORBG_X3_WARP_S3), filled lazily */
    uint16_t *X3w = reinterpret_cast<uint16_t *>(smem + nwarps * (bstride + 2 * kSlot * 4) +
                                                 warp * x3w_bytes);
    const int64_t n0 = codes[0].n;

    /* the warp's block sequence: `grab` consecutive blocks per atomic */
    int64_t pos = 0, end = 0;
    auto next_block = [&]() -> int64_t {
        if (pos >= end) {
            unsigned long long c = 0;
            if (lane == 0)
                c = atomicAdd(&counters[0], (unsigned long long)grab);
            c = __shfl_sync(FULL_MASK, c, 0);
            pos = (int64_t)c;
            end = min(pos + (int64_t)grab, B);
            if (pos >= B)
                return B;
        }
        return pos++;
    };
    auto stage = [&](int64_t b, int slot) {
        if (b < B) {
            const int cid = code_id ? code_id[b] : 0;
            if (cid >= 0 && cid < ncodes) {
                const int n = codes[cid].n;
                const int64_t lo = llr_off ? llr_off[b] : b * n0;
#pragma unroll
                for (int k = 0; k < KMAX; k++) {
                    const int i = k * 32 + lane;
                    if (i < n)
                        __pipeline_memcpy_async(ring + slot * kSlot + i, llr + lo + i, 4);
                }
            }
        }
        __pipeline_commit();
    };

    int64_t b = next_block();
    int slot = 0;
    stage(b, slot);
    int64_t bn = next_block();
    while (b < B) {
        stage(bn, slot ^ 1);
        __pipeline_wait_prior(1); /* block b's copies have landed */
        __syncwarp();
        const int cid = code_id ? code_id[b] : 0;
        if (cid < 0 || cid >= ncodes) {
            if (lane == 0) {
                q[b] = 0u;
                ab[b] = 2;
            }
        } else {
            const OrbgDeviceCode code = codes[cid];
            const int64_t co = cw_off ? cw_off[b] : b * n0;
            const float *l = ring + slot * kSlot;
#define ORBG_CALL_WARP(KK, WW)                                                                 \
    decode_block_warp<KK, WW, true, true>(code, l, cw + co, q + b, ab + b, cap, budget, bsm,  \
                                          lane, heavy, &counters[1], (unsigned long long)b,  \
                                          X3w)
            ORBG_DISPATCH(KMAX, WMAX, ORBG_CALL_WARP);
#undef ORBG_CALL_WARP
        }
        __syncwarp(); /* slot is free before it is refilled */
        b = bn;
        bn = next_block();
        slot ^= 1;
    }
    __pipeline_wait_prior(0);
}

}  // namespace

int orbg_grid_for(const void *kern, int threads, size_t smem, int ctas_per_sm, int *grid_out)
{
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return (int)e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return (int)e;
    if (smem + fa.sharedSizeBytes > 48 * 1024) { /* static + dynamic past 48 KB: opt in */
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return (int)e;
    if (occ < 1) return (int)cudaErrorInvalidConfiguration;
    int per_sm = ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ;
    *grid_out = sms * per_sm;
    return 0;
}

namespace {

template <int KMAX, int WMAX>
cudaError_t launch_batched_t(const OrbgDeviceCode *d_codes, int ncodes, int n_max, int w32_max,
                             const int32_t *code_id, const int64_t *llr_off, const float *llr,
                             int64_t B, uint32_t cap, uint32_t budget, uint8_t *cw,
                             const int64_t *cw_off, uint32_t *q, uint8_t *ab,
                             unsigned long long *scratch, int warps_per_cta, int ctas_per_sm,
                             int grab, int heavy_warps, uint32_t ntrip_max, uint32_t x3w_max,
                             cudaStream_t st)
{
    const int wpc = warps_per_cta > 0 ? (warps_per_cta > 8 ? 8 : warps_per_cta) : 8;
    const int g = grab < 1 ? 1 : grab;
    const uint32_t bstride = block_smem_bytes(n_max, w32_max);
    unsigned long long *counters = scratch;
    unsigned long long *heavy = scratch + kCounters;
    cudaError_t e;
    int grid = 0, rc;
    if ((e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * kCounters, st)) !=
        cudaSuccess)
        return e;
    /* phase 1: per warp, one block's working set and two LLR slots */
    auto k1 = orbg_batched_kernel<KMAX, WMAX>;
    const uint32_t x3w_bytes = triple_table_bytes(x3w_max);
    size_t smem1 = ((size_t)bstride + 2u * 32u * KMAX * sizeof(float) + x3w_bytes) * wpc;
    if ((rc = orbg_grid_for((const void *)k1, wpc * 32, smem1, ctas_per_sm, &grid)) != 0)
        return (cudaError_t)rc;
    int64_t units = (B + g - 1) / g;
    int64_t need = (units + wpc - 1) / wpc;
    if (grid > need) grid = (int)(need > 0 ? need : 1);
    k1<<<grid, wpc * 32, smem1, st>>>(d_codes, ncodes, code_id, llr_off, llr, B, cap, budget, cw,
                                      cw_off, q, ab, counters, heavy, bstride, x3w_bytes, g);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if (budget >= cap)
        return cudaSuccess; /* every block finished in phase 1 */
    /* phase 2 */
    return (cudaError_t)orbg_launch_heavy(d_codes, ncodes, n_max, w32_max, code_id, llr_off, llr,
                                          cap, cw, cw_off, q, ab, counters, heavy, heavy_warps,
                                          ntrip_max, st);
}

}  // namespace

size_t orbg_batched_scratch_bytes(int64_t B)
{
    return sizeof(unsigned long long) * ((size_t)kCounters + (size_t)(B > 0 ? B : 0));
}

int orbg_launch_batched(const OrbgDeviceCode *d_codes, int ncodes, int n_max, int w32_max,
                        const int32_t *code_id, const int64_t *llr_off, const float *llr,
                        int64_t B, uint32_t cap, uint32_t budget, uint8_t *cw,
                        const int64_t *cw_off, uint32_t *q, uint8_t *ab,
                        unsigned long long *scratch, int warps_per_cta, int ctas_per_sm, int grab,
                        int heavy_warps, uint32_t ntrip_max, uint32_t x3w_max, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
#define ORBG_B(KM, WM)                                                                       \
    return (int)launch_batched_t<KM, WM>(d_codes, ncodes, n_max, w32_max, code_id, llr_off, \
                                         llr, B, cap, budget, cw, cw_off, q, ab, scratch,     \
                                         warps_per_cta, ctas_per_sm, grab, heavy_warps,      \
                                         ntrip_max, x3w_max, st);
#define ORBG_BW(KM)                          \
    if (w32_max <= 1) { ORBG_B(KM, 1) }      \
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
