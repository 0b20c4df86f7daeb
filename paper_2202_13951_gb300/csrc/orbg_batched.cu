/*
 * orbg_batched.cu -- the batched form's launcher: picks the instantiation
 * (orbg_batched_inst.cu, kernels in orbg_batched.cuh) by the longest code
 * and widest syndrome of the call, and the grid-size helper the persistent
 * kernels share.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_internal.h"

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

size_t orbg_batched_scratch_bytes(int64_t B)
{
    return sizeof(unsigned long long) * ((size_t)ORBG_BATCHED_COUNTERS + (size_t)(B > 0 ? B : 0));
}

int orbg_launch_batched(const OrbgBatchedArgs &args)
{
    OrbgBatchedArgs a = args;
    if (a.code_id != nullptr)
        a.code0 = nullptr; /* per-block codes: the generic kernels */
    if (a.code0) {
        /* every block is code 0: size everything for it alone */
        a.n_max = a.code0->n;
        a.w32_max = a.code0->w32;
        a.ntrip_max = a.code0->ntrip;
        a.x3w_max = a.code0->x3w;
    }
#define ORBG_BW(K)                                           \
    return a.w32_max <= 1   ? orbg_launch_batched_k##K##w1(a) \
           : a.w32_max <= 2 ? orbg_launch_batched_k##K##w2(a) \
                            : orbg_launch_batched_k##K##w4(a);
    if (a.n_max <= 32)
        ORBG_BW(1)
    if (a.n_max <= 64)
        ORBG_BW(2)
    if (a.n_max <= 128)
        ORBG_BW(4)
    ORBG_BW(8)
#undef ORBG_BW
}
