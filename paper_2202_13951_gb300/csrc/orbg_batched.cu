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

size_t orbg_batched_scratch_bytes(int64_t B, int ncodes)
{
    const size_t b = (size_t)(B > 0 ? B : 0);
    const size_t h = b < ORBG_HANDOVER_MAX ? b : ORBG_HANDOVER_MAX;
    return 8 * (size_t)ORBG_BATCHED_COUNTERS + 16 * ((size_t)(ncodes > 0 ? ncodes : 0) + 1) +
           12 * b + 15 + (size_t)ORBG_HANDOVER_BYTES * h;
}

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortChunk = 4096; /* blocks per CTA of the scatter */

/* the sort bucket of block b: its code's, ids outside the set last */
__device__ __forceinline__ int sort_bucket(const int32_t *code_id, const int32_t *bucket,
                                           int64_t b, int ncodes)
{
    const int c = code_id[b];
    return c >= 0 && c < ncodes ? bucket[c] : ncodes;
}

__global__ void __launch_bounds__(kSortThreads) orbg_code_count_kernel(
    const int32_t *__restrict__ code_id, const int32_t *__restrict__ bucket, int64_t B,
    int ncodes, uint32_t *__restrict__ count)
{
    extern __shared__ uint32_t h[];
    for (int i = threadIdx.x; i <= ncodes; i += blockDim.x)
        h[i] = 0;
    __syncthreads();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[sort_bucket(code_id, bucket, b, ncodes)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i <= ncodes; i += blockDim.x)
        if (h[i])
            atomicAdd(&count[i], h[i]);
}

/* Each CTA scatters one chunk of kSortChunk blocks: it counts its chunk per
 * code, reserves a range of each code's slots with one global atomic per
 * code, and writes its blocks there (in chunk order within a code). */
__global__ void __launch_bounds__(kSortThreads) orbg_code_scatter_kernel(
    const int32_t *__restrict__ code_id, const int32_t *__restrict__ bucket, int64_t B, int ncodes,
    const uint32_t *__restrict__ count, uint32_t *__restrict__ cursor,
    uint32_t *__restrict__ perm)
{
    extern __shared__ uint32_t sh[];
    uint32_t *base = sh;              /* [ncodes + 1] first slot of each code */
    uint32_t *local = sh + ncodes + 1; /* [ncodes + 1] this chunk's count, then its cursor */
    const int64_t lo = (int64_t)blockIdx.x * kSortChunk;
    const int64_t hi = lo + kSortChunk < B ? lo + kSortChunk : B;
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int i = 0; i <= ncodes; i++) {
            base[i] = acc;
            acc += count[i];
        }
    }
    for (int i = threadIdx.x; i <= ncodes; i += blockDim.x)
        local[i] = 0;
    __syncthreads();
    for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x)
        atomicAdd(&local[sort_bucket(code_id, bucket, b, ncodes)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i <= ncodes; i += blockDim.x)
        local[i] = local[i] ? base[i] + atomicAdd(&cursor[i], local[i]) : 0u;
    __syncthreads();
    for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x)
        perm[atomicAdd(&local[sort_bucket(code_id, bucket, b, ncodes)], 1u)] = (uint32_t)b;
}

/* one warp per heavy-list entry; the lanes copy the codeword bytes */
__global__ void __launch_bounds__(256) orbg_heavy_gather_kernel(
    const OrbgDeviceCode *__restrict__ codes, const int32_t *__restrict__ code_id, int n0,
    const int64_t *__restrict__ cw_off, const uint8_t *__restrict__ cw,
    const uint32_t *__restrict__ q, const uint8_t *__restrict__ ab,
    const unsigned long long *__restrict__ counters, const unsigned long long *__restrict__ heavy,
    unsigned char *__restrict__ out, uint32_t cap, int n_max, uint8_t *__restrict__ to_cw,
    uint32_t *__restrict__ to_q, uint8_t *__restrict__ to_ab)
{
    const unsigned long long nheavy = counters[1];
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *(unsigned long long *)out = nheavy;
    const int lane = threadIdx.x & 31;
    const uint64_t step = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    if (to_cw) {
        /* straight into the caller's buffers, at the blocks' own places */
        for (uint64_t h = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nheavy;
             h += step) {
            const uint32_t b = (uint32_t)heavy[h];
            const int n = code_id ? codes[code_id[b]].n : n0;
            const int64_t o = cw_off ? cw_off[b] : (int64_t)b * n0;
            for (int j = lane; j < n; j += 32)
                to_cw[o + j] = cw[o + j];
            if (lane == 0) {
                to_q[b] = q[b];
                to_ab[b] = ab[b];
            }
        }
        return;
    }
    const uint64_t m = nheavy < cap ? nheavy : cap;
    uint32_t *bq = (uint32_t *)(out + 16);
    uint8_t *flag = out + 16 + 8 * (size_t)cap;
    uint8_t *cwo = out + orbg_gather_cw_at(cap);
    for (uint64_t h = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < m; h += step) {
        const uint32_t b = (uint32_t)heavy[h]; /* low half: the block */
        const int n = code_id ? codes[code_id[b]].n : n0;
        const int64_t o = cw_off ? cw_off[b] : (int64_t)b * n0;
        for (int j = lane; j < n; j += 32)
            cwo[h * (uint64_t)n_max + j] = cw[o + j];
        if (lane == 0) {
            bq[2 * h] = b;
            bq[2 * h + 1] = q[b];
            flag[h] = ab[b];
        }
    }
}

}  // namespace

int orbg_launch_heavy_gather(const OrbgDeviceCode *d_codes, const int32_t *code_id, int n0,
                             const int64_t *cw_off, const uint8_t *cw, const uint32_t *q,
                             const uint8_t *ab, const OrbgScratch &s, unsigned char *out,
                             uint32_t cap, int n_max, uint8_t *to_cw, uint32_t *to_q,
                             uint8_t *to_ab, void *stream)
{
    int dev = 0, sms = 1;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return (int)e;
    orbg_heavy_gather_kernel<<<(unsigned)sms * 2, 256, 0, (cudaStream_t)stream>>>(
        d_codes, code_id, n0, cw_off, cw, q, ab, s.counters, s.heavy, out, cap, n_max, to_cw, to_q,
        to_ab);
    return (int)cudaGetLastError();
}

int orbg_launch_code_sort(const int32_t *code_id, const int32_t *bucket, int64_t B, int ncodes,
                          const OrbgScratch &s, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const size_t sh1 = sizeof(uint32_t) * (size_t)(ncodes + 1);
    int dev = 0, sms = 1;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return (int)e;
    int64_t g1 = (B + kSortThreads - 1) / kSortThreads;
    if (g1 > (int64_t)sms * 8)
        g1 = (int64_t)sms * 8;
    orbg_code_count_kernel<<<(unsigned)g1, kSortThreads, sh1, st>>>(code_id, bucket, B, ncodes,
                                                                    s.count);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return (int)e;
    const int64_t g2 = (B + kSortChunk - 1) / kSortChunk;
    orbg_code_scatter_kernel<<<(unsigned)g2, kSortThreads, 2 * sh1, st>>>(
        code_id, bucket, B, ncodes, s.count, s.cursor, s.perm);
    return (int)cudaGetLastError();
}

int orbg_launch_exact(int K, int W, const OrbgBatchedArgs &a, const OrbgScratch &s,
                      unsigned long long *queue, int blo, int bhi, int pdl, int stride)
{
#define ORBG_EX(KK)                                                                         \
    return W <= 1   ? orbg_launch_exact_k##KK##w1(a, s, queue, blo, bhi, pdl, stride)       \
           : W == 2 ? orbg_launch_exact_k##KK##w2(a, s, queue, blo, bhi, pdl, stride)       \
                    : orbg_launch_exact_k##KK##w4(a, s, queue, blo, bhi, pdl, stride);
    if (K <= 1)
        ORBG_EX(1)
    if (K == 2)
        ORBG_EX(2)
    if (K == 4)
        ORBG_EX(4)
    ORBG_EX(8)
#undef ORBG_EX
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
