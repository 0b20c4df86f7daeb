/*
 * orbg_probe.cu -- roofline probes.  The integer pipe: how many lanes of
 * independent lop3.b32 (3-input XOR) an SM retires per clock (eight
 * independent dependency chains per thread).  Shared memory: how many
 * bytes an SM's 64-bit shared loads deliver per clock (lanes read
 * consecutive words, no bank conflicts).  1024 threads per CTA, one CTA
 * per SM; cycles from clock64 on each SM.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "orbg_internal.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeIters = 4096;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) orbg_lop3_probe_kernel(uint32_t *sink,
                                                                        long long *cycles,
                                                                        uint32_t seed)
{
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++)
        a[c] = seed * (threadIdx.x + 1) + c;
    const uint32_t b = seed ^ blockIdx.x, d = seed + 0x9E3779B9u;
    __syncthreads();
    long long t0 = clock64();
    for (int i = 0; i < kProbeIters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++)
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d));
    }
    __syncthreads();
    long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++)
        x ^= a[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = x;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

constexpr int kSmemWords = 4096; /* 32 KiB of 8-byte words */
constexpr int kSmemIters = 1024;
constexpr int kSmemUnroll = 8;

__global__ void __launch_bounds__(kProbeThreads) orbg_lds_probe_kernel(uint32_t *sink,
                                                                       long long *cycles,
                                                                       uint32_t seed)
{
    __shared__ uint2 buf[kSmemWords];
    for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x)
        buf[i] = make_uint2(seed * (uint32_t)i, seed ^ (uint32_t)i);
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    uint32_t x = 0, y = 0;
    long long t0 = clock64();
    for (int it = 0; it < kSmemIters; it++) {
#pragma unroll
        for (int u = 0; u < kSmemUnroll; u++) {
            /* word (thread + 512 u + 32 it) mod 4096: a warp reads 32
             * consecutive words, the eight loads of a step distinct words,
             * every step other ones; volatile loads, so none is merged */
            const uint32_t w = (threadIdx.x + 512u * (uint32_t)u + 32u * (uint32_t)it) &
                               (uint32_t)(kSmemWords - 1);
            uint32_t lo, hi;
            asm volatile("ld.volatile.shared.v2.u32 {%0, %1}, [%2];"
                         : "=r"(lo), "=r"(hi)
                         : "r"(base + 8u * w));
            x ^= lo;
            y ^= hi;
        }
    }
    __syncthreads();
    long long t1 = clock64();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = x ^ y;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

/* Runs `kern` on one CTA per SM twice (the first warms up); median cycles. */
template <class K>
int run_probe(K kern, double *median_cycles)
{
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return (int)e;
    uint32_t *sink = nullptr;
    long long *cyc = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(uint32_t) * (size_t)sms * kProbeThreads)) != cudaSuccess)
        return (int)e;
    if ((e = cudaMalloc(&cyc, sizeof(long long) * (size_t)sms)) != cudaSuccess) {
        cudaFree(sink);
        return (int)e;
    }
    std::vector<long long> h((size_t)sms);
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
        kern<<<sms, kProbeThreads>>>(sink, cyc, 12345u + rep);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpy(h.data(), cyc, sizeof(long long) * (size_t)sms, cudaMemcpyDeviceToHost);
    }
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess)
        return (int)e;
    std::sort(h.begin(), h.end());
    *median_cycles = (double)h[h.size() / 2];
    return 0;
}

}  // namespace

int orbg_launch_smem_probe(double *bytes_per_clk_per_sm)
{
    double cyc = 0;
    int rc = run_probe(orbg_lds_probe_kernel, &cyc);
    if (rc != 0)
        return rc;
    *bytes_per_clk_per_sm = (double)kProbeThreads * kSmemIters * kSmemUnroll * 8.0 / cyc;
    return 0;
}

int orbg_launch_int_probe(double *lanes_per_clk_per_sm)
{
    double cyc = 0;
    int rc = run_probe(orbg_lop3_probe_kernel, &cyc);
    if (rc != 0)
        return rc;
    *lanes_per_clk_per_sm = (double)kProbeThreads * kProbeIters * kChains / cyc;
    return 0;
}
