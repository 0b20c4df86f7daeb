/*
 * orbg_decode_block.cuh -- per-block device code of the basic-ORBGRAND
 * decoder, shared by the plain and the batched kernels.
 *
 * One warp decodes one received block (Algorithm 1 with the basic ORBGRAND
 * generator, Sec. III-B):
 *   1. coalesced load of the n FP32 LLRs; hard decision y_i = [L_i > 0];
 *      reliability key (FP32 bits of |L_i|, i) (Sec. III-A);
 *   2. warp bitonic sort of the keys in registers -> pi (Sec. III-A; the
 *      paper names bitonic sorting networks as one option, Sec. IV-B);
 *   3. permuted columns hperm[p] = H[:, pi_p] into shared memory, plus a
 *      zero column at p = n; starting syndrome s0 = H y (Sec. I);
 *   4. the query order as runs (orbg_internal.h): lane l of a warp step
 *      takes run l of a group of 32, XORs its prefix columns into s0 and
 *      walks the run, testing s0 (+) prefix (+) hperm[a] (+) hperm[b] == 0;
 *      the warp keeps the smallest hit index (__reduce_min_sync) and stops
 *      once no later group can hold a smaller one, or the cap is passed;
 *   5. codeword y (+) z* (or y if abandoned), query count, abandon flag.
 * Every loop is bounded by the table size or the run length; no kernel
 * waits on another thread's progress.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_internal.h"

#define FULL_MASK 0xFFFFFFFFu

namespace orbg_dev {

/* ---------------------------------------------------------------- vectors */

template <int W> struct Syn;
template <> struct Syn<1> { typedef uint32_t T; };
template <> struct Syn<2> { typedef uint2 T; };
template <> struct Syn<4> { typedef uint4 T; };

__device__ __forceinline__ uint32_t sx(uint32_t a, uint32_t b) { return a ^ b; }
__device__ __forceinline__ uint2 sx(uint2 a, uint2 b) { return make_uint2(a.x ^ b.x, a.y ^ b.y); }
__device__ __forceinline__ uint4 sx(uint4 a, uint4 b)
{
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}
__device__ __forceinline__ bool sz(uint32_t a) { return a == 0u; }
__device__ __forceinline__ bool sz(uint2 a) { return (a.x | a.y) == 0u; }
__device__ __forceinline__ bool sz(uint4 a) { return (a.x | a.y | a.z | a.w) == 0u; }
template <typename T> __device__ __forceinline__ T szero();
template <> __device__ __forceinline__ uint32_t szero<uint32_t>() { return 0u; }
template <> __device__ __forceinline__ uint2 szero<uint2>() { return make_uint2(0u, 0u); }
template <> __device__ __forceinline__ uint4 szero<uint4>() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ uint32_t shfl_xor_all(uint32_t v, int m) { return __shfl_xor_sync(FULL_MASK, v, m); }
__device__ __forceinline__ uint2 shfl_xor_all(uint2 v, int m)
{
    return make_uint2(__shfl_xor_sync(FULL_MASK, v.x, m), __shfl_xor_sync(FULL_MASK, v.y, m));
}
__device__ __forceinline__ uint4 shfl_xor_all(uint4 v, int m)
{
    return make_uint4(__shfl_xor_sync(FULL_MASK, v.x, m), __shfl_xor_sync(FULL_MASK, v.y, m),
                      __shfl_xor_sync(FULL_MASK, v.z, m), __shfl_xor_sync(FULL_MASK, v.w, m));
}

template <int W>
__device__ __forceinline__ typename Syn<W>::T load_col(const uint32_t *__restrict__ hcol, int j)
{
    typedef typename Syn<W>::T T;
    return __ldg(reinterpret_cast<const T *>(hcol) + j);
}

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m)
{
    uint32_t lo = __shfl_xor_sync(FULL_MASK, (uint32_t)v, m);
    uint32_t hi = __shfl_xor_sync(FULL_MASK, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

/* Shared memory of one warp: hperm[n+1] syndromes, then pi[256], cw[256]. */
__host__ __device__ __forceinline__ uint32_t warp_smem_bytes(int n, int w32)
{
    uint32_t h = (uint32_t)(n + 1) * 4u * (uint32_t)w32;
    h = (h + 15u) & ~15u;
    return h + 256u + 256u;
}

/* ------------------------------------------------------------ one block */

template <int K, int W>
__device__ void decode_block(const OrbgDeviceCode &code, const float *__restrict__ llr,
                             uint8_t *__restrict__ cw_out, uint32_t *__restrict__ q_out,
                             uint8_t *__restrict__ ab_out, uint32_t cap,
                             unsigned char *__restrict__ wsm, int lane)
{
    typedef typename Syn<W>::T T;
    const int n = code.n;
    T *h = reinterpret_cast<T *>(wsm);
    uint8_t *pi = wsm + (((uint32_t)(n + 1) * sizeof(T) + 15u) & ~15u);
    uint8_t *cw = pi + 256;

    /* 1. load, hard decision, keys, s0 */
    uint64_t key[K];
    T s0 = szero<T>();
    bool nan = false;
#pragma unroll
    for (int k = 0; k < K; k++) {
        int i = k * 32 + lane;
        if (i < n) {
            float L = __ldg(llr + i);
            nan |= (L != L);
            uint32_t bits = __float_as_uint(L) & 0x7FFFFFFFu;
            key[k] = ((uint64_t)bits << 32) | (uint32_t)i;
            uint8_t y = L > 0.0f ? 1 : 0;
            cw[i] = y;
            if (y)
                s0 = sx(s0, load_col<W>(code.hcol, i));
        } else {
            key[k] = 0xFFFFFFFF00000000ull | (uint32_t)i; /* padding sorts last */
        }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1)
        s0 = sx(s0, shfl_xor_all(s0, m));
    if (__any_sync(FULL_MASK, nan)) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < K; k++) {
            int i = k * 32 + lane;
            if (i < n)
                cw_out[i] = cw[i];
        }
        if (lane == 0) {
            *q_out = 0u;
            *ab_out = 2;
        }
        return;
    }

    /* 2. bitonic sort; position e = lane*K + k after the sort */
#pragma unroll
    for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= K) {
                const int lm = stride / K;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const int e = lane * K + k;
                    uint64_t o = shfl_xor_u64(key[k], lm);
                    bool asc = (e & size) == 0;
                    bool lower = (e & stride) == 0;
                    uint64_t mn = key[k] < o ? key[k] : o;
                    uint64_t mx = key[k] < o ? o : key[k];
                    key[k] = (lower == asc) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    if ((k & stride) == 0) {
                        const int k2 = k | stride;
                        const int e = lane * K + k;
                        bool asc = (e & size) == 0;
                        uint64_t a = key[k], b = key[k2];
                        bool sw = asc ? (a > b) : (a < b);
                        key[k] = sw ? b : a;
                        key[k2] = sw ? a : b;
                    }
                }
            }
        }
    }

    /* 3. pi and permuted columns; zero column at n */
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int e = lane * K + k;
        if (e < n) {
            int idx = (int)(uint32_t)key[k];
            pi[e] = (uint8_t)idx;
            h[e] = load_col<W>(code.hcol, idx);
        }
    }
    if (lane == 0)
        h[n] = szero<T>();
    __syncwarp();

    /* 4. runs in groups of 32 */
    const uint32_t limit = cap;          /* hits above the cap do not count */
    uint32_t best = 0xFFFFFFFFu;
    uint32_t my_t = 0xFFFFFFFFu;         /* hit this lane found and kept */
    uint32_t my_run = 0, my_j = 0;
    const uint4 *runs4 = reinterpret_cast<const uint4 *>(code.runs);
    for (uint32_t g = 0; g < code.ngroups; g++) {
        uint32_t floor = __ldg(code.group_floor + g);
        if (floor >= best || floor > limit)
            break;
        uint32_t e = g * ORBG_GROUP + (uint32_t)lane;
        uint32_t mine = 0xFFFFFFFFu, mj = 0;
        if (e < code.nruns) {
            uint4 v0 = __ldg(runs4 + 2 * e);
            uint4 v1 = __ldg(runs4 + 2 * e + 1);
            const uint32_t tstart = v0.x;
            const int pair_sum = (int)(v0.y & 0xFFFFu);
            int a = (int)(v0.y >> 16);
            const int len = (int)(v0.z & 0xFFu);
            const int npre = (int)((v0.z >> 8) & 0xFFu);
            if (tstart < best && tstart <= limit) {
                T P = s0;
#pragma unroll
                for (int i = 0; i < ORBG_RUN_MAX_PRE; i++) {
                    if (i >= npre)
                        break;
                    uint32_t wd = (i < 4) ? v0.w : (i < 8) ? v1.x : (i < 12) ? v1.y
                                : (i < 16) ? v1.z : v1.w;
                    P = sx(P, h[(wd >> (8 * (i & 3))) & 0xFFu]);
                }
                int b = pair_sum - a;
                for (int j = 0; j < len; j++, a++, b--) {
                    T s = sx(sx(P, h[a]), h[b]);
                    if (sz(s)) {
                        mine = tstart + (uint32_t)j;
                        mj = (uint32_t)j;
                        break;
                    }
                }
            }
        }
        uint32_t gbest = __reduce_min_sync(FULL_MASK, mine);
        if (gbest < best) {
            best = gbest;
            if (mine == gbest) {
                my_t = mine;
                my_run = e;
                my_j = mj;
            }
        }
    }

    /* 5. output */
    const bool hit = best <= limit;
    if (hit && my_t == best) {
        /* the lane that owns the winning run applies the flips */
        const OrbgRun *rp = code.runs + my_run;
        int npre = rp->npre;
        for (int i = 0; i < npre; i++)
            cw[pi[rp->pre[i]]] ^= 1;
        int a = (int)rp->a0 + (int)my_j;
        if (a < n) {
            int b = (int)rp->pair_sum - a;
            cw[pi[a]] ^= 1;
            cw[pi[b]] ^= 1;
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < K; k++) {
        int i = k * 32 + lane;
        if (i < n)
            cw_out[i] = cw[i];
    }
    if (lane == 0) {
        *q_out = hit ? best : cap;
        *ab_out = hit ? 0 : 1;
    }
    __syncwarp();
}

/* Runtime dispatch on (n, syndrome width), warp-uniform; only variants up to
 * (KMAX keys per lane, WMAX syndrome words) are instantiated. */
template <int K, int WMAX>
__device__ __forceinline__ void decode_w(const OrbgDeviceCode &code, const float *llr, uint8_t *cw,
                                         uint32_t *q, uint8_t *ab, uint32_t cap,
                                         unsigned char *wsm, int lane)
{
    const int w = code.w32;
    if constexpr (WMAX >= 4) {
        if (w > 2) {
            decode_block<K, 4>(code, llr, cw, q, ab, cap, wsm, lane);
            return;
        }
    }
    if constexpr (WMAX >= 2) {
        if (w == 2) {
            decode_block<K, 2>(code, llr, cw, q, ab, cap, wsm, lane);
            return;
        }
    }
    decode_block<K, 1>(code, llr, cw, q, ab, cap, wsm, lane);
}

template <int KMAX, int WMAX>
__device__ __forceinline__ void decode_any(const OrbgDeviceCode &code, const float *llr,
                                           uint8_t *cw, uint32_t *q, uint8_t *ab, uint32_t cap,
                                           unsigned char *wsm, int lane)
{
    const int n = code.n;
    if constexpr (KMAX >= 8) {
        if (n > 128) {
            decode_w<8, WMAX>(code, llr, cw, q, ab, cap, wsm, lane);
            return;
        }
    }
    if constexpr (KMAX >= 4) {
        if (n > 64) {
            decode_w<4, WMAX>(code, llr, cw, q, ab, cap, wsm, lane);
            return;
        }
    }
    if constexpr (KMAX >= 2) {
        if (n > 32) {
            decode_w<2, WMAX>(code, llr, cw, q, ab, cap, wsm, lane);
            return;
        }
    }
    decode_w<1, WMAX>(code, llr, cw, q, ab, cap, wsm, lane);
}

}  // namespace orbg_dev
