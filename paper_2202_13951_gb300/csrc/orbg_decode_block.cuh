/*
 * orbg_decode_block.cuh -- per-block device code of the basic-ORBGRAND
 * decoder, shared by the plain and the batched kernels.
 *
 * Decoding one received block (Algorithm 1 with the basic ORBGRAND
 * generator, Sec. III-B):
 *   1. coalesced load of the n FP32 LLRs; hard decision y_i = [L_i > 0];
 *      reliability key (FP32 bits of |L_i|, i) (Sec. III-A); starting
 *      syndrome s0 = H y (Sec. I).  If s0 = 0, y is a codeword and query 1
 *      (the zero pattern) decodes: no sort is needed;
 *   2. the reliability order pi (Sec. III-A): for blocks decided inside the
 *      flat table only its leading ranks, extracted as warp minima; else a
 *      warp bitonic sort of the keys in registers (the paper names bitonic
 *      sorting networks as one option, Sec. IV-B);
 *   3. permuted columns hperm[p] = H[:, pi_p] into shared memory, after a
 *      zero column read by unused prefix slots;
 *   4. the query order as runs (orbg_internal.h): lane l of a warp step
 *      takes run l of a group of 32, XORs its prefix columns into s0 and
 *      walks the run, testing s0 (+) prefix (+) hperm[a] (+) hperm[b] == 0;
 *      the smallest hit index is kept and the search stops once no later
 *      group can hold a smaller one, or the cap is passed;
 *   5. codeword y (+) z* (or y if abandoned), query count, abandon flag.
 *
 * Two ways to run step 4: one warp walks all groups of its block
 * (decode_block_warp), or all warps of a CTA share one block and take its
 * groups in turn, with the best index in shared memory (decode_block_cta).
 * The second keeps a block that needs 1e6 queries from running on a single
 * warp.  Every loop is bounded by the table size or the run length; no
 * thread waits on another's progress beyond __syncthreads.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_internal.h"

#define FULL_MASK 0xFFFFFFFFu
#define ORBG_NONE 0xFFFFFFFFu

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

/* Shared memory of one block in flight: hperm[n+1] full syndromes, then
 * (for W > 1) h0[n+1], the first 32-bit word of each, then pi[256] and the
 * staged codeword cw[256].  Entry 0 of hperm and h0 is a zero column
 * (BlockSmem). */
__host__ __device__ __forceinline__ uint32_t block_smem_bytes(int n, int w32)
{
    uint32_t h = (uint32_t)(n + 1) * 4u * (uint32_t)w32;
    h = (h + 15u) & ~15u;
    uint32_t h0 = w32 > 1 ? (((uint32_t)(n + 1) * 4u + 15u) & ~15u) : 0u;
    return h + h0 + 256u + 256u;
}

/* Triple table: X3[i] = low 16 bits of h0[c0] ^ h0[a0] ^ h0[b0] for triple
 * i of the code's triple list (a match is verified on the whole syndrome
 * unless n - k <= 16, where 16 bits are the whole syndrome). */
__host__ __device__ __forceinline__ uint32_t triple_table_bytes(uint32_t ntrip)
{
    return (ntrip * 2u + 15u) & ~15u;
}

/* Fills X3[lo, hi) from the triple list; `stride` threads starting at `t`. */
__device__ __forceinline__ void build_x3(const OrbgDeviceCode &code, const uint32_t *h0,
                                         uint16_t *X3, uint32_t lo, uint32_t hi, uint32_t t,
                                         uint32_t stride)
{
    for (uint32_t i = lo + t; i < hi; i += stride) {
        const uint32_t c = __ldg(code.trip + i);
        X3[i] = (uint16_t)(h0[c & 0xFFu] ^ h0[(c >> 8) & 0xFFu] ^ h0[(c >> 16) & 0xFFu]);
    }
}

/* h[r] (and h0[r]) is the column of sorted position r, 0 <= r < n; the
 * entry before it, h[-1], is the zero column, so a 1-based position p (0 =
 * none) reads h[p - 1] with no test. */
template <int W> struct BlockSmem {
    typedef typename Syn<W>::T T;
    T *h;
    uint32_t *h0;
    uint8_t *pi;
    uint8_t *cw;
    __device__ __forceinline__ BlockSmem(unsigned char *base, int n)
    {
        h = reinterpret_cast<T *>(base) + 1;
        unsigned char *p = base + (((uint32_t)(n + 1) * sizeof(T) + 15u) & ~15u);
        if (W > 1) {
            h0 = reinterpret_cast<uint32_t *>(p) + 1;
            p += ((uint32_t)(n + 1) * 4u + 15u) & ~15u;
        } else {
            h0 = reinterpret_cast<uint32_t *>(base) + 1;
        }
        pi = p;
        cw = pi + 256;
    }
};

__device__ __forceinline__ uint32_t first_word(uint32_t v) { return v; }
__device__ __forceinline__ uint32_t first_word(uint2 v) { return v.x; }
__device__ __forceinline__ uint32_t first_word(uint4 v) { return v.x; }

/* LLR reads: from shared memory (LS, staged ahead by the batched kernel)
 * or from global memory through the read-only path. */
template <bool LS>
__device__ __forceinline__ float llr_at(const float *__restrict__ llr, int i)
{
    if (LS)
        return llr[i];
    return __ldg(llr + i);
}

/* Sort keys are 32 bits: (|L| bits with the low DROP bits dropped) << IB | i,
 * with IB index bits (32 K <= 2^IB).  The truncation merges reliabilities
 * that differ only in the dropped bits; inside such a tie the key orders by
 * index, which is the exact order unless the full bits disagree -- checked
 * after the sort (sort_block). */
template <int K> struct KeyBits {
    static constexpr int IB = K == 1 ? 5 : K == 2 ? 6 : K == 4 ? 7 : 8; /* 32*K <= 2^IB */
    static constexpr int DROP = IB - 1;                                  /* 31 + IB - DROP = 32 */
    static constexpr uint32_t IMASK = (1u << IB) - 1u;
};

/* ------------------------------------------------------- step 1: load */

/* Loads the block, writes y into cw, builds the K 32-bit sort keys per lane
 * and returns s0 (identical in every lane).  *nan is warp-uniform. */
template <int K, int W, bool LS = false>
__device__ __forceinline__ typename Syn<W>::T load_block(const OrbgDeviceCode &code,
                                                         const float *__restrict__ llr,
                                                         uint32_t (&key)[K], uint8_t *cw,
                                                         int lane, bool *nan_out)
{
    typedef typename Syn<W>::T T;
    typedef KeyBits<K> KB;
    const int n = code.n;
    T s0 = szero<T>();
    bool nan = false;
#pragma unroll
    for (int k = 0; k < K; k++) {
        int i = k * 32 + lane;
        uint32_t bits = 0xFFFFFFFFu; /* padding sorts last */
        if (i < n) {
            float L = llr_at<LS>(llr, i);
            nan |= (L != L);
            bits = __float_as_uint(L) & 0x7FFFFFFFu;
            uint8_t y = L > 0.0f ? 1 : 0;
            cw[i] = y;
            if (y)
                s0 = sx(s0, load_col<W>(code.hcol, i));
        }
        key[k] = ((bits >> KB::DROP) << KB::IB) | ((uint32_t)i & KB::IMASK);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1)
        s0 = sx(s0, shfl_xor_all(s0, m));
    *nan_out = __any_sync(FULL_MASK, nan);
    return s0;
}

/* ------------------------------------------------------- step 2: sort */

/* Bitonic sort of 32*K unique keys held K per lane; afterwards position
 * e = lane*K + k holds the e-th smallest.  The network's merge levels and
 * its strides across lanes are loops (the compare-exchanges of one step,
 * over the lane's K keys, are unrolled): the code stays small enough to
 * remain in the instruction cache while the warps of an SM sort block after
 * block, where the fully unrolled network (about 1,300 instructions for
 * K = 8) was fetched anew for every block. */
template <int K>
__device__ __forceinline__ void sort_keys(uint64_t (&key)[K], int lane)
{
#pragma unroll 1
    for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll 1
        for (int stride = size >> 1; stride >= K; stride >>= 1) {
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
        }
#pragma unroll
        for (int stride = K / 2; stride > 0; stride >>= 1) {
            if (stride > (size >> 1))
                continue;
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

/* Bitonic sort of 32*K unique 32-bit keys held K per lane (loops as
 * sort_keys). */
template <int K>
__device__ __forceinline__ void bitonic32(uint32_t (&key)[K], int lane)
{
#pragma unroll 1
    for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll 1
        for (int stride = size >> 1; stride >= K; stride >>= 1) {
            const int lm = stride / K;
#pragma unroll
            for (int k = 0; k < K; k++) {
                const int e = lane * K + k;
                const uint32_t o = __shfl_xor_sync(FULL_MASK, key[k], lm);
                const bool takemin = ((e & size) == 0) == ((e & stride) == 0);
                key[k] = takemin ? min(key[k], o) : max(key[k], o);
            }
        }
#pragma unroll
        for (int stride = K / 2; stride > 0; stride >>= 1) {
            if (stride > (size >> 1))
                continue;
#pragma unroll
            for (int k = 0; k < K; k++) {
                if ((k & stride) == 0) {
                    const int k2 = k | stride;
                    const int e = lane * K + k;
                    const bool asc = (e & size) == 0;
                    const uint32_t lo = min(key[k], key[k2]), hi = max(key[k], key[k2]);
                    key[k] = asc ? lo : hi;
                    key[k2] = asc ? hi : lo;
                }
            }
        }
    }
}

/* The same networks fully unrolled (sort_keys, bitonic32): faster where
 * one kernel sorts for a single code, whose code then stays cached. */
template <int K>
__device__ __forceinline__ void sort_keys_unrolled(uint64_t (&key)[K], int lane)
{
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
}

/* Bitonic sort of 32*K unique 32-bit keys held K per lane. */
template <int K>
__device__ __forceinline__ void bitonic32_unrolled(uint32_t (&key)[K], int lane)
{
#pragma unroll
    for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= K) {
                const int lm = stride / K;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const int e = lane * K + k;
                    const uint32_t o = __shfl_xor_sync(FULL_MASK, key[k], lm);
                    const bool takemin = ((e & size) == 0) == ((e & stride) == 0);
                    key[k] = takemin ? min(key[k], o) : max(key[k], o);
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    if ((k & stride) == 0) {
                        const int k2 = k | stride;
                        const int e = lane * K + k;
                        const bool asc = (e & size) == 0;
                        const uint32_t lo = min(key[k], key[k2]), hi = max(key[k], key[k2]);
                        key[k] = asc ? lo : hi;
                        key[k2] = asc ? hi : lo;
                    }
                }
            }
        }
    }
}

/*
 * Sort the 32-bit keys, then check every adjacent pair whose truncated
 * reliabilities are equal against the full bits; if any is out of order,
 * sort exact 64-bit keys (bits << 32 | i) rebuilt from the LLRs instead.
 * Afterwards key[k] holds the received index of sorted position lane*K + k.
 */
template <int K, bool LS = false, bool ROLL = true>
__device__ __forceinline__ void sort_block(uint32_t (&key)[K], const float *__restrict__ llr,
                                           int n, int lane)
{
    typedef KeyBits<K> KB;
    if (ROLL)
        bitonic32<K>(key, lane);
    else
        bitonic32_unrolled<K>(key, lane);
    bool bad = false;
    const uint32_t next_first = __shfl_down_sync(FULL_MASK, key[0], 1);
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int e = lane * K + k;
        const uint32_t nxt = (k + 1 < K) ? key[k + 1 < K ? k + 1 : k] : next_first;
        if (e + 1 < n && (key[k] >> KB::IB) == (nxt >> KB::IB)) {
            const uint32_t ba =
                __float_as_uint(llr_at<LS>(llr, (int)(key[k] & KB::IMASK))) & 0x7FFFFFFFu;
            const uint32_t bb =
                __float_as_uint(llr_at<LS>(llr, (int)(nxt & KB::IMASK))) & 0x7FFFFFFFu;
            bad |= ba > bb;
        }
    }
    if (__any_sync(FULL_MASK, bad)) {
        uint64_t k64[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int i = k * 32 + lane;
            const uint32_t bits =
                i < n ? (__float_as_uint(llr_at<LS>(llr, i)) & 0x7FFFFFFFu) : 0xFFFFFFFFu;
            k64[k] = ((uint64_t)bits << 32) | (uint32_t)i;
        }
        if (ROLL)
            sort_keys<K>(k64, lane);
        else
            sort_keys_unrolled<K>(k64, lane);
#pragma unroll
        for (int k = 0; k < K; k++)
            key[k] = (uint32_t)k64[k];
        return;
    }
#pragma unroll
    for (int k = 0; k < K; k++)
        key[k] &= KB::IMASK;
}

/* ------------------------------------------------- step 3: permutation */

template <int K, int W>
__device__ __forceinline__ void build_perm(const OrbgDeviceCode &code, const uint32_t (&key)[K],
                                           const BlockSmem<W> &sm, int lane)
{
    const int n = code.n;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int e = lane * K + k;
        if (e < n) {
            const int idx = (int)key[k];
            sm.pi[e] = (uint8_t)idx;
            const typename Syn<W>::T col = load_col<W>(code.hcol, idx);
            sm.h[e] = col;
            if (W > 1)
                sm.h0[e] = first_word(col);
        }
    }
    if (lane == 0) {
        sm.h[-1] = szero<typename Syn<W>::T>();
        if (W > 1)
            sm.h0[-1] = 0u;
    }
}

/* ------------------------------------- step 2': the leading ranks only */

/*
 * Most blocks finish inside the flat table, whose patterns flip only the
 * ORBG_FLAT_RANKS least reliable positions.  For those the full sort is
 * replaced by extracting the smallest keys one at a time (a warp minimum
 * per rank) until the ranks a flat step needs are known; the full sort runs
 * only when the walk leaves the flat table.  Each lane first sorts its own
 * K keys, so its smallest is key[0].
 */
template <int K>
__device__ __forceinline__ void sort_lane(uint32_t (&key)[K])
{
#pragma unroll
    for (int i = 0; i < K; i++)
#pragma unroll
        for (int j = 0; j + 1 < K - i; j++) {
            const uint32_t lo = min(key[j], key[j + 1]), hi = max(key[j], key[j + 1]);
            key[j] = lo;
            key[j + 1] = hi;
        }
}

/* Extracts ranks have .. upto-1 (upto <= 32): lane r keeps rank r's key in
 * *mine.  Returns true if two consecutive ranks (this call's or the last
 * earlier one, in *prev) have equal truncated reliabilities: then the
 * truncated order may differ from the exact one and the caller sorts
 * exactly instead. */
template <int K>
__device__ __forceinline__ bool extract_ranks(uint32_t (&key)[K], int have, int upto,
                                              uint32_t *prev, uint32_t *mine, int lane)
{
    typedef KeyBits<K> KB;
    bool tie = false;
    uint32_t pv = *prev, mn = *mine;
    for (int r = have; r < upto; r++) {
        const uint32_t g = __reduce_min_sync(FULL_MASK, key[0]);
        tie |= (g >> KB::IB) == (pv >> KB::IB);
        if (key[0] == g) {
#pragma unroll
            for (int k = 0; k + 1 < K; k++)
                key[k] = key[k + 1];
            key[K - 1] = 0xFFFFFFFFu;
        }
        if (lane == r)
            mn = g;
        pv = g;
    }
    *prev = pv;
    *mine = mn;
    return tie;
}

/* Permuted columns of ranks lo .. hi-1 from the lanes holding them. */
template <int K, int W>
__device__ __forceinline__ void perm_ranks(const OrbgDeviceCode &code, uint32_t mine, int lo,
                                           int hi, const BlockSmem<W> &sm, int lane)
{
    if (lane >= lo && lane < hi) {
        const int idx = (int)(mine & KeyBits<K>::IMASK);
        sm.pi[lane] = (uint8_t)idx;
        const typename Syn<W>::T col = load_col<W>(code.hcol, idx);
        sm.h[lane] = col;
        if (W > 1)
            sm.h0[lane] = first_word(col);
    }
}

/* The K truncated keys of a lane, in load order (as load_block makes them). */
template <int K, bool LS>
__device__ __forceinline__ void make_keys(const float *__restrict__ llr, int n, int lane,
                                          uint32_t (&key)[K])
{
    typedef KeyBits<K> KB;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int i = k * 32 + lane;
        const uint32_t bits =
            i < n ? (__float_as_uint(llr_at<LS>(llr, i)) & 0x7FFFFFFFu) : 0xFFFFFFFFu;
        key[k] = ((bits >> KB::DROP) << KB::IB) | ((uint32_t)i & KB::IMASK);
    }
}

/* -------------------------------------------------- step 4: one run */

/* A run record (orbg_internal.h) as two 16-byte loads:
 * v0.x tstart, v0.y count | npre << 16 | kind << 24, v0.z aux,
 * v0.w prefix positions 0..3, v1 prefix positions 4..19. */
__device__ __forceinline__ int run_count(const uint4 &v0) { return (int)(v0.y & 0xFFFFu); }
__device__ __forceinline__ int run_npre(const uint4 &v0) { return (int)((v0.y >> 16) & 0xFFu); }
__device__ __forceinline__ int run_kind(const uint4 &v0) { return (int)(v0.y >> 24); }

/* Syndrome of a run's prefix: s0 (+) the prefix columns, over the W-word
 * syndromes h or over their first words h0.  Prefix positions are stored
 * 1-based with 0 in the unused slots, which read the zero column h[-1]:
 * the first eight loads need no test of npre. */
template <typename T>
__device__ __forceinline__ T prefix_syndrome(const uint4 &v0, const uint4 &v1,
                                             const T *__restrict__ h, const T s0, int npre)
{
    T p[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint32_t wd = i < 4 ? v0.w : v1.x;
        p[i] = h[(int)((wd >> (8 * (i & 3))) & 0xFFu) - 1];
    }
    T P = sx(sx(sx(s0, p[0]), sx(p[1], p[2])), sx(sx(p[3], p[4]), sx(p[5], sx(p[6], p[7]))));
    if (npre > 8) {
#pragma unroll
        for (int i = 8; i < ORBG_RUN_MAX_PRE; i++) {
            if (i >= npre)
                break;
            const uint32_t wd = (i < 12) ? v1.y : (i < 16) ? v1.z : v1.w;
            P = sx(P, h[(int)((wd >> (8 * (i & 3))) & 0xFFu) - 1]);
        }
    }
    return P;
}

/* Positions (0-based) a query flips besides the prefix: kind 1 hit value
 * is a (1-based), the pair (a, S - a); kind 2 hit value is the pattern's
 * offset j in the run, the pair (a_0 + j da, b_0 - j db); kind 3 hit value
 * is the triple index.  Writes up to three positions, returns how many. */
template <bool STRIDE = true>
__device__ __forceinline__ int query_tail(const uint4 &v0, uint32_t hit, const uint32_t *trip,
                                          int *pos)
{
    const int kind = run_kind(v0);
    if (kind == ORBG_RUN_PAIRS) {
        const int S = (int)(v0.z & 0xFFu), a = (int)hit;
        pos[0] = a - 1;
        pos[1] = S - a - 1;
        return 2;
    }
    if (STRIDE && kind == ORBG_RUN_STRIDE) {
        const int j = (int)hit;
        pos[0] = (int)(v0.z & 0xFFu) + j * (int)((v0.z >> 16) & 0xFFu) - 1;
        pos[1] = (int)((v0.z >> 8) & 0xFFu) - j * (int)(v0.z >> 24) - 1;
        return 2;
    }
    if (kind == ORBG_RUN_TRIPLES) {
        const uint32_t t = __ldg(trip + hit);
        pos[0] = (int)(t & 0xFFu);
        pos[1] = (int)((t >> 8) & 0xFFu);
        pos[2] = (int)((t >> 16) & 0xFFu);
        return 3;
    }
    return 0;
}

/* Full-width check of a query whose first word matched (rare: kept out of
 * line so it costs the scan loops no registers). */
template <int W>
__device__ __noinline__ bool verify_query(const uint4 &v0, const uint4 &v1,
                                          const typename Syn<W>::T *__restrict__ h,
                                          const typename Syn<W>::T s0, int n, uint32_t hit,
                                          const uint32_t *trip)
{
    typedef typename Syn<W>::T T;
    T P = prefix_syndrome<T>(v0, v1, h, s0, run_npre(v0));
    int pos[3];
    const int k = query_tail(v0, hit, trip, pos);
    for (int i = 0; i < k; i++)
        P = sx(P, h[pos[i]]);
    return sz(P);
}

/* Pair run: queries (a, b) = (a_0 + j da, b_0 - j db), j = 0, 1, ... (kind
 * 1: a_0 = a_lo, b_0 = S - a_lo, da = db = 1; kind 2, only where STRIDE: as
 * stored); two queries per step, first words from h0; a first-word match is
 * checked on all W words outside the scan loop (a false match, probability
 * 2^-32 per query, resumes it).  Returns the offset of the first hit or -1,
 * and the hit value for query_tail in *hit (kind 1: a; kind 2: the offset).
 * STRIDE = false (kernels of code sets without strided runs) compiles the
 * kind-1 walk alone: the extra registers cost the mixed-code kernels. */
template <int W, bool STRIDE>
__device__ __forceinline__ int walk_pairs(const uint4 &v0, const uint4 &v1,
                                          const typename Syn<W>::T *__restrict__ h,
                                          const uint32_t *__restrict__ h0,
                                          const typename Syn<W>::T s0, uint32_t P0, int n,
                                          uint32_t *hit)
{
    const int len = run_count(v0);
    if constexpr (!STRIDE) {
        const int S = (int)(v0.z & 0xFFu);
        const int a_first = (int)((v0.z >> 8) & 0xFFu);
        int j = 0;
        for (;;) {
            int cand = -1;
            for (; j < len; j += 2) {
                const int a = a_first + j;
                const int b = S - a;
                /* the second slot is clamped into the table and masked past the run */
                const int a1 = min(a + 1, n), b1 = max(b - 1, 1);
                const bool m0 = (h0[a - 1] ^ h0[b - 1]) == P0;
                const bool m1 = ((h0[a1 - 1] ^ h0[b1 - 1]) == P0) && (j + 1 < len);
                if (m0 || m1) {
                    cand = j + (m0 ? 0 : 1);
                    break;
                }
            }
            if (cand < 0)
                return -1;
            if (W == 1 ||
                verify_query<W>(v0, v1, h, s0, n, (uint32_t)(a_first + cand), nullptr)) {
                *hit = (uint32_t)(a_first + cand);
                return cand;
            }
            j = cand + 1;
        }
    }
    const bool stride = run_kind(v0) == ORBG_RUN_STRIDE;
    const int a_first = stride ? (int)(v0.z & 0xFFu) : (int)((v0.z >> 8) & 0xFFu);
    const int b_first =
        stride ? (int)((v0.z >> 8) & 0xFFu) : (int)(v0.z & 0xFFu) - a_first;
    const int da = stride ? (int)((v0.z >> 16) & 0xFFu) : 1;
    const int db = stride ? (int)(v0.z >> 24) : 1;
    int j = 0;
    for (;;) {
        int cand = -1;
        int a = a_first + j * da, b = b_first - j * db;
        for (; j < len; j += 2, a += 2 * da, b -= 2 * db) {
            /* the second slot is clamped into the table and masked past the run */
            const int a1 = min(a + da, n), b1 = max(b - db, 1);
            const bool m0 = (h0[a - 1] ^ h0[b - 1]) == P0;
            const bool m1 = ((h0[a1 - 1] ^ h0[b1 - 1]) == P0) && (j + 1 < len);
            if (m0 || m1) {
                cand = j + (m0 ? 0 : 1);
                break;
            }
        }
        if (cand < 0)
            return -1;
        const uint32_t hv = stride ? (uint32_t)cand : (uint32_t)(a_first + cand);
        if (W == 1 || verify_query<W>(v0, v1, h, s0, n, hv, nullptr)) {
            *hit = hv;
            return cand;
        }
        j = cand + 1;
    }
}

/* Walk one run of the warp table unless it cannot beat `best`.  Returns the
 * run's first hit index (or ORBG_NONE) and the hit value for the flips. */
template <int W, bool STRIDE = true>
__device__ __forceinline__ uint32_t search_run_warp(const uint4 &v0, const uint4 &v1,
                                                    const typename Syn<W>::T *__restrict__ h,
                                                    const uint32_t *__restrict__ h0,
                                                    const typename Syn<W>::T s0, uint32_t best,
                                                    uint32_t cap, int n, uint32_t *hit)
{
    const uint32_t tstart = v0.x;
    if (!(tstart < best && tstart <= cap))
        return ORBG_NONE;
    const uint32_t P0 = prefix_syndrome<uint32_t>(v0, v1, h0, first_word(s0), run_npre(v0));
    if (run_kind(v0) == ORBG_RUN_SINGLE) {
        if (P0 == 0u && (W == 1 || verify_query<W>(v0, v1, h, s0, n, 0u, nullptr))) {
            *hit = 0u;
            return tstart;
        }
        return ORBG_NONE;
    }
    const int j = walk_pairs<W, STRIDE>(v0, v1, h, h0, s0, P0, n, hit);
    return j < 0 ? ORBG_NONE : tstart + (uint32_t)j;
}

/* Nonzero iff one of the two 16-bit halves of t is zero (the lowest zero
 * half always sets its flag; a borrow can only add flags above it). */
__device__ __forceinline__ uint32_t zero16(uint32_t t)
{
    return (t - 0x00010001u) & ~t & 0x80008000u;
}

/* Walk one run of the CTA table: kind 3 tests the X3 range [aux, aux +
 * count) against the low 16 bits of the prefix syndrome, four queries per
 * step.  Entries at or past x3lim are not built: those queries are formed
 * from the triple list instead (slower, used only near the end of a warp's
 * own table). */
template <int W, bool STRIDE = true>
__device__ __forceinline__ uint32_t search_run_cta(const uint4 &v0, const uint4 &v1,
                                                   const typename Syn<W>::T *__restrict__ h,
                                                   const uint32_t *__restrict__ h0,
                                                   const uint16_t *__restrict__ X3,
                                                   uint32_t x3lim,
                                                   const uint32_t *__restrict__ trip,
                                                   const typename Syn<W>::T s0, uint32_t best,
                                                   uint32_t cap, int n, bool exact16,
                                                   uint32_t *hit)
{
    const uint32_t tstart = v0.x;
    if (!(tstart < best && tstart <= cap))
        return ORBG_NONE;
    const uint32_t P0 = prefix_syndrome<uint32_t>(v0, v1, h0, first_word(s0), run_npre(v0));
    const int kind = run_kind(v0);
    if (kind == ORBG_RUN_TRIPLES) {
        const int len = run_count(v0);
        const uint32_t x0 = v0.z;
        const uint16_t p16 = (uint16_t)P0;
        const bool exact = W == 1 && exact16;
        int j = 0;
        if (x0 + (uint32_t)len <= x3lim) {
            /* aligned 16-byte chunks of eight entries (the table starts on
             * a 16-byte boundary and its allocation is a whole number of
             * chunks), tested at once for an entry equal to p16; a step
             * with one is re-read entry by entry, skipping the entries
             * outside the run */
            const uint32_t end = x0 + (uint32_t)len;
            const uint32_t pp = (uint32_t)p16 * 0x00010001u;
            const uint4 *X4 = reinterpret_cast<const uint4 *>(X3);
            /* two chunks per step; the second is read only inside the run
             * (past its end the table may end) */
            for (uint32_t c = x0 & ~7u; c < end; c += 16u) {
                const uint4 va = X4[c >> 3];
                const bool two = c + 8u < end;
                const uint4 vb = two ? X4[(c >> 3) + 1u] : va;
                if (zero16(va.x ^ pp) | zero16(va.y ^ pp) | zero16(va.z ^ pp) |
                    zero16(va.w ^ pp) | zero16(vb.x ^ pp) | zero16(vb.y ^ pp) |
                    zero16(vb.z ^ pp) | zero16(vb.w ^ pp)) {
                    for (uint32_t e = max(c, x0); e < min(c + 16u, end); e++) {
                        if (X3[e] == p16 &&
                            (exact || verify_query<W>(v0, v1, h, s0, n, e, trip))) {
                            *hit = e;
                            return tstart + (e - x0);
                        }
                    }
                }
            }
            return ORBG_NONE;
        }
        for (; j < len; j++) { /* entries not built: form each triple */
            const uint32_t t = x0 + (uint32_t)j;
            const uint32_t c = __ldg(trip + t);
            const uint32_t v = h0[c & 0xFFu] ^ h0[(c >> 8) & 0xFFu] ^ h0[(c >> 16) & 0xFFu];
            if (v == P0 && (W == 1 || verify_query<W>(v0, v1, h, s0, n, t, trip))) {
                *hit = t;
                return tstart + (uint32_t)j;
            }
        }
        return ORBG_NONE;
    }
    if (kind == ORBG_RUN_SINGLE) {
        if (P0 == 0u && (W == 1 || verify_query<W>(v0, v1, h, s0, n, 0u, nullptr))) {
            *hit = 0u;
            return tstart;
        }
        return ORBG_NONE;
    }
    const int j = walk_pairs<W, STRIDE>(v0, v1, h, h0, s0, P0, n, hit);
    return j < 0 ? ORBG_NONE : tstart + (uint32_t)j;
}

__device__ __forceinline__ void load_run(const OrbgTable &tb, uint32_t e, uint4 *v0, uint4 *v1)
{
    if (e < tb.nruns) {
        const uint4 *runs4 = reinterpret_cast<const uint4 *>(tb.runs);
        *v0 = __ldg(runs4 + 2 * e);
        *v1 = __ldg(runs4 + 2 * e + 1);
    } else {
        *v0 = make_uint4(ORBG_NONE, 0u, 0u, 0u); /* tstart = NONE: never searched */
        *v1 = make_uint4(0u, 0u, 0u, 0u);
    }
}

/* ----------------------------------------------------- step 5: output */

/* The owner of the winning run applies its flips to the staged codeword. */
template <bool STRIDE = true>
__device__ __forceinline__ void apply_flips(const OrbgTable &tb, uint32_t run, uint32_t hit,
                                            const uint32_t *trip, const uint8_t *pi,
                                            uint8_t *cw)
{
    const uint4 *runs4 = reinterpret_cast<const uint4 *>(tb.runs);
    const uint4 v0 = __ldg(runs4 + 2 * run), v1 = __ldg(runs4 + 2 * run + 1);
    const int npre = run_npre(v0);
    for (int i = 0; i < npre; i++) {
        const uint32_t wd = i < 4 ? v0.w : i < 8 ? v1.x : i < 12 ? v1.y : i < 16 ? v1.z : v1.w;
        cw[pi[(int)((wd >> (8 * (i & 3))) & 0xFFu) - 1]] ^= 1;
    }
    int pos[3];
    const int k = query_tail<STRIDE>(v0, hit, trip, pos);
    for (int i = 0; i < k; i++)
        cw[pi[pos[i]]] ^= 1;
}

/* ---------------------------------------------------- the flat table */

/* Flat-table pattern t (1-based): up to ORBG_FLAT_POS positions. */
__device__ __forceinline__ int flat_pos(const uint2 &e, int i)
{
    return (int)(((i < 4 ? e.x : e.y) >> (8 * (i & 3))) & 0xFFu); /* 1-based, 0 = none */
}

/* Flat-table entry t (1-based) or, past the table or the cap, an entry with
 * no positions whose rank count is 0. */
__device__ __forceinline__ uint2 flat_entry(const OrbgDeviceCode &code, uint32_t t, uint32_t cap)
{
    if (t > code.nflat || t > cap)
        return make_uint2(0u, 0u);
    return __ldg(reinterpret_cast<const uint2 *>(code.flat) + (t - 1));
}

/* The step byte of entry e: ranks needed (bits 0-4), largest weight
 * (bits 5-7). */
__device__ __forceinline__ uint32_t flat_step(const uint2 &e) { return e.y >> 24; }

/* Is flat pattern e a hit?  wmax (warp-uniform) bounds its weight.  (An
 * entry with no positions is tested as the zero pattern: callers pass only
 * entries of real queries past query 1.) */
template <int W>
__device__ __forceinline__ bool flat_test(const typename Syn<W>::T *__restrict__ h,
                                          const uint32_t *__restrict__ h0,
                                          const typename Syn<W>::T s0, const uint2 &e, int n,
                                          int wmax = ORBG_FLAT_POS)
{
    typedef typename Syn<W>::T T;
    uint32_t P0 = first_word(s0);
#pragma unroll
    for (int i = 0; i < ORBG_FLAT_POS; i++) {
        if (i >= wmax)
            break;
        const int q = flat_pos(e, i);
        P0 ^= h0[q - 1];
    }
    if (P0 != 0u)
        return false;
    if (W > 1) {
        T P = s0;
        for (int i = 0; i < ORBG_FLAT_POS; i++) {
            const int q = flat_pos(e, i);
            if (q)
                P = sx(P, h[q - 1]);
        }
        if (!sz(P))
            return false;
    }
    return true;
}

/* Lane's query of flat step `base` (queries base+1 .. base+32): returns its
 * index if it is a hit, else ORBG_NONE. */
template <int W>
__device__ __forceinline__ uint32_t flat_query(const OrbgDeviceCode &code,
                                               const typename Syn<W>::T *__restrict__ h,
                                               const uint32_t *__restrict__ h0,
                                               const typename Syn<W>::T s0, uint32_t base,
                                               uint32_t cap, int lane)
{
    const uint32_t t = base + (uint32_t)lane + 1u;
    if (t > code.nflat || t > cap)
        return ORBG_NONE;
    const uint2 e = flat_entry(code, t, cap);
    return flat_test<W>(h, h0, s0, e, code.n) ? t : ORBG_NONE;
}

/* Flips of flat pattern t into the staged codeword. */
__device__ __forceinline__ void apply_flat_flips(const OrbgDeviceCode &code, uint32_t t,
                                                 const uint8_t *pi, uint8_t *cw)
{
    const uint2 e = __ldg(reinterpret_cast<const uint2 *>(code.flat) + (t - 1));
    for (int i = 0; i < ORBG_FLAT_POS; i++) {
        const int q = flat_pos(e, i);
        if (q)
            cw[pi[q - 1]] ^= 1;
    }
}

/* First group of `tb` holding a query >= q (reach is non-decreasing). */
__device__ __forceinline__ uint32_t group_reaching(const OrbgTable &tb, uint32_t q)
{
    uint32_t lo = 0, hi = tb.ngroups;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(tb.group_reach + mid) >= q)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------ one warp, one block */

/*
 * Decode one block with one warp over the warp table.  Groups are walked
 * from 0 while their floor (the smallest first index of any later run) is
 * below the best hit, at most `cap`, and at most `budget`.  If the walk
 * stops on the budget with the result still open, the block is not
 * written: its index is appended to heavy[] (when heavy != NULL) for
 * decode_block_cta, with its reliability order and starting syndrome in
 * the handover record of the same slot when one is free (hand_cap; bit 63
 * of the heavy[] entry says so).  On the CTA table (TRIP) a walk that
 * reaches groups needing triple sums past the warp's own table
 * (ORBG_X3_WARP_S3) with no hit stops there and is listed the same way,
 * whatever the budget; on the warp table, with budget >= cap every block
 * finishes here.  LS: llr points into shared memory (the batched kernel
 * stages it there).
 */
template <int K, int W, bool LS = false, bool TRIP = false, bool PF = true, bool ROLL = true,
          bool STRIDE = true>
__device__ void decode_block_warp(const OrbgDeviceCode &code, const float *__restrict__ llr,
                                  uint8_t *__restrict__ cw_out, uint32_t *__restrict__ q_out,
                                  uint8_t *__restrict__ ab_out, uint32_t cap, uint32_t budget,
                                  unsigned char *__restrict__ bsm, int lane,
                                  unsigned long long *heavy, unsigned long long *heavy_count,
                                  unsigned long long block_index, uint16_t *X3w = nullptr,
                                  unsigned char *hand = nullptr, uint32_t hand_cap = 0)
{
    typedef typename Syn<W>::T T;
    const int n = code.n;
    const OrbgTable &tb = TRIP ? code.cta : code.warp;
    BlockSmem<W> sm(bsm, n);
    uint32_t key[K];
    bool nan;
    const T s0 = load_block<K, W, LS>(code, llr, key, sm.cw, lane, &nan);
    uint32_t best = ORBG_NONE, my_t = ORBG_NONE, my_run = 0, my_hit = 0;
    uint32_t handover = 0;
    bool done = true;
    if (nan) {
        best = ORBG_NONE - 1; /* marker: NaN block */
    } else if (sz(s0)) {
        best = 1u;            /* query 1, the zero pattern, is a codeword */
    } else {
        /* the flat table: 32 consecutive queries per step, in query order,
         * so the first step with a hit holds the answer.  Ranks are
         * extracted as the steps need them (one more than needed, so that a
         * tie across the boundary is seen); a tie sorts everything exactly. */
        sort_lane<K>(key);
        if (lane == 0) {
            sm.h[-1] = szero<T>();
            if (W > 1)
                sm.h0[-1] = 0u;
        }
        bool sorted = false;
        int have = 0;
        uint32_t prev = 0xFFFFFFFFu, mine_key = 0xFFFFFFFFu;
        for (uint32_t base = 0; base < code.nflat && base < cap; base += 32u) {
            const uint32_t t = base + (uint32_t)lane + 1u;
            const uint2 e = flat_entry(code, t, cap);
            /* every entry of a step carries the step byte; entries past the
             * table are zero */
            const uint32_t step = __reduce_max_sync(FULL_MASK, flat_step(e));
            if (!sorted) {
                const int upto = min((int)(step & 31u) + 1, n);
                if (upto > have) {
                    if (extract_ranks<K>(key, have, upto, &prev, &mine_key, lane)) {
                        make_keys<K, LS>(llr, n, lane, key);
                        sort_block<K, LS, ROLL>(key, llr, n, lane);
                        build_perm<K, W>(code, key, sm, lane);
                        sorted = true;
                    } else {
                        perm_ranks<K, W>(code, mine_key, have, upto, sm, lane);
                        have = upto;
                    }
                    __syncwarp();
                }
            }
            const uint32_t mine =
                (e.x | e.y << 8) != 0u && flat_test<W>(sm.h, sm.h0, s0, e, n, (int)(step >> 5))
                    ? t
                    : ORBG_NONE;
            const uint32_t gbest = __reduce_min_sync(FULL_MASK, mine);
            if (gbest != ORBG_NONE) {
                best = gbest;
                if (mine == gbest) {
                    my_t = mine;
                    my_run = ORBG_NONE; /* a flat-table hit */
                }
                break;
            }
        }
        if (best == ORBG_NONE && !sorted && cap > code.nflat) {
            /* leaving the flat table: every rank is needed (unless the
             * cap ended the search inside it: the walk below then stops at
             * its first floor, past the cap) */
            make_keys<K, LS>(llr, n, lane, key);
            sort_block<K, LS, ROLL>(key, llr, n, lane);
            build_perm<K, W>(code, key, sm, lane);
            __syncwarp();
        }
        uint32_t stop = ORBG_NONE;
        if (best == ORBG_NONE) {
            /* then the runs, from the first group past the flat table; the
             * budget (and, on the CTA table, the warp's own triple table)
             * only ends the walk while no hit is known */
            const uint32_t g0 = tb.flat_group;
            int built = 5;         /* triple sums whose X3 entries exist */
            uint32_t x3lim = 0;    /* X3 entries built */
            /* PF: group g + 1's runs, floor and triple need are loaded while
             * g is searched (costs registers: off where they are short) */
            uint4 n0, n1;
            uint32_t nfloor = 0;
            int nneed = 0;
            if (PF) {
                load_run(tb, g0 * ORBG_GROUP + (uint32_t)lane, &n0, &n1);
                nfloor = g0 < tb.ngroups ? __ldg(tb.group_floor + g0) : ORBG_NONE;
                nneed = TRIP && g0 < tb.ngroups ? (int)__ldg(tb.group_s3 + g0) : 0;
            }
            for (uint32_t g = g0; g < tb.ngroups; g++) {
                uint4 v0, v1;
                uint32_t floor;
                int need_g = 0;
                if (PF) {
                    floor = nfloor;
                    need_g = nneed;
                    v0 = n0;
                    v1 = n1;
                } else {
                    floor = __ldg(tb.group_floor + g);
                }
                if (floor >= best || floor > cap || (best == ORBG_NONE && floor > budget)) {
                    stop = floor;
                    break;
                }
                if (PF && g + 1u < tb.ngroups) {
                    load_run(tb, (g + 1u) * ORBG_GROUP + (uint32_t)lane, &n0, &n1);
                    nfloor = __ldg(tb.group_floor + g + 1u);
                    if (TRIP)
                        nneed = (int)__ldg(tb.group_s3 + g + 1u);
                }
                if (TRIP) {
                    const int need = PF ? need_g : (int)__ldg(tb.group_s3 + g);
                    if (need > built) {
                        if (best == ORBG_NONE && need > ORBG_X3_WARP_S3) {
                            stop = floor;
                            break;
                        }
                        const int upto = min(need, ORBG_X3_WARP_S3);
                        if (upto > built) {
                            const uint32_t lo = __ldg(code.x3off + built + 1);
                            x3lim = __ldg(code.x3off + upto + 1);
                            build_x3(code, sm.h0, X3w, lo, x3lim, (uint32_t)lane, 32u);
                            __syncwarp();
                            built = upto;
                        }
                    }
                }
                if (!PF)
                    load_run(tb, g * ORBG_GROUP + (uint32_t)lane, &v0, &v1);
                uint32_t hv = 0;
                uint32_t mine;
                if (TRIP)
                    mine = search_run_cta<W, STRIDE>(v0, v1, sm.h, sm.h0, X3w, x3lim, code.trip, s0,
                                             best, cap, n, code.exact16 != 0, &hv);
                else
                    mine = search_run_warp<W, STRIDE>(v0, v1, sm.h, sm.h0, s0, best, cap, n, &hv);
                const uint32_t gbest = __reduce_min_sync(FULL_MASK, mine);
                if (gbest < best) {
                    best = gbest;
                    if (mine == gbest) {
                        my_t = mine;
                        my_run = g * ORBG_GROUP + (uint32_t)lane;
                        my_hit = hv;
                    }
                }
            }
        }
        done = stop >= best || stop > cap; /* exhausted tables give stop = NONE */
        handover = stop;
    }
    if (!done) {
        /* every query below `handover` was tested without a hit; the block
         * is fully sorted here (the walk past the flat table sorts it) */
        if (heavy != nullptr) {
            unsigned long long slot = 0;
            if (lane == 0)
                slot = atomicAdd(heavy_count, 1ull);
            slot = __shfl_sync(FULL_MASK, slot, 0);
            const bool keep = slot < (unsigned long long)hand_cap;
            if (keep) {
                unsigned char *rec = hand + slot * ORBG_HANDOVER_BYTES;
#pragma unroll
                for (int k = 0; k < K; k++) {
                    const int e = lane * K + k;
                    if (e < n)
                        rec[e] = sm.pi[e];
                }
                if (lane == 0)
                    *reinterpret_cast<T *>(rec + 256) = s0;
            }
            if (lane == 0)
                heavy[slot] = block_index | ((unsigned long long)handover << 32) |
                              (keep ? 1ull << 63 : 0ull);
        }
        __syncwarp();
        return;
    }
    const bool is_nan = best == ORBG_NONE - 1;
    const bool hit = !is_nan && best <= cap;
    if (hit && my_t == best) {
        if (my_run == ORBG_NONE)
            apply_flat_flips(code, my_t, sm.pi, sm.cw);
        else
            apply_flips<STRIDE>(tb, my_run, my_hit, code.trip, sm.pi, sm.cw);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < K; k++) {
        int i = k * 32 + lane;
        if (i < n)
            cw_out[i] = sm.cw[i];
    }
    if (lane == 0) {
        *q_out = is_nan ? 0u : hit ? best : cap;
        *ab_out = is_nan ? 2 : hit ? 0 : 1;
    }
    __syncwarp();
}

/* ------------------------------------------------ one CTA, one block */

/*
 * All warps of the CTA decode one block over the CTA table.  Warp 0 loads
 * and sorts; all threads then fill the triple table X3 from the permuted
 * first-word columns; then warp w walks groups w, w + nw, w + 2 nw, ...
 * Each warp stops at its first group whose floor is at least the shared
 * best (or above the cap): floors never decrease with the group index and
 * the best never increases, so no group that could hold the final best is
 * skipped.
 */
template <int K, int W, bool STRIDE = true>
__device__ void decode_block_cta(const OrbgDeviceCode &code, const float *__restrict__ llr,
                                 uint8_t *__restrict__ cw_out, uint32_t *__restrict__ q_out,
                                 uint8_t *__restrict__ ab_out, uint32_t cap,
                                 unsigned char *__restrict__ bsm, uint16_t *__restrict__ X3,
                                 uint32_t *s_best, typename Syn<W>::T *s_s0, uint32_t from,
                                 int warp, int lane, int nwarps,
                                 const unsigned char *__restrict__ rec = nullptr)
{
    typedef typename Syn<W>::T T;
    const int n = code.n;
    const OrbgTable &tb = code.cta;
    BlockSmem<W> sm(bsm, n);
    if (rec != nullptr) {
        /* phase 1's handover record: the block's order and starting
         * syndrome; every thread takes a share of the positions */
        for (int i = (int)threadIdx.x; i < n; i += (int)blockDim.x) {
            sm.cw[i] = __ldg(llr + i) > 0.0f ? 1 : 0;
            const int idx = (int)rec[i];
            sm.pi[i] = (uint8_t)idx;
            const T col = load_col<W>(code.hcol, idx);
            sm.h[i] = col;
            if (W > 1)
                sm.h0[i] = first_word(col);
        }
        if (threadIdx.x == 0) {
            sm.h[-1] = szero<T>();
            if (W > 1)
                sm.h0[-1] = 0u;
            *s_best = ORBG_NONE;
            *s_s0 = *reinterpret_cast<const T *>(rec + 256);
        }
    } else if (warp == 0) {
        uint32_t key[K];
        bool nan;
        const T s0 = load_block<K, W>(code, llr, key, sm.cw, lane, &nan);
        if (nan || sz(s0)) {
            /* not expected here (the warp pass finishes these), but exact */
            if (lane == 0)
                *s_best = nan ? ORBG_NONE - 1 : 1u;
        } else {
            sort_block<K>(key, llr, n, lane);
            build_perm<K, W>(code, key, sm, lane);
            if (lane == 0) {
                *s_best = ORBG_NONE;
                *s_s0 = s0;
            }
        }
    }
    __syncthreads();
    const uint32_t start = *s_best;
    if (start == ORBG_NONE)
        build_x3(code, sm.h0, X3, 0u, code.ntrip, threadIdx.x, blockDim.x);
    __syncthreads();
    uint32_t my_t = ORBG_NONE, my_run = 0, my_hit = 0;
    if (start == ORBG_NONE) {
        const T s0 = *s_s0;
        bool stopped = false;
        uint32_t g = (uint32_t)warp;
        if (from <= code.nflat) {
            /* flat table, steps interleaved over the warps: a warp that sees
             * a hit, or a step at or past the best, has nothing left to do
             * below the best (every query <= nflat is some warp's step) */
            for (uint32_t base = 32u * (uint32_t)warp; base < code.nflat && base < cap;
                 base += 32u * (uint32_t)nwarps) {
                if (base + 1u >= *((volatile uint32_t *)s_best)) {
                    stopped = true;
                    break;
                }
                const uint32_t mine = flat_query<W>(code, sm.h, sm.h0, s0, base, cap, lane);
                const uint32_t gbest = __reduce_min_sync(FULL_MASK, mine);
                if (gbest != ORBG_NONE) {
                    if (mine == gbest) {
                        my_t = mine;
                        my_run = ORBG_NONE;
                        atomicMin(s_best, mine);
                    }
                    stopped = true;
                    break;
                }
            }
            g += tb.flat_group;
        } else {
            /* every query below `from` was tested by the warp pass */
            g += group_reaching(tb, from);
        }
        if (!stopped) {
            uint4 n0, n1;
            load_run(tb, g * ORBG_GROUP + (uint32_t)lane, &n0, &n1);
            uint32_t nfloor = g < tb.ngroups ? __ldg(tb.group_floor + g) : ORBG_NONE;
            for (; g < tb.ngroups; g += (uint32_t)nwarps) {
                const uint32_t floor = nfloor;
                const uint32_t best = *((volatile uint32_t *)s_best);
                if (floor >= best || floor > cap)
                    break;
                const uint4 v0 = n0, v1 = n1;
                /* the warp's next group, loaded while this one is searched */
                const uint32_t gn = g + (uint32_t)nwarps;
                load_run(tb, gn * ORBG_GROUP + (uint32_t)lane, &n0, &n1);
                nfloor = gn < tb.ngroups ? __ldg(tb.group_floor + gn) : ORBG_NONE;
                uint32_t hv = 0;
                const uint32_t mine =
                    search_run_cta<W, STRIDE>(v0, v1, sm.h, sm.h0, X3, code.ntrip, code.trip, s0, best,
                                      cap, n, code.exact16 != 0, &hv);
                const uint32_t gbest = __reduce_min_sync(FULL_MASK, mine);
                if (gbest != ORBG_NONE) {
                    if (mine == gbest) {
                        my_t = mine;
                        my_run = g * ORBG_GROUP + (uint32_t)lane;
                        my_hit = hv;
                        atomicMin(s_best, mine);
                    }
                }
            }
        }
    }
    __syncthreads();
    const uint32_t best = *s_best;
    const bool is_nan = best == ORBG_NONE - 1;
    const bool hit = !is_nan && best <= cap;
    if (start == ORBG_NONE && hit && my_t == best) {
        if (my_run == ORBG_NONE)
            apply_flat_flips(code, my_t, sm.pi, sm.cw);
        else
            apply_flips<STRIDE>(tb, my_run, my_hit, code.trip, sm.pi, sm.cw);
    }
    __syncthreads();
    for (int i = warp * 32 + lane; i < n; i += nwarps * 32)
        cw_out[i] = sm.cw[i];
    if (warp == 0 && lane == 0) {
        *q_out = is_nan ? 0u : hit ? best : cap;
        *ab_out = is_nan ? 2 : hit ? 0 : 1;
    }
    __syncthreads();
}

/* ----------------------------------------------------------- dispatch */

/* Runtime dispatch on (n, syndrome width), warp-uniform; only variants up to
 * (KMAX keys per lane, WMAX syndrome words) are instantiated. */
#define ORBG_DISPATCH(KMAX, WMAX, CALL)                                   \
    do {                                                                  \
        const int n_ = code.n, w_ = code.w32;                             \
        bool done_ = false;                                               \
        if constexpr (KMAX >= 8) {                                        \
            if (!done_ && n_ > 128) { ORBG_DISPATCH_W(8, WMAX, CALL); done_ = true; } \
        }                                                                 \
        if constexpr (KMAX >= 4) {                                        \
            if (!done_ && n_ > 64) { ORBG_DISPATCH_W(4, WMAX, CALL); done_ = true; } \
        }                                                                 \
        if constexpr (KMAX >= 2) {                                        \
            if (!done_ && n_ > 32) { ORBG_DISPATCH_W(2, WMAX, CALL); done_ = true; } \
        }                                                                 \
        if (!done_) { ORBG_DISPATCH_W(1, WMAX, CALL); }                  \
    } while (0)

#define ORBG_DISPATCH_W(KK, WMAX, CALL)                                   \
    do {                                                                  \
        bool dw_ = false;                                                 \
        if constexpr (WMAX >= 4) {                                        \
            if (w_ > 2) { CALL(KK, 4); dw_ = true; }                      \
        }                                                                 \
        if constexpr (WMAX >= 2) {                                        \
            if (!dw_ && w_ == 2) { CALL(KK, 2); dw_ = true; }             \
        }                                                                 \
        if (!dw_) { CALL(KK, 1); }                                        \
    } while (0)

}  // namespace orbg_dev
