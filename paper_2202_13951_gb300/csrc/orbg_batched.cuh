/*
 * orbg_batched.cuh -- phase 1 of the batched form.  orbg_batched_inst.cu
 * instantiates it once per (keys per lane, syndrome width) pair; the build
 * compiles those twelve objects in parallel.
 *
 * Phase 1 (orbg_batched_kernel): each warp pulls `grab` blocks at a time
 * from an atomic work queue and decodes each with decode_block_warp, giving
 * it a query budget.  Most blocks finish inside the budget (at high SNR
 * query 1 already decodes).  A block still open when its warp reaches the
 * budget is appended to a heavy list.
 * Phase 2 (orbg_heavy_kernel, orbg_heavy.cuh): each CTA pulls heavy blocks
 * one at a time and decodes each with all its warps (decode_block_cta), so a
 * block that needs up to 1e6 queries is searched by a whole SM instead of a
 * single warp.
 * Both phases compute the exact first hit of the same query order, so the
 * result equals the plain form's block for block.
 *
 * ONE: every block belongs to one code, passed by value as a kernel
 * parameter (constant bank) and decoded with its exact keys-per-lane K and
 * syndrome width W; otherwise each block's code comes from the device array
 * and K, W are dispatched per block up to KMAX, WMAX.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_pipeline.h>

#include "orbg_decode_block.cuh"
#include "orbg_heavy.cuh"

namespace orbg_batched_impl {

using namespace orbg_dev;

constexpr int kCounters = ORBG_BATCHED_COUNTERS;

/* resident phase-1 CTAs per SM the register allocation is sized for: three
 * for one code or one decoder variant (80 registers, no spills), two for
 * the kernel that dispatches per block (holding every variant it spilled at
 * 80; at two it holds them in registers) */
#ifndef ORBG_PHASE1_MIN_CTAS
#define ORBG_PHASE1_MIN_CTAS 3
#endif
#ifndef ORBG_PHASE1_MIN_CTAS_MIXED
#define ORBG_PHASE1_MIN_CTAS_MIXED 2
#endif

/* How a phase-1 kernel finds each block's decoder: P1_ONE every block is
 * the code in the kernel's parameters; P1_GENERIC each block's code from the
 * device array, dispatched to K <= KMAX, W <= WMAX; P1_EXACT each block's
 * code from the device array, all of keys per lane KMAX and width WMAX (one
 * decoder variant per launch, the blocks taken from their sort buckets). */
enum { P1_ONE = 0, P1_GENERIC = 1, P1_EXACT = 2 };

template <int KMAX, int WMAX, int MODE, bool STRIDE = true>
__global__ void __launch_bounds__(256, MODE == P1_GENERIC ? ORBG_PHASE1_MIN_CTAS_MIXED
                                                          : ORBG_PHASE1_MIN_CTAS)
    orbg_batched_kernel(
    const OrbgDeviceCode *__restrict__ codes, int ncodes, const int32_t *__restrict__ code_id,
    const int64_t *__restrict__ llr_off, const float *__restrict__ llr, int64_t B, uint32_t cap,
    uint32_t budget, uint8_t *__restrict__ cw, const int64_t *__restrict__ cw_off,
    uint32_t *__restrict__ q, uint8_t *__restrict__ ab, unsigned long long *__restrict__ counters,
    unsigned long long *__restrict__ queue, unsigned long long *__restrict__ heavy,
    const uint32_t *__restrict__ perm,
    unsigned char *__restrict__ hand, uint32_t hand_cap, unsigned long long b_base,
    uint32_t bstride, uint32_t x3w_bytes, int grab, const uint32_t *__restrict__ range_count,
    int blo, int bhi, const __grid_constant__ OrbgDeviceCode code0)
{
    constexpr bool ONE = MODE == P1_ONE;
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
    const int64_t n0 = ONE ? code0.n : codes[0].n;

    /* the queue's slots: all B, or (range_count: the per-bucket counts of
     * the sort into perm) the slots of buckets [blo, bhi) */
    int64_t slot_lo = 0, slot_hi = B;
    if (range_count) {
        uint32_t before = 0, inside = 0;
        for (int i = lane; i < bhi; i += 32) {
            const uint32_t c = range_count[i];
            if (i < blo)
                before += c;
            else
                inside += c;
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            before += __shfl_xor_sync(FULL_MASK, before, m);
            inside += __shfl_xor_sync(FULL_MASK, inside, m);
        }
        slot_lo = before;
        slot_hi = (int64_t)before + inside;
    }
    /* the warp's block sequence: `grab` consecutive queue slots per atomic;
     * with perm (mixed codes) slot i holds the block perm[i], so that the
     * blocks of one decoder variant are decoded together.  A warp that finds
     * the queue empty lets a programmatically dependent launch (the next
     * variant's) start on the SMs this one's last blocks leave idle. */
    int64_t pos = 0, end = 0;
    auto next_block = [&]() -> int64_t {
        if (pos >= end) {
            unsigned long long c = 0;
            if (lane == 0)
                c = atomicAdd(queue, (unsigned long long)grab);
            c = __shfl_sync(FULL_MASK, c, 0);
            pos = slot_lo + (int64_t)c;
            end = min(pos + (int64_t)grab, slot_hi);
            if (pos >= slot_hi) {
                asm volatile("griddepcontrol.launch_dependents;");
                return B;
            }
        }
        const int64_t slot = pos++;
        return perm ? (int64_t)__ldg(perm + slot) : slot;
    };
    auto stage = [&](int64_t b, int slot) {
        if (b < B) {
            const int cid = ONE ? 0 : code_id ? code_id[b] : 0;
            if (cid >= 0 && cid < ncodes) {
                const int n = ONE ? code0.n : codes[cid].n;
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
        const int cid = ONE ? 0 : code_id ? code_id[b] : 0;
        const int64_t co = cw_off ? cw_off[b] : b * n0;
        const float *l = ring + slot * kSlot;
        if (ONE) {
            /* one code, read from the kernel's parameters: K and W are exact;
             * its sort is unrolled unless it is the 256-key one (for mixed
             * codes, where several decoder variants share the instruction
             * cache, the sort's stage loops stay rolled) */
            decode_block_warp<KMAX, WMAX, true, true, (KMAX <= 4), (KMAX >= 8)>(code0, l, cw + co, q + b, ab + b,
                                                            cap, budget, bsm, lane, heavy,
                                                            &counters[1],
                                                            b_base + (unsigned long long)b, X3w,
                                                            hand, hand_cap);
        } else if (cid < 0 || cid >= ncodes) {
            if (lane == 0) {
                q[b] = 0u;
                ab[b] = 2;
            }
        } else if (MODE == P1_EXACT) {
            /* one decoder variant: K and W exact; the block's descriptor is
             * read where it is used (a register copy of it spilled) */
            decode_block_warp<KMAX, WMAX, true, true, (KMAX <= 4), (KMAX >= 8), STRIDE>(
                codes[cid], l, cw + co, q + b, ab + b, cap, budget, bsm, lane, heavy, &counters[1],
                b_base + (unsigned long long)b, X3w, hand, hand_cap);
        } else {
            const OrbgDeviceCode code = codes[cid];
#define ORBG_CALL_WARP(KK, WW)                                                                 \
    decode_block_warp<KK, WW, true, true, false, true>(code, l, cw + co, q + b, ab + b, cap, \
                                                 budget, bsm, lane, heavy, &counters[1],    \
                                                 b_base + (unsigned long long)b, X3w, hand,  \
                                                 hand_cap)
            ORBG_DISPATCH(KMAX, WMAX, ORBG_CALL_WARP);
#undef ORBG_CALL_WARP
        }
        __syncwarp(); /* slot is free before it is refilled */
        b = bn;
        bn = next_block();
        slot ^= 1;
    }
    __pipeline_wait_prior(0);
    /* a launch that may have started before the previous one in its stream
     * ended completes only after it (a no-op for any other launch), so the
     * next ordinary launch sees every phase-1 block finished */
    asm volatile("griddepcontrol.wait;" ::: "memory");
}


/* Phase 1 of one decoder variant (K, W): the blocks of sort buckets
 * [blo, bhi) of ss.perm (blo < 0: every block, in order), on its own queue.
 * pdl: the launch may begin while the previous launch in the stream (the
 * previous variant's) finishes its last blocks.  STRIDE: the set holds
 * codes with strided pair runs. */
template <int K, int W, bool STRIDE>
int launch_exact_t(const OrbgBatchedArgs &a, const OrbgScratch &ss, unsigned long long *queue,
                   int blo, int bhi, int pdl)
{
    const int wpc = a.warps_per_cta > 0 ? (a.warps_per_cta > 8 ? 8 : a.warps_per_cta) : 8;
    const int g = a.grab < 1 ? 1 : a.grab;
    const int nk = a.n_max < 32 * K ? a.n_max : 32 * K;
    const uint32_t bstride = block_smem_bytes(nk, W);
    auto k1 = orbg_batched_kernel<K, W, P1_EXACT, STRIDE>;
    const uint32_t x3w_bytes = triple_table_bytes(a.x3w_max);
    const size_t smem1 = ((size_t)bstride + 2u * 32u * K * sizeof(float) + x3w_bytes) * wpc;
    int grid = 0;
    int rc = orbg_grid_for((const void *)k1, wpc * 32, smem1, a.ctas_per_sm, &grid);
    if (rc != 0)
        return rc;
    if (blo < 0) {
        const int64_t need = ((a.B + g - 1) / g + wpc - 1) / wpc;
        if (grid > need)
            grid = (int)(need > 0 ? need : 1);
    }
    const bool sorted = blo >= 0;
    OrbgDeviceCode c0{};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(wpc * 32));
    cfg.dynamicSmemBytes = smem1;
    cfg.stream = (cudaStream_t)a.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return (int)cudaLaunchKernelEx(
        &cfg, k1, a.d_codes, a.ncodes, a.code_id, a.llr_off, a.llr, a.B, a.cap, a.budget, a.cw,
        a.cw_off, a.q, a.ab, ss.counters, queue, ss.heavy,
        sorted ? (const uint32_t *)ss.perm : (const uint32_t *)nullptr, ss.hand, ss.hand_cap,
        (unsigned long long)a.scratch_base, bstride, x3w_bytes, g,
        sorted ? (const uint32_t *)ss.count : (const uint32_t *)nullptr, blo, bhi, c0);
}

template <int KMAX, int WMAX, bool ONE>
cudaError_t launch_t(const OrbgBatchedArgs &a)
{
    const int wpc = a.warps_per_cta > 0 ? (a.warps_per_cta > 8 ? 8 : a.warps_per_cta) : 8;
    const int g = a.grab < 1 ? 1 : a.grab;
    const uint32_t bstride = block_smem_bytes(a.n_max, a.w32_max);
    const OrbgScratch sc =
        orbg_scratch_layout(a.scratch, a.scratch_B > 0 ? a.scratch_B : a.B, a.ncodes);
    unsigned long long *counters = sc.counters;
    unsigned long long *heavy = sc.heavy;
    cudaStream_t st = (cudaStream_t)a.stream;
    cudaError_t e;
    int grid = 0, rc;
    if (a.stage == 2) {
        /* phase 2 over the open blocks every chunk's phase 1 listed */
        return launch_heavy_t<KMAX, WMAX, ONE>(a, counters, heavy, sc.hand);
    }
    /* this launch's slot: its queue heads, bucket counts and cursors, and
     * its blocks' part of the order array */
    const int slot = a.stage == 1 && a.slot == 1 ? 1 : 0;
    const size_t nc = (size_t)a.ncodes + 1;
    unsigned long long *queue = counters + (slot ? 3 : 0);
    unsigned long long *vqueue = counters + 8 + ORBG_MAX_VARIANTS * slot;
    OrbgScratch ss = sc;
    ss.count = sc.count + 2 * nc * slot;
    ss.cursor = ss.count + nc;
    ss.perm = sc.perm + (a.stage == 1 ? a.scratch_base : 0);
    if (a.stage == 0 || a.first_chunk) {
        if ((e = cudaMemsetAsync(a.scratch, 0, sc.zero_bytes, st)) != cudaSuccess)
            return e;
    } else {
        /* a later chunk: fresh queues and bucket counts in its slot; the
         * open-block list and the phase-2 cursor carry on */
        if ((e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(vqueue, 0, ORBG_MAX_VARIANTS * sizeof(unsigned long long),
                                 st)) != cudaSuccess ||
            (e = cudaMemsetAsync(ss.count, 0, 2 * nc * sizeof(uint32_t), st)) != cudaSuccess)
            return e;
    }
    if (!ONE && a.code_id != nullptr && a.var.n >= 1 && a.var.n <= ORBG_MAX_VARIANTS &&
        a.var.d_bucket != nullptr) {
        /* per-block codes: one launch per decoder variant, each a kernel of
         * that variant alone; with several variants the blocks are first
         * grouped by variant (a counting sort by bucket), and each launch
         * after the first may start while the one before finishes */
        const bool sorted = a.var.n > 1;
        if (sorted && (rc = orbg_launch_code_sort(a.code_id, a.var.d_bucket, a.B, a.ncodes, ss,
                                                  st)) != 0)
            return (cudaError_t)rc;
        for (int v = 0; v < a.var.n; v++) {
            rc = orbg_launch_exact(a.var.k[v], a.var.w[v], a, ss, vqueue + v,
                                   sorted ? a.var.blo[v] : -1, a.var.bhi[v], v > 0,
                                   a.has_stride);
            if (rc != 0)
                return (cudaError_t)rc;
        }
    } else {
        /* phase 1: per warp, one block's working set, two LLR slots and its
         * own triple table */
        auto k1 = orbg_batched_kernel<KMAX, WMAX, ONE ? P1_ONE : P1_GENERIC>;
        const uint32_t x3w_bytes = triple_table_bytes(a.x3w_max);
        size_t smem1 = ((size_t)bstride + 2u * 32u * KMAX * sizeof(float) + x3w_bytes) * wpc;
        if ((rc = orbg_grid_for((const void *)k1, wpc * 32, smem1, a.ctas_per_sm, &grid)) != 0)
            return (cudaError_t)rc;
        int64_t units = (a.B + g - 1) / g;
        int64_t need = (units + wpc - 1) / wpc;
        if (grid > need) grid = (int)(need > 0 ? need : 1);
        OrbgDeviceCode c0{};
        if (ONE)
            c0 = *a.code0;
        k1<<<grid, wpc * 32, smem1, st>>>(a.d_codes, a.ncodes, a.code_id, a.llr_off, a.llr, a.B,
                                          a.cap, a.budget, a.cw, a.cw_off, a.q, a.ab, counters,
                                          queue, heavy, nullptr, sc.hand, sc.hand_cap,
                                          (unsigned long long)a.scratch_base, bstride, x3w_bytes,
                                          g, nullptr, 0, 0, c0);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    /* phase 2 runs whatever the budget: a phase-1 walk on the CTA table also
     * stops, open, where it needs triple sums past the warp's own table
     * (decode_block_warp), so the list can hold blocks with a budget at or
     * above the cap too (with an empty list the launch only reads its
     * length) */
    if (a.stage == 1)
        return cudaSuccess; /* phase 2 comes later, over every chunk's list */
    return launch_heavy_t<KMAX, WMAX, ONE>(a, counters, heavy, sc.hand);
}

/* Phases 1 and 2 for keys-per-lane bound KMAX and syndrome width WMAX. */
template <int KMAX, int WMAX>
int launch_kw(const OrbgBatchedArgs &a)
{
    return a.code0 ? (int)launch_t<KMAX, WMAX, true>(a) : (int)launch_t<KMAX, WMAX, false>(a);
}

}  // namespace orbg_batched_impl
