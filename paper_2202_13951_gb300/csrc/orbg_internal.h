/*
 * orbg_internal.h -- data shared between the host side of the library and
 * its CUDA kernels.
 *
 * The query order (Sec. III-B: increasing logistic weight W; this library's
 * tie reading: Hamming weight w ascending, then positions lexicographic) is
 * held as tables of "runs" of consecutive query indices.  Two tables per
 * code, each covering the whole order:
 *
 * Warp table (one warp decodes a block):
 *   kind 0  one pattern of weight 0 or 1 (the prefix is the pattern);
 *   kind 1  a prefix v_1 < ... < v_{w-2} and every pair a < b <= n after it
 *           with a + b = S, a ascending from a_lo;
 *   kind 2  (m-segment orders) a prefix and the pairs (a_0 + j da, b_0 - j db),
 *           j = 0, 1, ...: a pair whose positions lie in two segments of
 *           slopes beta, beta' with beta da = beta' db keeps its weight.
 * CTA table (a CTA decodes a block and first builds the block's triple
 * table X3: the first syndrome word of every triple c < a < b <= n with
 * c + a + b <= S3max, ordered by that sum, then c, then a):
 *   kind 0  as above;
 *   kind 1  as above, used for w = 2 and for triples beyond S3max;
 *   kind 3  a prefix v_1 < ... < v_{w-3} and every triple after it with
 *           c + a + b = S3: a contiguous range of X3, tested against one
 *           prefix syndrome.  Cut into chunks of at most 8..255 queries
 *           (longer deeper in the order).
 * Runs are stored class by class ((W, w) ascending); inside a class they are
 * sorted by length so that the 32 lanes of a warp, which take 32
 * consecutive runs, loop for about the same number of queries.  Every run
 * keeps its own first query index, so the decoder still reports the first
 * hit of the paper's order; a group floor (the smallest first index over
 * runs of groups >= g) tells a warp when no later group can hold an earlier
 * hit.
 */
#ifndef ORBG_INTERNAL_H
#define ORBG_INTERNAL_H

#include <stdint.h>

#define ORBG_GROUP 32          /* runs per warp step: one per lane */
#define ORBG_RUN_MAX_PRE 20    /* prefix positions stored per run */
#define ORBG_MAX_LOGISTIC 255  /* deepest logistic weight a table may reach */
#define ORBG_X3_MAX 16384      /* triple-table entries (32 KiB of shared memory, 16 bits each) */
#define ORBG_X3_WARP_S3 44     /* triple sums a phase-1 warp keeps in its own table */

enum { ORBG_RUN_SINGLE = 0, ORBG_RUN_PAIRS = 1, ORBG_RUN_STRIDE = 2, ORBG_RUN_TRIPLES = 3 };

/* One run: 32 bytes, read by a lane as two 16-byte loads. */
struct OrbgRun {
    uint32_t tstart;    /* 1-based query index of the run's first pattern */
    uint16_t count;     /* patterns in the run, >= 1 */
    uint8_t npre;       /* prefix positions used */
    uint8_t kind;       /* ORBG_RUN_* */
    uint32_t aux;       /* kind 1: S | a_lo << 8 (1-based); kind 2: a_0 | b_0 << 8 | da << 16 |
                         * db << 24 (pattern j's pair is a_0 + j da, b_0 - j db); kind 3:
                         * first X3 index */
    uint8_t pre[ORBG_RUN_MAX_PRE]; /* 1-based prefix positions, ascending; 0 = unused */
};

struct OrbgTable {
    const OrbgRun *runs;         /* [nruns] */
    const uint32_t *group_floor; /* [ngroups] */
    const uint32_t *group_reach; /* [ngroups]: largest query index in groups <= g */
    const uint8_t *group_s3;     /* [ngroups]: largest triple sum any run in groups <= g reads */
    uint32_t nruns;
    uint32_t ngroups;
    uint32_t flat_group;         /* first group holding a query beyond the flat table */
};

/* The flat table: the first `nflat` patterns of the order, 8 bytes each:
 * up to 7 positions, 1-based (0 = unused), then a byte describing the
 * pattern's step of 32: bits 0-4 the number of sorted ranks the step needs
 * (the largest position of that step or an earlier one, at most
 * ORBG_FLAT_RANKS), bits 5-7 the step's largest Hamming weight.  A warp
 * tests 32 consecutive patterns per step before it turns to runs. */
#define ORBG_FLAT_MAX 256
#define ORBG_FLAT_POS 7
#define ORBG_FLAT_RANKS 31

/* What a kernel needs of one code (passed by value or from a device array). */
struct OrbgDeviceCode {
    const uint32_t *hcol;        /* [n][w32]: column j of H, row i at bit i%32 of word i/32 */
    OrbgTable warp;              /* runs of kinds 0, 1 */
    OrbgTable cta;               /* runs of kinds 0, 1, 3 */
    const uint32_t *trip;        /* [ntrip]: c0 | a0 << 8 | b0 << 16 (0-based), X3 order */
    const uint32_t *x3off;       /* [s3max + 2]: first X3 index of each triple sum */
    uint32_t ntrip;
    int32_t s3max;               /* largest triple sum in X3 */
    uint32_t x3w;                /* X3 entries of sums <= ORBG_X3_WARP_S3 (a warp's own table) */
    int32_t exact16;             /* n - k <= 16: 16-bit X3 entries are whole syndromes */
    const uint32_t *flat;        /* [2 * nflat] flat-table patterns, 8 bytes each */
    uint32_t nflat;
    uint32_t max_cap;
    int32_t n;
    int32_t r;
    int32_t w32;                 /* syndrome words: 1, 2 or 4 */
};

#ifdef __cplusplus
static_assert(sizeof(OrbgRun) == 32, "run record must be 32 bytes");
#endif

/* Host-side table builder (orbg_tables.cpp). */
#ifdef __cplusplus
#include <vector>
struct OrbgTables {
    std::vector<OrbgRun> runs;           /* warp table */
    std::vector<uint32_t> group_floor;
    std::vector<OrbgRun> runs_cta;       /* CTA table */
    std::vector<uint32_t> group_floor_cta;
    std::vector<uint32_t> trip;          /* X3 order */
    std::vector<uint8_t> flat;           /* 8 bytes per pattern */
    std::vector<uint32_t> reach, reach_cta;
    std::vector<uint8_t> s3_cta;         /* group_s3 of the CTA table */
    std::vector<uint32_t> x3off;
    int s3max = 0;
    uint32_t nflat = 0, flat_group = 0, flat_group_cta = 0;
    uint64_t patterns = 0;  /* query indices covered (last index) */
    int wmax_logistic = 0;  /* deepest logistic weight in the table */
};
/* The tables for the order of increasing reliability weight J0 w + beta W
 * (one-line full ORBGRAND; J0 = 0, beta = 1 is basic ORBGRAND). */
#define ORBG_MAX_LINE 1024
int orbg_build_tables(int n, uint64_t cap, OrbgTables *out, long J0 = 0, long beta = 1);
/* The m-segment model of Eq. relest_seg: segment i = 1..m covers the
 * sorted positions I[i-1] < j <= I[i] (I[0] = 0, I[m] = n) and position j
 * weighs J[i-1] + beta[i-1] (j - I[i-1]); beta >= 1, J[i-1] >= -beta[i-1]. */
#define ORBG_MAX_SEG 8
#define ORBG_MAX_MODEL (1L << 20) /* largest J or beta of a model */
struct OrbgModel {
    int m;
    int I[ORBG_MAX_SEG + 1];
    long J[ORBG_MAX_SEG];
    long beta[ORBG_MAX_SEG];
};
/* The tables for the m-segment order (reliability weight, then Hamming
 * weight, then positions lexicographically): single, pair and strided pair
 * runs. */
int orbg_build_tables_model(int n, uint64_t cap, const OrbgModel &md, OrbgTables *out);
int orbg_run_pattern(const OrbgRun &r, int j, const uint32_t *trip, int *v);

/* GF(2) helpers on dense 0/1 byte matrices (row-major). */
int orbg_gf2_rank(const uint8_t *M, int rows, int cols);
int orbg_gf2_nullspace(const uint8_t *M, int rows, int cols,
                       std::vector<uint8_t> *basis, int *dim);

/* Kernel launchers (orbg_plain.cu, orbg_batched.cu).  Return a cudaError_t value. */
int orbg_launch_plain(const OrbgDeviceCode &code, const float *llr, int64_t B,
                      uint32_t cap, uint8_t *cw, uint32_t *q, uint8_t *ab,
                      void *stream);
/* One batched call (orbg_batched.cu); buffers on the device.  code0: host
 * copy of code 0's descriptor, or NULL; with code_id == NULL every block is
 * code 0 and the kernels take it from their parameters. */
/* The decoder variants of a code set: keys per lane K (n <= 32, 64, 128,
 * 256: 1, 2, 4, 8) and syndrome words W (1, 2, or 4 for 3-4 words), in the
 * order a mixed-code call's phase 1 takes them.  The device table d_bucket
 * gives each code its sort bucket, numbered so that the codes of one
 * variant hold consecutive buckets [blo, bhi); bucket ncodes collects ids
 * outside the set and belongs to the last variant. */
#define ORBG_MAX_VARIANTS 12
struct OrbgVariants {
    int n;
    int k[ORBG_MAX_VARIANTS], w[ORBG_MAX_VARIANTS];
    int blo[ORBG_MAX_VARIANTS], bhi[ORBG_MAX_VARIANTS];
    const int32_t *d_bucket; /* [ncodes] */
};
struct OrbgBatchedArgs {
    const OrbgDeviceCode *d_codes;
    const OrbgDeviceCode *code0;
    int ncodes, n_max, w32_max;
    OrbgVariants var;            /* the set's decoder variants (mixed-code calls) */
    int has_stride;              /* a code of the set has strided pair runs (kind 2) */
    const int32_t *code_id;
    const int64_t *llr_off;
    const float *llr;
    int64_t B;
    uint32_t cap, budget;
    uint8_t *cw;
    const int64_t *cw_off;
    uint32_t *q;
    uint8_t *ab;
    unsigned long long *scratch;
    int warps_per_cta, ctas_per_sm, grab, heavy_warps;
    uint32_t ntrip_max, x3w_max;
    void *stream;
    /* Staged calls (the host-buffer pipeline: phase 1 chunk by chunk as the
     * LLRs arrive, then one phase 2 over every chunk's open blocks).
     * stage 0: both phases; 1: phase 1 of one chunk, blocks scratch_base ..
     * scratch_base + B - 1 of the whole batch (the pointers already point at
     * the chunk), first_chunk clears the scratch; 2: phase 2 only, over the
     * whole batch (pointers and B of the whole batch).  scratch_B: the
     * batch's block count the scratch is laid out for (0 = B).  slot (stage
     * 1): the queue and code counts this launch uses (0 or 1); a launch
     * resets its slot's unless it clears the whole scratch. */
    int stage;
    int slot;
    int first_chunk;
    int64_t scratch_base;
    int64_t scratch_B;
};
int orbg_launch_batched(const OrbgBatchedArgs &args);
/* orbg_batched_inst.cu, one per (keys per lane K, syndrome words W): both
 * phases, and phase 1 of that decoder variant alone over sort buckets
 * [blo, bhi) (blo < 0: every block) on `queue` (pdl: the launch may begin
 * while the previous one in the stream finishes). */
struct OrbgScratch;
#define ORBG_DECLARE_BATCHED(K, W)                                                   \
    int orbg_launch_batched_k##K##w##W(const OrbgBatchedArgs &a);                    \
    int orbg_launch_exact_k##K##w##W(const OrbgBatchedArgs &a, const OrbgScratch &s, \
                                     unsigned long long *queue, int blo, int bhi, int pdl, \
                                     int stride);
ORBG_DECLARE_BATCHED(1, 1) ORBG_DECLARE_BATCHED(1, 2) ORBG_DECLARE_BATCHED(1, 4)
ORBG_DECLARE_BATCHED(2, 1) ORBG_DECLARE_BATCHED(2, 2) ORBG_DECLARE_BATCHED(2, 4)
ORBG_DECLARE_BATCHED(4, 1) ORBG_DECLARE_BATCHED(4, 2) ORBG_DECLARE_BATCHED(4, 4)
ORBG_DECLARE_BATCHED(8, 1) ORBG_DECLARE_BATCHED(8, 2) ORBG_DECLARE_BATCHED(8, 4)
#undef ORBG_DECLARE_BATCHED
/* Device scratch of one batched call over B blocks of a set of ncodes codes,
 * in this order: ORBG_BATCHED_COUNTERS 64-bit counters (0: queue head of
 * slot 0, 1: open-block count, 2: phase-2 cursor, 3: queue head of slot 1,
 * 8 + ORBG_MAX_VARIANTS s + v: the queue head of variant v in slot s); for
 * each of two slots, per-bucket block counts and fill cursors (ncodes + 1
 * uint32 each, the last for code ids outside the set); the list of open
 * blocks (B uint64); the blocks in phase 1's order, grouped by decoder
 * variant (B uint32).  The counters, counts and cursors start at zero.  A
 * phase-1 launch uses one slot's queues and counts, so two launches over
 * different chunks of a batch (the host-buffer pipeline's two decode
 * streams) can run at the same time. */
#define ORBG_BATCHED_COUNTERS (8 + 2 * ORBG_MAX_VARIANTS)
#define ORBG_MAX_CODES 1024      /* codes in one set */
size_t orbg_batched_scratch_bytes(int64_t B, int ncodes);
/* Then, 16-byte aligned, up to ORBG_HANDOVER_MAX handover records: for the
 * i-th block phase 1 leaves open, its reliability order (256 bytes: the
 * received index of each sorted position) and its starting syndrome (16
 * bytes), so that phase 2 need not sort the block again. */
#define ORBG_HANDOVER_MAX 32768
#define ORBG_HANDOVER_BYTES 272
struct OrbgScratch {
    unsigned long long *counters;
    uint32_t *count, *cursor;     /* slot 0's; slot 1's follow at + 2 (ncodes + 1) */
    unsigned long long *heavy;
    uint32_t *perm;
    unsigned char *hand;          /* handover records */
    uint32_t hand_cap;            /* records available */
    size_t zero_bytes;            /* bytes from the start that must be zero */
};
inline OrbgScratch orbg_scratch_layout(void *base, int64_t B, int ncodes)
{
    OrbgScratch s;
    unsigned char *p = (unsigned char *)base;
    const size_t nc = (size_t)(ncodes > 0 ? ncodes : 0) + 1;
    const size_t b = (size_t)(B > 0 ? B : 0);
    s.counters = (unsigned long long *)p;
    s.count = (uint32_t *)(p + 8 * ORBG_BATCHED_COUNTERS);
    s.cursor = s.count + nc;
    s.zero_bytes = 8 * ORBG_BATCHED_COUNTERS + 16 * nc;
    s.heavy = (unsigned long long *)(p + s.zero_bytes);
    s.perm = (uint32_t *)(s.heavy + b);
    const size_t hoff = ((size_t)((unsigned char *)(s.perm + b) - p) + 15) & ~(size_t)15;
    s.hand = p + hoff;
    s.hand_cap = (uint32_t)(b < ORBG_HANDOVER_MAX ? b : ORBG_HANDOVER_MAX);
    return s;
}
/* Order the blocks of a mixed-code call by the bucket of their code
 * (bucket[code id]; ids outside the set go to bucket ncodes): a counting
 * sort into perm, so that each decoder variant's blocks hold consecutive
 * slots and one launch per variant decodes them; returns a cudaError_t. */
int orbg_launch_code_sort(const int32_t *code_id, const int32_t *bucket, int64_t B, int ncodes,
                          const OrbgScratch &s, void *stream);
/* orbg_launch_exact_k*w* for keys per lane K and syndrome words W. */
int orbg_launch_exact(int K, int W, const OrbgBatchedArgs &a, const OrbgScratch &s,
                      unsigned long long *queue, int blo, int bhi, int pdl, int stride);
/* Outputs of the blocks phase 2 decoded, gathered after the last launch of a
 * batch whose other results already went to the host.  At `out` (memory the
 * device writes, here host-mapped) the heavy list's length (uint64).  With
 * to_cw, to_q, to_ab (the caller's output buffers, device-writable host
 * memory laid out as cw, q, ab) every listed block's outputs are written
 * there in place; otherwise `out` also takes, for the list's first `cap`
 * entries, the block index and query count (uint32 pairs), the flag byte,
 * and from orbg_gather_cw_at(cap) the codeword bytes at a stride of n_max.
 * code_id / cw_off NULL: one code of length n0, dense codewords.  Returns a
 * cudaError_t. */
#ifdef __CUDACC__
__host__ __device__
#endif
inline size_t orbg_gather_cw_at(uint32_t cap) { return (16 + 9 * (size_t)cap + 15) & ~(size_t)15; }
inline size_t orbg_gather_bytes(uint32_t cap, int n_max)
{
    return orbg_gather_cw_at(cap) + (size_t)cap * (size_t)n_max;
}
int orbg_launch_heavy_gather(const OrbgDeviceCode *d_codes, const int32_t *code_id, int n0,
                             const int64_t *cw_off, const uint8_t *cw, const uint32_t *q,
                             const uint8_t *ab, const OrbgScratch &s, unsigned char *out,
                             uint32_t cap, int n_max, uint8_t *to_cw, uint32_t *to_q,
                             uint8_t *to_ab, void *stream);
int orbg_grid_for(const void *kern, int threads, size_t smem, int ctas_per_sm, int *grid_out);

/* A named range on the NVTX timeline for the span of a scope (header-only
 * NVTX v3: a no-op unless a profiler such as Nsight Systems is attached). */
#include <nvtx3/nvToolsExt.h>
struct OrbgRange {
    explicit OrbgRange(const char *name) { nvtxRangePushA(name); }
    ~OrbgRange() { nvtxRangePop(); }
    OrbgRange(const OrbgRange &) = delete;
    OrbgRange &operator=(const OrbgRange &) = delete;
};

/* What a launch needs of a code set (orbg_api.cpp owns the struct). */
#include "../../include/orbg.h"
struct OrbgSetView {
    const OrbgDeviceCode *d_codes;
    OrbgDeviceCode code0;        /* host copy of code 0's descriptor */
    int ncodes, n_max, w32_max;
    OrbgVariants var;
    int has_stride;
    uint32_t ntrip_max;
    uint32_t x3w_max;
    uint32_t cap_min;
    orbg_tuning tuning;
};
int orbg_codeset_view(const orbg_codeset *set, OrbgSetView *out);
int orbg_codeset_lengths(const orbg_codeset *set, std::vector<int> *n_of);
/* Records a cudaError_t for orbg_last_cuda_error; returns the orbg status. */
int orbg_note_cuda_error(int cuda_error);
/* Fitted one-line decoding (orbg_fit.cu): over B one-line model records,
 * present[J_0 + 1] = 1 for every J_0 met, and cid[b] = lut[J_0 + 1]; NaN
 * blocks count as J_0 = 0 and J_0 is held within [-1, top].  present and
 * lut hold top + 2 entries.  Return a cudaError_t. */
int orbg_fit_mark_lines(const int32_t *models, int64_t B, int32_t top, uint8_t *present,
                        void *stream);
/* orbg_fit_models' launch without its argument checks (B >= 1, 1 <= n <=
 * 256, 1 <= lines <= 8, device buffers); returns a cudaError_t. */
int orbg_fit_launch(const float *llr, int64_t B, int n, int lines, int divisible,
                    int32_t *models, void *stream);
int orbg_fit_map_lines(const int32_t *models, int64_t B, int32_t top, const int32_t *lut,
                       int32_t *cid, void *stream);
/* The per-block fitted decoder (orbg_fitted_search_inst.cu, one per keys per
 * lane K): every block fitted (Sec. III-E) and searched in its own order, in
 * three launches; scratch: orbg_fitsearch_scratch_bytes(B) device bytes
 * (counters, the list of blocks the second launch searches, the list of
 * those it leaves to the third, and for each open block a handover record
 * of ORBG_FIT_HAND_BYTES: order, model, starting syndrome).
 * Return a cudaError_t value. */
#define ORBG_FIT_HAND_BYTES 384
inline size_t orbg_fitsearch_scratch_bytes(int64_t B)
{
    const size_t b = (size_t)(B > 0 ? B : 0);
    return 64 + 2 * ((4 * b + 15) & ~(size_t)15) + (size_t)ORBG_FIT_HAND_BYTES * b;
}
#define ORBG_DECLARE_FITSEARCH(K)                                                         \
    int orbg_launch_fitsearch_k##K(const OrbgDeviceCode &code, const float *llr, int64_t B, \
                                   uint32_t cap, int lines, int divisible, uint8_t *cw,     \
                                   uint32_t *q, uint8_t *ab, int32_t *models,               \
                                   unsigned char *scratch, void *stream);
ORBG_DECLARE_FITSEARCH(1) ORBG_DECLARE_FITSEARCH(2) ORBG_DECLARE_FITSEARCH(4)
ORBG_DECLARE_FITSEARCH(8)
#undef ORBG_DECLARE_FITSEARCH
int orbg_launch_int_probe(double *lanes_per_clk_per_sm);
int orbg_launch_smem_probe(double *bytes_per_clk_per_sm);
#endif

#endif /* ORBG_INTERNAL_H */
