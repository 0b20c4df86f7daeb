/*
 * orbg.h -- C ABI of the GB300 ORBGRAND decoder.
 *
 * Basic ORBGRAND (Duffy, An, Medard, arXiv 2202.13951): for each received
 * block, sort the bit positions by reliability |LLR| (Sec. III-A), query
 * noise patterns z in increasing logistic weight w_L(z) = sum_i i z_i
 * (Eq. lw, Eq. fractionation, Eq. intpart2), and return the first y (+) z
 * that is a code-book member, i.e. whose syndrome H (y (+) z) is zero
 * (Algorithm 1; membership of a linear code by a matrix multiply and
 * compare, Sec. I), or abandon after the query cap (Sec. IV-A).
 * Full ORBGRAND (Sec. III-D, III-E) replaces the logistic weight by the
 * reliability weight of a one-line or piece-wise linear model of the
 * ordered reliabilities: orbg_load_code_line and orbg_load_code_model load
 * a code for a fixed line or model, orbg_fit_models fits each block's
 * model on the device, and orbg_fitted_* decodes every block in the order
 * of its own fitted line.
 *
 * Query order fixed by this library where the paper leaves ties arbitrary:
 *   - bits with equal |LLR| are ordered by their received index;
 *   - within one logistic weight W, patterns of lower Hamming weight come
 *     first; within (W, w), flipped positions in lexicographic order (the
 *     order the Landslide generator, Algorithm 2, produces);
 *   - the zero pattern is query 1; hard decision y_i = 1 iff LLR_i > 0
 *     (+0 and -0 give 0); +-Inf is allowed (most reliable).
 *
 * Conventions for every function:
 *   - returns ORBG_OK (0) or a negative orbg_status; nothing is thrown;
 *   - on error, output buffers are unspecified;
 *   - abandonment is a per-block result, not an error;
 *   - buffers are owned by the caller.  Each may be a device pointer or a
 *     host pointer (detected per pointer), except where a function asks
 *     for device memory only (orbg_fit_models, orbg_fitted_decode).  With
 *     all buffers on the device the call is asynchronous on `cuda_stream`
 *     (NULL = the legacy default stream) and the buffers must stay valid
 *     until the stream reaches the call's end.  With any host buffer the
 *     library stages the data through device memory, copies results back
 *     and synchronises the stream before returning;
 *   - telling host from device pointers (cudaPointerGetAttributes) never
 *     clears a CUDA error that the caller's earlier work left pending.
 */
#ifndef ORBG_H
#define ORBG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ORBG_API __attribute__((visibility("default")))
#else
#define ORBG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum orbg_status {
    ORBG_OK = 0,
    ORBG_EINVAL = -1,   /* null pointer, bad size, entry not 0/1, bad kind */
    ORBG_ERANK = -2,    /* matrix rank differs from what n, k require */
    ORBG_ELIMIT = -3,   /* n > 256, n-k > 128, or cap beyond the handle's reserve */
    ORBG_ENAN = -4,     /* a NaN LLR was seen (reported by host-buffer calls) */
    ORBG_ENOMEM = -5,   /* host or device allocation failed */
    ORBG_ECUDA = -6,    /* a CUDA call failed; see orbg_last_cuda_error() */
    ORBG_ETIMEOUT = -7  /* a bounded device wait ran out */
} orbg_status;

enum { ORBG_MAT_H = 0, ORBG_MAT_G = 1 };

/* Limits of this version. */
#define ORBG_MAX_N 256
#define ORBG_MAX_R 128
#define ORBG_MAX_QUERY_CAP (1u << 25)
#define ORBG_DEFAULT_QUERY_CAP (1u << 20)

/* Per-block values written to abandoned[b]. */
#define ORBG_BLOCK_DECODED 0
#define ORBG_BLOCK_ABANDONED 1
#define ORBG_BLOCK_NAN 2       /* block had a NaN LLR: codeword = hard decision, queries = 0 */

typedef struct orbg_code orbg_code;       /* opaque, library-owned */
typedef struct orbg_codeset orbg_codeset; /* opaque, library-owned */

/*
 * Load a binary linear code of length n and dimension k.
 *   mat   : host memory, row-major bytes, each 0 or 1; copied.
 *           kind ORBG_MAT_H: (n-k) x n parity-check matrix, rank n-k.
 *           kind ORBG_MAT_G: k x n generator matrix, rank k; the library
 *           derives a parity-check matrix spanning its null space.
 *   n     : 1..256;  n-k : 1..128.
 *   max_query_cap : the largest query cap later decode calls may use
 *           (0 = ORBG_DEFAULT_QUERY_CAP, at most ORBG_MAX_QUERY_CAP).  The
 *           handle holds the query-order tables up to that depth.
 *   out   : receives the handle.  It owns device copies of H and of the
 *           tables on the device current at load time, until
 *           orbg_free_code.  The load synchronises that device.
 * Errors: EINVAL, ERANK, ELIMIT, ENOMEM, ECUDA.
 * Paper: Algorithm 1's code-book membership function (Sec. I: matrix
 * multiply and compare for a linear code).
 */
ORBG_API int orbg_load_code(const uint8_t *mat, int kind, int n, int k,
                   uint32_t max_query_cap, orbg_code **out);

/*
 * One-line full ORBGRAND (Sec. III-D, Eq. relest_seg with one segment):
 * as orbg_load_code, but the handle's query order sorts noise patterns by
 * increasing reliability weight J0 w_H + beta w_L, the sorted position j
 * counting J0 + beta j (Eq. wu_i), ties as for basic ORBGRAND (Hamming
 * weight ascending, then lexicographic).  J0: 0..1024, beta: 1..1024;
 * J0 = 0, beta = 1 is orbg_load_code.  Every decode entry point decodes
 * in the handle's order.  Errors as orbg_load_code; EINVAL for J0 or beta
 * out of range; ELIMIT when the order up to max_query_cap reaches a
 * logistic weight above 255 (a large J0 at a large cap; the same line as a
 * one-segment orbg_load_code_model has no such limit).
 */
ORBG_API int orbg_load_code_line(const uint8_t *mat, int kind, int n, int k,
                                 uint32_t max_query_cap, int32_t J0, int32_t beta,
                                 orbg_code **out);

/*
 * m-segment full ORBGRAND (Sec. III-D, Eq. relest_seg): as orbg_load_code,
 * but the handle's query order sorts noise patterns by increasing
 * reliability weight under a piece-wise linear model of m segments
 * (1..8): with I_0 = 0, I_m = n and the anchors I_1 < ... < I_{m-1}
 * (host array `anchors`, m - 1 entries, inside 1..n-1), sorted position j
 * of segment i, I_{i-1} < j <= I_i, counts J_{i-1} + beta_i (j - I_{i-1}).
 * J: host array J_0..J_{m-1}; beta: host array beta_1..beta_m.  beta_i:
 * 1..2^20; J_{i-1}: -beta_i..2^20, so that no position counts below 0
 * (Eq. quant gives J_0 = -beta_1 when the least reliable bit rounds to
 * zero).  Ties: Hamming weight ascending, then positions lexicographically;
 * the empty pattern is query 1.  The orders of orbg_load_code and
 * orbg_load_code_line are the one-segment cases (J_0 = J0, beta_1 =
 * beta), built here without triple runs.  Every decode entry point decodes
 * in the handle's order.  Arrays are read during the call only.  Errors as
 * orbg_load_code; EINVAL for a model out of range; ELIMIT when the order
 * up to max_query_cap needs a position above 255 in a pattern's leading
 * positions or more than 22 flipped positions.
 */
ORBG_API int orbg_load_code_model(const uint8_t *mat, int kind, int n, int k,
                                  uint32_t max_query_cap, int m, const int32_t *anchors,
                                  const int32_t *J, const int32_t *beta, orbg_code **out);

/* Release a handle (NULL is allowed).  Not stream-ordered: no decode call
 * using it may still be in flight. */
ORBG_API int orbg_free_code(orbg_code *code);

/* Copy of the handle's parity-check matrix, (n-k) x n row-major bytes, and
 * its sizes; any output pointer may be NULL.  Host only, no CUDA call. */
ORBG_API int orbg_code_info(const orbg_code *code, int *n, int *k,
                   uint32_t *max_query_cap, uint8_t *H_out);

/*
 * Plain form: one launch, one warp per block, blocks in a static grid.
 *   llr       : [B][n] FP32 LLRs, row-major, LLR = log f(Y|1)/f(Y|0).
 *   B         : number of blocks (0 is a no-op).
 *   query_cap : 1..max_query_cap of the handle; abandon after this many
 *               queries (Sec. IV-A).  A hit at exactly query_cap decodes.
 *   codeword  : [B][n] bytes 0/1: y (+) z* for the first hit z*, or the hard
 *               decision y if abandoned.
 *   queries   : [B] the 1-based index of the hit in the query order, or
 *               query_cap if abandoned (0 for a NaN block).
 *   abandoned : [B] ORBG_BLOCK_DECODED / _ABANDONED / _NAN.
 * Errors: EINVAL, ELIMIT, ENOMEM, ECUDA; ENAN only for host-buffer calls
 * (device-buffer calls report NaN blocks through abandoned[b] alone).
 * Paper: Algorithm 1 with the basic ORBGRAND generator (Sec. III-B).
 */
ORBG_API int orbg_decode(const orbg_code *code, const float *llr, int64_t B,
                uint32_t query_cap, uint8_t *codeword, uint32_t *queries,
                uint8_t *abandoned, void *cuda_stream);

/*
 * A set of loaded codes that one batched launch may mix.  The codes must
 * stay loaded while the set is used; the set holds a device copy of their
 * descriptors (made synchronously here).  ncodes: 1..1024.
 */
ORBG_API int orbg_codeset_create(const orbg_code *const *codes, int ncodes,
                        orbg_codeset **out);
ORBG_API int orbg_codeset_free(orbg_codeset *set);

/*
 * Batched form: two persistent phases.  In the first (one launch, or one per
 * decoder variant of a code set), warps pull blocks from an atomic work
 * queue and decode each alone up to a query budget; in the second (one
 * launch), every CTA takes one still-open block at a time and searches it
 * with all its warps.  Blocks with very different query counts, and blocks
 * of different codes, balance across the GPU.
 *   code_id    : [B] index into the set per block, or NULL (all code 0).
 *   llr_offset : [B] element offset of block b in llr, or NULL
 *                (dense: b * n of code 0).
 *   cw_offset  : [B] byte offset of block b in codeword, or NULL (dense).
 *   Other arguments as orbg_decode; query_cap must be within every code's
 *   max_query_cap.
 * The call uses 287 + 16 ncodes + 12 B + 272 min(B, 32768) bytes of
 * stream-ordered device scratch (queue counters, per-code block counts, the
 * list of still-open blocks, the blocks' order grouped by decoder variant,
 * and the reliability order of up to 32,768 still-open blocks, which the
 * second launch reuses), allocated on cuda_stream from the library's pool
 * (orbg_pool_trim).  With code_id given, the first launch is one launch per
 * decoder variant among the set's codes (length class n <= 32, 64, 128,
 * 256 and syndrome width 1, 2 or 3-4 words), each of that variant alone;
 * with several variants the blocks are first grouped by variant on the
 * device, and each variant's launch may begin while the previous one
 * finishes (programmatic dependent launch).  A code id outside the set
 * gives its block queries 0 and flag ORBG_BLOCK_NAN with its codeword
 * bytes untouched (with host layout arrays and offsets: ORBG_EINVAL).
 * Host buffers (staged through stream-ordered device copies): a call with
 * every buffer on the host, B >= 131072 and a layout that places the
 * blocks in order without overlap (dense, or offsets that never go back)
 * is cut into up to eight chunks on four library-owned streams (created
 * on the set's first such call): each chunk's copy in, then the first
 * launch over it on one of two decode streams in turn (so a chunk's launch
 * can fill what the previous one leaves idle), then its results out; the
 * second launch runs once over the blocks every chunk left open, and their
 * results are written over the copies (by the device straight into page-
 * locked output buffers, else through a host-mapped staging buffer).  One
 * such call runs at a time per set.  cuda_stream waits for the streams and
 * is synchronised before the call returns, as for any host-buffer call.
 * With host buffers and offsets, codeword bytes between blocks are
 * unspecified afterwards.
 * Results are identical to orbg_decode's block by block.
 * Paper: Algorithm 1 per block; the batching is this library's.
 */
ORBG_API int orbg_decode_batched(const orbg_codeset *set, const int32_t *code_id,
                        const int64_t *llr_offset, const float *llr,
                        int64_t B, uint32_t query_cap, uint8_t *codeword,
                        const int64_t *cw_offset, uint32_t *queries,
                        uint8_t *abandoned, void *cuda_stream);

/*
 * Batched decode that allocates nothing (the paper has no counterpart; this
 * is a deployment variant of orbg_decode_batched).
 *
 * For callers that must not allocate device memory while decoding, e.g. a
 * receiver that reserves all its GPU memory at start-up and treats a later
 * allocation as a failure, or code that cannot let an allocation block
 * behind other device work inside its latency budget.  orbg_decode_batched
 * allocates its scratch on the stream on every call; this variant uses a
 * fixed array compiled into the library instead, and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   - Same arguments, layout and results as orbg_decode_batched, except
 *     that every buffer must be device memory (host buffers would need
 *     staging): EINVAL otherwise.
 *   - B <= ORBG_NOALLOC_MAX_BLOCKS (524,288), else ELIMIT.  Larger batches
 *     can be split into several calls.
 *   - The array is 12 * ORBG_NOALLOC_MAX_BLOCKS + 16,672 + 272 * 32,768
 *     bytes (14.5 MiB + 16,672 B) of device memory per GPU that loads the
 *     library, held until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (with that device current) and keeps it; make that first call before
 *     any stream capture.  The kept address belongs to the device's primary
 *     context (the runtime API's): it is invalid after cudaDeviceReset and
 *     in a context made with the driver API on that device, where this
 *     entry point must not be called.
 *   - All calls on a device share the one array; the counters that must
 *     start at zero are cleared on cuda_stream at the start of each call.
 *     Calls whose work overlaps on the GPU (other streams, or other host
 *     threads) race on the array and give wrong results: serialise them.
 */
#define ORBG_NOALLOC_MAX_BLOCKS (1 << 19)
ORBG_API int orbg_decode_batched_noalloc(const orbg_codeset *set,
                                         const int32_t *code_id,
                                         const int64_t *llr_offset,
                                         const float *llr, int64_t B,
                                         uint32_t query_cap, uint8_t *codeword,
                                         const int64_t *cw_offset,
                                         uint32_t *queries, uint8_t *abandoned,
                                         void *cuda_stream);

/*
 * Tuning of the batched form, per code set (the autotuner writes these):
 *   warps_per_cta   phase 1: warps per CTA, one block per warp (1..16; 0 = 8)
 *   ctas_per_sm     phase 1: resident CTAs per SM (0 = as many as fit)
 *   blocks_per_grab phase 1: blocks a warp takes per work-queue atomic
 *                   (1..1024; 0 = 4)
 *   warp_budget     phase 1: queries of a block's order a single warp walks
 *                   before handing the block to phase 2 (0 = 16384).  A warp
 *                   also hands a block on, whatever the budget, where its
 *                   walk first needs triple sums past its own triple table
 *                   (query 14,798 of basic ORBGRAND), so budgets above that
 *                   act alike; phase 2 runs in every call
 *   heavy_warps     phase 2: warps per CTA sharing one block (1..16; 0 = 8)
 * None of these change any result.
 */
typedef struct orbg_tuning {
    int warps_per_cta;
    int ctas_per_sm;
    int blocks_per_grab;
    uint32_t warp_budget;
    int heavy_warps;
} orbg_tuning;

/* t = NULL restores the defaults.  Not stream-ordered: set it while no
 * batched call on this set is being enqueued. */
ORBG_API int orbg_codeset_set_tuning(orbg_codeset *set, const orbg_tuning *t);
ORBG_API int orbg_codeset_get_tuning(const orbg_codeset *set, orbg_tuning *t);

/*
 * Serving: continuous batching of decode requests over a code set.
 *
 * orbg_server_create starts a dispatcher thread on the current device with
 * a device memory pool and a pinned host pool of mem_budget_bytes each
 * (0 = 1 GiB) and `streams` CUDA streams (0 = 4).  orbg_server_submit
 * queues a request (its LLRs are copied, so the caller's buffer is free on
 * return).  The dispatcher packs waiting requests, oldest first, into the
 * next batch while the batch's footprint -- LLRs, outputs, per-block layout
 * arrays and kernel scratch -- still fits the free part of both pools
 * (admission by memory footprint), and runs each batch as one mixed-code
 * batched decode on a free stream; batches on different streams overlap,
 * and requests that arrive while batches run join the next batch.  The
 * code tables stay on the device.  Results are the same, block for block,
 * as orbg_decode_batched would give for the request alone.
 *   query_cap        : per-block cap for every request (<= each code's reserve)
 *   max_batch_blocks : largest batch in blocks (0 = 2^20)
 *   submit           : code_index into the set; B >= 1 blocks of that
 *                      code's n LLRs, row-major host memory; request_id is
 *                      the caller's (must not be in use).  ELIMIT if the
 *                      request alone could never fit the pools.
 *   poll             : waits up to timeout_us for finished requests and
 *                      writes up to max_ids of their ids; returns the
 *                      count (or a negative status).  Each id is reported
 *                      once.
 *   fetch            : copies a finished request's codeword [B][n], queries
 *                      [B], abandoned [B] (any pointer may be NULL) to host
 *                      memory, with its latency from submit to completion
 *                      in seconds, and forgets the request.
 *   cancel           : withdraws a request: it is never reported by poll
 *                      and fetch no longer finds it.  One still waiting is
 *                      removed; one already in a batch still runs on the
 *                      device (its blocks share the batch's launch) and its
 *                      results are dropped when the batch finishes; one
 *                      finished but not yet fetched is discarded.  EINVAL
 *                      if the server knows no such id (never submitted,
 *                      already fetched or cancelled).
 *   destroy          : waits for submitted work, then frees everything.
 * The server's own extension, not the paper's (the paper decodes one block
 * at a time, Algorithm 1).
 */
typedef struct orbg_server orbg_server;
typedef struct orbg_server_stats {
    uint64_t submitted, completed;
    uint64_t blocks_submitted, blocks_done;
    uint64_t batches, max_batch_blocks, max_inflight_batches;
    uint64_t pending, inflight_batches;
    uint64_t cancelled;  /* requests withdrawn by orbg_server_cancel */
} orbg_server_stats;

ORBG_API int orbg_server_create(const orbg_codeset *set, size_t mem_budget_bytes,
                                uint32_t query_cap, int streams,
                                int64_t max_batch_blocks, orbg_server **out);
ORBG_API int orbg_server_submit(orbg_server *srv, uint64_t request_id,
                                int code_index, const float *llr, int64_t B);
ORBG_API int orbg_server_poll(orbg_server *srv, uint64_t *ids, int max_ids,
                              int timeout_us);
ORBG_API int orbg_server_fetch(orbg_server *srv, uint64_t request_id,
                               uint8_t *codeword, uint32_t *queries,
                               uint8_t *abandoned, double *latency_s);
ORBG_API int orbg_server_cancel(orbg_server *srv, uint64_t request_id);
ORBG_API int orbg_server_stats_get(orbg_server *srv, orbg_server_stats *out);
ORBG_API int orbg_server_destroy(orbg_server *srv);

/*
 * Trace replay on a server, for measuring it: request i (code[i], B[i]
 * blocks at element llr_off[i] of llr_all) is submitted arrival_s[i]
 * seconds after the call starts, from a second thread, while this thread
 * polls and fetches; outputs go to cw_all at element llr_off[i] and to
 * q_all / ab_all at block blk_off[i]; latency_s[i] is its latency and
 * *wall_s the replay's duration.  Host memory throughout.
 */
ORBG_API int orbg_server_replay(orbg_server *srv, int64_t nreq,
                                const double *arrival_s, const int32_t *code,
                                const int64_t *B, const int64_t *llr_off,
                                const int64_t *blk_off, const float *llr_all,
                                uint8_t *cw_all, uint32_t *q_all,
                                uint8_t *ab_all, double *latency_s,
                                double *wall_s);

/*
 * Autotuner for the batched form: times orbg_decode_batched on the given
 * sample (device buffers, same arguments as orbg_decode_batched) under
 * candidate tunings -- coordinate descent over warp_budget, heavy_warps,
 * blocks_per_grab, warps_per_cta and ctas_per_sm, repeated (at most three
 * passes) while a pass changes the tuning, each candidate the median of
 * `reps` timed runs (CUDA events on cuda_stream, after one warm-up) --
 * keeps the fastest on the set and writes it to *best (may be NULL).
 * Synchronises the stream.  The outputs are overwritten by every trial and
 * hold the sample's (tuning-independent) results at the end.  The
 * library's own addition; the paper has no counterpart.
 */
ORBG_API int orbg_codeset_autotune(orbg_codeset *set, const int32_t *code_id,
                                   const int64_t *llr_offset, const float *llr,
                                   int64_t B, uint32_t query_cap,
                                   uint8_t *codeword, const int64_t *cw_offset,
                                   uint32_t *queries, uint8_t *abandoned,
                                   int reps, void *cuda_stream,
                                   orbg_tuning *best);

/*
 * Roofline probe: issue rate of independent 32-bit 3-input logic ops
 * (lop3.b32, the instruction a syndrome XOR compiles to) per SM per clock,
 * in lanes (threads x instructions), measured with clock64 on every SM of
 * the current device.  Synchronous; allocates and frees a small buffer.
 */
ORBG_API int orbg_probe_int_lanes(double *lanes_per_clk_per_sm);

/*
 * Roofline probe for shared memory: bytes per SM per clock that 64-bit
 * shared loads deliver (a warp reads 32 consecutive 8-byte words, so no
 * bank conflicts), measured with clock64 on every SM of the current
 * device.  The column and triple-table reads of the search are shared
 * loads.  Synchronous; allocates and frees a small buffer.  The library's
 * own addition; the paper has no counterpart.
 */
ORBG_API int orbg_probe_smem_bytes(double *bytes_per_clk_per_sm);

/*
 * The query order this library decodes in, for inspection and tests: the
 * first `count` noise patterns for length n (1..256), expanded from the
 * same tables the kernels read (table 0: the one-warp-per-block table;
 * table 1: the CTA table of the batched form's second phase; both hold
 * the same order; table 2: the flat table of the leading patterns both
 * start with, which stops after at most 256 patterns).  out: host memory, [count][n+1] int32 rows
 * holding w, then the w flipped positions (1-based, in increasing
 * reliability order, ascending), then zeros.  Returns the number of rows
 * written (fewer than count once the 2^n patterns run out), or a negative
 * status.  Host only, no CUDA call.  Paper: Sec. III-B (Eq. lw, Eq.
 * fractionation, Eq. intpart), ties as read at the top of this header.
 */
ORBG_API int64_t orbg_query_order(int n, uint32_t count, int table,
                                  int32_t *out);

/* The same for the one-line order of orbg_load_code_line (Sec. III-D). */
ORBG_API int64_t orbg_query_order_line(int n, uint32_t count, int table, int32_t J0,
                                       int32_t beta, int32_t *out);

/* The same for the m-segment order of orbg_load_code_model (Sec. III-D,
 * Eq. relest_seg); the model's arguments as there.  Tables 0 and 1 are the
 * same run list. */
ORBG_API int64_t orbg_query_order_model(int n, uint32_t count, int table, int m,
                                        const int32_t *anchors, const int32_t *J,
                                        const int32_t *beta, int32_t *out);

/*
 * Per-block piece-wise linear fitting and quantisation (Sec. III-E, Eq. Q,
 * Eq. quant) on the device: for each of B blocks of n LLRs (llr, [B][n]
 * FP32, device memory) the ordered reliability curve L_1 <= ... <= L_n of
 * |LLR| is fitted with up to `lines` (1..8) lines and quantised into the
 * model of orbg_load_code_model.  Anchors start at indices 1 and floor(n/2);
 * each further anchor splits the first (edge) interval at its largest
 * vertical gap between chord and curve (the smaller index on equal gaps),
 * stopping early when there is none; the centre line covers the rest.
 * Q = the smallest segment slope; beta_i = [s_i / Q], J_0 = [L_1 / Q] -
 * beta_1, J_i = [L_{I_i} / Q], [x] rounding half away from zero;
 * divisible != 0 makes each J_{i-1} a multiple of beta_i ([J/beta] beta).
 * n < 4, a flat stretch (Q <= 0) or a quantised ratio above 2^24 gives the
 * basic model (m = 1, J_0 = 0, beta_1 = 1).  models: device memory,
 * [B][ORBG_FIT_STRIDE] int32 per block: m, then the anchors I_1..I_7 (m - 1
 * used), then J_0..J_7 (m used), then beta_1..beta_8 (m used), unused
 * entries 0; m = 0 marks a block with a NaN LLR.  Stream-ordered on
 * cuda_stream.  Errors: EINVAL (sizes, NULL or host pointers), ECUDA.
 */
#define ORBG_FIT_STRIDE 24
ORBG_API int orbg_fit_models(const float *llr, int64_t B, int n, int lines, int divisible,
                             int32_t *models, void *cuda_stream);

/*
 * Full ORBGRAND with one line fitted per block (Sec. III-E with one line,
 * then the order of Sec. III-D): each block is decoded in the one-line
 * order of its own fit (beta = 1, J_0 = [L_1 / Q] - 1, Q the slope from
 * L_1 to L_{floor(n/2)}), the paper's "1-line" variant.  The object keeps,
 * for the given code (not owned; it must outlive the object), one handle
 * per J_0 met so far (built on first use with the code's max_query_cap;
 * J_0 above n(n+1)/2, which orders by Hamming weight first, is held at
 * n(n+1)/2 + 1), and a code set over them.  divisible != 0 selects the
 * J-divisible quantisation (the same line when beta = 1).
 * orbg_fitted_decode: device buffers only -- llr [B][n] FP32, codeword
 * [B][n], queries [B], abandoned [B] as orbg_decode; models: NULL or a
 * device buffer [B][ORBG_FIT_STRIDE] that receives each block's fit
 * (orbg_fit_models).  It fits on cuda_stream, reads back which J_0s occur
 * (synchronising cuda_stream), and decodes all blocks in one batched call
 * with each block's own order; results equal the one-line decoder of each
 * block's line.  Errors: EINVAL (NULL or host buffers), ELIMIT
 * (query_cap above the code's max_query_cap, more than 1024 distinct
 * lines, or a line whose order puts position 256 of an n = 256 code within
 * the cap), ENOMEM, ECUDA.  One call at a time per object (serialised).
 * orbg_fitted_free releases the object and its handles (NULL is allowed);
 * like orbg_free_code it is not stream-ordered: no decode call on the
 * object may still be in flight.
 */
typedef struct orbg_fitted orbg_fitted;
ORBG_API int orbg_fitted_create(const orbg_code *code, int divisible, orbg_fitted **out);
ORBG_API int orbg_fitted_decode(orbg_fitted *f, const float *llr, int64_t B,
                                uint32_t query_cap, uint8_t *codeword, uint32_t *queries,
                                uint8_t *abandoned, int32_t *models, void *cuda_stream);
ORBG_API int orbg_fitted_free(orbg_fitted *f);

/*
 * Full ORBGRAND with a piece-wise linear model fitted to each block, any
 * number of lines (Sec. III-E, Eq. Q, Eq. quant, then the order of Sec.
 * III-D, Eq. relest_seg): the paper's 1- to 4-line variants of Sec. IV.
 * One launch; per block, on the device: the reliability sort, the fit of
 * orbg_fit_models (same anchors, same quantisation, plain or J-divisible),
 * and a search of the block's own order -- noise patterns by increasing
 * reliability weight (the sum over flipped sorted positions j of
 * J_{i-1} + beta_i (j - I_{i-1}), i the segment of j), ties by Hamming
 * weight and then positions lexicographically, the empty pattern first --
 * for the first code-book member within query_cap queries.  The results
 * equal, block by block, orbg_decode on a handle loaded with
 * orbg_load_code_model for that block's fitted model.
 *   code      : the code (its query-order tables are not used: any
 *               query_cap up to ORBG_MAX_QUERY_CAP is allowed).
 *   llr, B, codeword, queries, abandoned : as orbg_decode (host or device).
 *   lines     : 1..8;  divisible : 0 or 1 (Eq. quant's J-divisible form).
 *   models    : NULL, or [B][ORBG_FIT_STRIDE] int32 receiving each block's
 *               model record as orbg_fit_models writes it.
 *   abandoned[b] may also be ORBG_BLOCK_RANGE: the block's model would
 *   need reliability weights above 2^26 - 1 (far beyond any cap's reach
 *   for a model fitted to AWGN blocks) before its result is known, or its
 *   search exceeded its step guard; codeword = hard decision, queries = 0.
 * Device-buffer calls are asynchronous on cuda_stream and use 8 bytes of
 * stream-ordered device scratch (the work-queue counter).
 * Errors: EINVAL, ELIMIT (query_cap above ORBG_MAX_QUERY_CAP), ENOMEM,
 * ECUDA; ENAN only for host-buffer calls, as orbg_decode.
 */
#define ORBG_BLOCK_RANGE 3
ORBG_API int orbg_decode_fitted(const orbg_code *code, const float *llr, int64_t B,
                                uint32_t query_cap, int lines, int divisible,
                                uint8_t *codeword, uint32_t *queries, uint8_t *abandoned,
                                int32_t *models, void *cuda_stream);

/* Static description of a status code (never NULL). */
ORBG_API const char *orbg_status_string(int status);

/* The last CUDA error code seen by this thread (0 if none). */
ORBG_API int orbg_last_cuda_error(void);

/* Device memory of calls that stage host buffers, and their scratch, comes
 * from a stream-ordered pool the library keeps per device, which holds
 * freed memory for the next call instead of returning it at every
 * synchronisation (so a repeated large host-buffer batch does not map and
 * unmap its buffers each time).  This returns what the current device's
 * pool holds unused to the driver; memory of calls still in flight stays.
 * Returns ORBG_OK, or ORBG_ECUDA. */
ORBG_API int orbg_pool_trim(void);

/* Library version, major * 10000 + minor * 100 + patch: 200 for 0.2.0 (0.2 added
 * orbg_server_cancel and the cancelled count at the end of orbg_server_stats). */
ORBG_API int orbg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ORBG_H */
