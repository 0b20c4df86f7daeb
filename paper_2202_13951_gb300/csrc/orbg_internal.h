/*
 * orbg_internal.h -- data shared between the host side of the library and
 * its CUDA kernels.
 *
 * The query order (Sec. III-B: increasing logistic weight W; this library's
 * tie reading: Hamming weight w ascending, then positions lexicographic) is
 * held as a table of "runs".  A pattern of weight w >= 2 is a prefix
 * v_1 < ... < v_{w-2} followed by a pair a < b with a + b = S fixed by W;
 * for one prefix, the lexicographic order walks a upward, so the prefix's
 * patterns form one run of consecutive query indices.  Patterns of weight
 * 0 and 1 are runs of length one whose pair is the all-zero column twice.
 *
 * Runs are stored class by class ((W, w) ascending); inside a class they are
 * sorted by run length so that the 32 lanes of a warp, which take 32
 * consecutive runs, loop for about the same number of queries.  Every run
 * keeps its own first query index, so the decoder still reports the first
 * hit of the paper's order; group_floor[g] (the smallest first index over
 * runs of groups >= g) tells a warp when no later group can hold an earlier
 * hit.
 */
#ifndef ORBG_INTERNAL_H
#define ORBG_INTERNAL_H

#include <stdint.h>

#define ORBG_GROUP 32        /* runs per warp step: one per lane */
#define ORBG_RUN_MAX_PRE 20  /* prefix positions stored per run */

/* One run: 32 bytes, read by a lane as two 16-byte loads. */
struct OrbgRun {
    uint32_t tstart;    /* 1-based query index of the run's first pattern */
    uint16_t pair_sum;  /* a0 + b0 for 0-based pair positions a0 < b0 */
    uint16_t a0;        /* first a0; runs of one pattern: a0 = b0 = n */
    uint8_t len;        /* patterns in the run, >= 1 */
    uint8_t npre;       /* prefix positions used */
    uint8_t pad[2];
    uint8_t pre[ORBG_RUN_MAX_PRE]; /* 0-based prefix positions, ascending */
};

/* What a kernel needs of one code (passed by value or from a device array). */
struct OrbgDeviceCode {
    const uint32_t *hcol;        /* [n][w32]: column j of H, row i at bit i%32 of word i/32 */
    const OrbgRun *runs;         /* [nruns] */
    const uint32_t *group_floor; /* [ngroups] */
    uint32_t nruns;
    uint32_t ngroups;
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
    std::vector<OrbgRun> runs;
    std::vector<uint32_t> group_floor;
    uint64_t patterns = 0;  /* query indices covered (last index) */
    int wmax_logistic = 0;  /* deepest logistic weight in the table */
};
int orbg_build_tables(int n, uint64_t cap, OrbgTables *out);

/* GF(2) helpers on dense 0/1 byte matrices (row-major). */
int orbg_gf2_rank(const uint8_t *M, int rows, int cols);
int orbg_gf2_nullspace(const uint8_t *M, int rows, int cols,
                       std::vector<uint8_t> *basis, int *dim);

/* Kernel launchers (orbg_kernels.cu).  Return a cudaError_t value. */
int orbg_launch_plain(const OrbgDeviceCode &code, const float *llr, int64_t B,
                      uint32_t cap, uint8_t *cw, uint32_t *q, uint8_t *ab,
                      void *stream);
int orbg_launch_batched(const OrbgDeviceCode *d_codes, int ncodes, int n_max,
                        int w32_max, const int32_t *code_id,
                        const int64_t *llr_off, const float *llr, int64_t B,
                        uint32_t cap, uint32_t budget, uint8_t *cw,
                        const int64_t *cw_off, uint32_t *q, uint8_t *ab,
                        unsigned long long *scratch, int warps_per_cta,
                        int ctas_per_sm, int grab, int heavy_warps, void *stream);
/* device scratch the batched form needs for B blocks: counters (queue head,
 * open-block count, phase-2 cursor) and the list of open blocks */
#define ORBG_BATCHED_COUNTERS 8
size_t orbg_batched_scratch_bytes(int64_t B);
int orbg_launch_heavy(const OrbgDeviceCode *d_codes, int ncodes, int n_max, int w32_max,
                      const int32_t *code_id, const int64_t *llr_off, const float *llr,
                      uint32_t cap, uint8_t *cw, const int64_t *cw_off, uint32_t *q, uint8_t *ab,
                      unsigned long long *counters, const unsigned long long *heavy,
                      int heavy_warps, void *stream);
int orbg_grid_for(const void *kern, int threads, size_t smem, int ctas_per_sm, int *grid_out);

/* What a launch needs of a code set (orbg_api.cpp owns the struct). */
#include "../../include/orbg.h"
struct OrbgSetView {
    const OrbgDeviceCode *d_codes;
    int ncodes, n_max, w32_max;
    uint32_t cap_min;
    orbg_tuning tuning;
};
int orbg_codeset_view(const orbg_codeset *set, OrbgSetView *out);
/* Records a cudaError_t for orbg_last_cuda_error; returns the orbg status. */
int orbg_note_cuda_error(int cuda_error);
int orbg_launch_int_probe(double *lanes_per_clk_per_sm);
#endif

#endif /* ORBG_INTERNAL_H */
