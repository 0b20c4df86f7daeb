/*
 * orbg_fitted_search_inst.cu -- the per-block fitted decoder's kernel
 * (orbg_fitted_search.cuh) for codes of n <= 32 ORBG_FS_K, each syndrome
 * width.  The build compiles this file once per K in 1, 2, 4, 8.
 */
#include "orbg_fitted_search.cuh"

#ifndef ORBG_FS_K
#define ORBG_FS_K 1
#endif

#define ORBG_FS_CAT(kk) orbg_launch_fitsearch_k##kk
#define ORBG_FS_NAME(k) ORBG_FS_CAT(k)

int ORBG_FS_NAME(ORBG_FS_K)(const OrbgDeviceCode &code, const float *llr, int64_t B,
                            uint32_t cap, int lines, int divisible, uint8_t *cw, uint32_t *q,
                            uint8_t *ab, int32_t *models, unsigned char *scratch,
                            void *stream)
{
    using namespace orbg_fitsearch;
    if (code.w32 <= 1)
        return launch_fitsearch<ORBG_FS_K, 1>(code, llr, B, cap, lines, divisible, cw, q, ab,
                                              models, scratch, stream);
    if (code.w32 == 2)
        return launch_fitsearch<ORBG_FS_K, 2>(code, llr, B, cap, lines, divisible, cw, q, ab,
                                              models, scratch, stream);
    return launch_fitsearch<ORBG_FS_K, 4>(code, llr, B, cap, lines, divisible, cw, q, ab, models,
                                          scratch, stream);
}
