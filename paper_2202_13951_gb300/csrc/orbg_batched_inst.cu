/*
 * orbg_batched_inst.cu -- one instantiation of the batched form's kernels
 * (orbg_batched.cuh) for codes of n <= 32 ORBG_INST_K and ORBG_INST_W
 * syndrome words, and of the phase-1 kernel of exactly that decoder
 * variant (mixed-code calls launch one per variant).  The build compiles this file once per pair (K in
 * 1, 2, 4, 8; W in 1, 2, 4), defining the two macros.
 */
#include "orbg_batched.cuh"

#ifndef ORBG_INST_K
#define ORBG_INST_K 1
#endif
#ifndef ORBG_INST_W
#define ORBG_INST_W 1
#endif

#define ORBG_INST_CAT(kk, ww) orbg_launch_batched_k##kk##w##ww
#define ORBG_INST_NAME(k, w) ORBG_INST_CAT(k, w)

int ORBG_INST_NAME(ORBG_INST_K, ORBG_INST_W)(const OrbgBatchedArgs &a)
{
    return orbg_batched_impl::launch_kw<ORBG_INST_K, ORBG_INST_W>(a);
}

#define ORBG_INST_CAT_EX(kk, ww) orbg_launch_exact_k##kk##w##ww
#define ORBG_INST_NAME_EX(k, w) ORBG_INST_CAT_EX(k, w)

int ORBG_INST_NAME_EX(ORBG_INST_K, ORBG_INST_W)(const OrbgBatchedArgs &a, const OrbgScratch &s,
                                                unsigned long long *queue, int blo, int bhi,
                                                int pdl, int stride)
{
    return stride ? orbg_batched_impl::launch_exact_t<ORBG_INST_K, ORBG_INST_W, true>(
                        a, s, queue, blo, bhi, pdl)
                  : orbg_batched_impl::launch_exact_t<ORBG_INST_K, ORBG_INST_W, false>(
                        a, s, queue, blo, bhi, pdl);
}
