/* Host build of the device fit's steps (paper_2202_13951_gb300/csrc/
 * orbg_fit.cuh), so that a CPU test can compare them with the oracle's fit:
 * the same 256-slot bitonic network (+inf in the unused slots), its stages
 * in the kernel's order with each stage's pairs taken in turn, then the
 * same anchor search and quantisation. */
#include <math.h>
#include <stdint.h>

#include "orbg_fit.cuh"

extern "C" int fit_host(const float *llr, int n, int lines, int divisible, int32_t *out)
{
    float s[256];
    if (n < 1 || n > 256 || lines < 1 || lines > ORBG_FIT_SEG)
        return -1;
    for (int i = 0; i < 256; i++)
        s[i] = i < n ? fabsf(llr[i]) : INFINITY;
    for (int k = 2; k <= 256; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1)
            for (int t = 0; t < 128; t++)
                orbg_fit::bitonic_step(s, k, j, t);
    for (int i = 1; i < n; i++)
        if (!(s[i - 1] <= s[i]))
            return -2; /* not sorted */
    for (int i = 0; i < ORBG_FIT_WORDS; i++)
        out[i] = 0;
    orbg_fit::fit_sorted(s, n, lines, divisible, out);
    return 0;
}
