/* Host build of the device fit's steps (paper_2202_13951_gb300/csrc/
 * orbg_fit.cuh), so that a CPU test can compare them with the oracle's fit.
 * The sort here is the library's only in outcome (ascending |LLR|). */
#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "orbg_fit.cuh"

extern "C" int fit_host(const float *llr, int n, int lines, int divisible, int32_t *out)
{
    float s[256];
    if (n < 1 || n > 256 || lines < 1 || lines > ORBG_FIT_SEG)
        return -1;
    for (int i = 0; i < n; i++)
        s[i] = fabsf(llr[i]);
    std::sort(s, s + n);
    for (int i = 0; i < ORBG_FIT_WORDS; i++)
        out[i] = 0;
    orbg_fit::fit_sorted(s, n, lines, divisible, out);
    return 0;
}
