/*
 * orbg_fit.cuh -- the per-block fit of Sec. III-E on one sorted curve:
 * anchor search and quantisation (Eq. Q, Eq. quant).  Host and device:
 * the device kernel (orbg_fit.cu) calls it from one lane per block, and a
 * host build lets the same steps be checked on the CPU.  Every floating-
 * point operation is a separate IEEE double operation (on the device the
 * _rn intrinsics, which are never fused into a multiply-add), so both
 * builds give the same integers.
 */
#ifndef ORBG_FIT_CUH
#define ORBG_FIT_CUH

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define ORBG_FIT_HD __host__ __device__
#else
#define ORBG_FIT_HD
#endif

#define ORBG_FIT_SEG 8     /* lines at most */
#define ORBG_FIT_WORDS 24  /* int32 per block: m, anchors[7], J[8], beta[8] */

namespace orbg_fit {

ORBG_FIT_HD inline double add(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
ORBG_FIT_HD inline double sub(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
ORBG_FIT_HD inline double mul(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
ORBG_FIT_HD inline double dvd(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}

/* One compare-exchange of the ascending bitonic sort over `slots` (a power
 * of two) values: stage (k, j) compares index i and i + j for the slots / 2
 * indices i with bit j clear, t = 0 .. slots/2 - 1 numbering them, in
 * direction (i & k) == 0 (ascending).  Stages run for k = 2, 4, .., slots
 * and, inside each, j = k/2, k/4, .., 1; every pair of a stage is
 * independent of the others. */
ORBG_FIT_HD inline void bitonic_step(float *s, int k, int j, int t)
{
    const int i = (t / j) * 2 * j + (t % j);
    const int l = i + j;
    const float va = s[i], vb = s[l];
    if ((va > vb) == ((i & k) == 0)) {
        s[i] = vb;
        s[l] = va;
    }
}

/* [x]: rounding half away from zero */
ORBG_FIT_HD inline long long round_half_away(double x)
{
    return (long long)(x < 0.0 ? -floor(add(-x, 0.5)) : floor(add(x, 0.5)));
}

/* L_j, 1-based, from the sorted values */
ORBG_FIT_HD inline double Lj(const float *s, int j) { return (double)s[j - 1]; }

/* The vertical gap at index j between the chord of the ordered curve over
 * [lo, hi] and the curve itself (the anchor search of Sec. III-E). */
ORBG_FIT_HD inline double chord_gap(const float *s, int lo, int hi, int j)
{
    const double Llo = Lj(s, lo);
    const double rise = sub(Lj(s, hi), Llo);
    const double chord = add(Llo, dvd(mul(rise, (double)(j - lo)), (double)(hi - lo)));
    return fabs(sub(chord, Lj(s, j)));
}

/* Eq. Q and Eq. quant for the anchors a[0] = 1 < a[1] < ... < a[na-1]
 * (the last the centre floor(n/2)): writes out as fit_sorted does (out
 * holds the basic model on entry). */
ORBG_FIT_HD inline void quantise(const float *s, const int *a, int na, int divisible,
                                 int32_t *out)
{
    const double kFitMax = 16777216.0; /* 2^24 */
    const int m = na - 1;
    double sl[ORBG_FIT_SEG];
    sl[0] = dvd(sub(Lj(s, a[1]), Lj(s, 1)), (double)(a[1] - 1));
    for (int i = 2; i <= m; i++)
        sl[i - 1] = dvd(sub(Lj(s, a[i]), Lj(s, a[i - 1])), (double)(a[i] - a[i - 1]));
    double Q = sl[0];
    for (int i = 1; i < m; i++)
        if (sl[i] < Q)
            Q = sl[i];
    if (!(Q > 0.0))
        return;
    for (int i = 0; i < m; i++)
        if (!(dvd(sl[i], Q) <= kFitMax) || !(dvd(Lj(s, a[i]), Q) <= kFitMax))
            return;
    long long J[ORBG_FIT_SEG], beta[ORBG_FIT_SEG];
    for (int i = 0; i < m; i++)
        beta[i] = round_half_away(dvd(sl[i], Q));
    J[0] = round_half_away(dvd(Lj(s, 1), Q)) - beta[0];
    for (int i = 1; i < m; i++)
        J[i] = round_half_away(dvd(Lj(s, a[i]), Q));
    if (divisible)
        for (int i = 0; i < m; i++)
            J[i] = round_half_away(dvd((double)J[i], (double)beta[i])) * beta[i];
    out[0] = m;
    for (int i = 1; i < m; i++)
        out[i] = a[i];
    for (int i = 0; i < m; i++) {
        out[8 + i] = (int32_t)J[i];
        out[16 + i] = (int32_t)beta[i];
    }
}

/*
 * s: the n reliabilities in ascending order.  Writes out[0..23]: m, the
 * anchors I_1..I_{m-1} at 1.., J_0..J_{m-1} at 8.., beta_1..beta_m at
 * 16.. (out zeroed by the caller).  Anchors start at 1 and floor(n/2);
 * each further anchor splits the first interval at its largest chord gap
 * (smaller index on ties) until `lines` segments or no gap; Q = the
 * smallest slope; beta_i = [s_i / Q], J_0 = [L_1 / Q] - beta_1, J_i =
 * [L_{I_i} / Q]; divisible: J_{i-1} <- [J_{i-1} / beta_i] beta_i.  n < 4,
 * Q <= 0 or a ratio above 2^24 (or not finite): the basic model.
 */
ORBG_FIT_HD inline void fit_sorted(const float *s, int n, int lines, int divisible, int32_t *out)
{
    int a[ORBG_FIT_SEG + 1];
    int na = 2;
    out[0] = 1;
    out[8] = 0;  /* J_0 */
    out[16] = 1; /* beta_1 */
    if (n < 4)
        return;
    a[0] = 1;
    a[1] = n / 2;
    while (na - 1 < lines) {
        const int lo = a[0], hi = a[1];
        int best = -1;
        double gap = 0.0;
        for (int j = lo + 1; j < hi; j++) {
            const double g = chord_gap(s, lo, hi, j);
            if (g > gap) {
                gap = g;
                best = j;
            }
        }
        if (best < 0)
            break;
        for (int k = na; k > 1; k--)
            a[k] = a[k - 1];
        a[1] = best;
        na++;
    }
    quantise(s, a, na, divisible, out);
}

}  // namespace orbg_fit

#endif /* ORBG_FIT_CUH */
