/*
 * orbg_fitted_search.cuh -- full ORBGRAND with a piece-wise linear model
 * fitted to each block (Sec. III-E), searched in that block's own order
 * (Sec. III-D), one warp per block.
 *
 * Per block, in three launches (each kernel's code stays small enough for
 * the instruction cache: in one fused kernel the fit's double-precision code
 * and the search's tree walk, run by different warps of an SM at once, made
 * instruction fetch the largest stall).  The first launch does steps 1-3
 * and finishes the blocks that need no search; the second takes the others
 * from an open list, with their order and model in a handover record, one
 * warp per block; a block whose search grows long there goes to the third,
 * where all warps of a CTA search it (so the few longest blocks, which one
 * warp each would finish long after the rest, end sooner):
 *   1. load, hard decision y, starting syndrome s0 = H y (as the other
 *      decoders: load_block);
 *   2. the exact reliability order pi (sort_block) and the ordered curve
 *      L_1 <= ... <= L_n;
 *   3. the fit: anchors by the largest chord gap (every lane takes a share of
 *      the indices; the warp keeps the largest gap, the smaller index on
 *      ties), then Eq. Q and Eq. quant on one lane (orbg_fit.cuh, the same
 *      double operations as the oracle);
 *   4. the integer weight rho_j of every sorted position j (Eq. relest_seg:
 *      J_{i-1} + beta_i (j - I_{i-1}) on segment i) and the suffix minima
 *      msuf_j = min over j' >= j of rho_j';
 *   5. the search for the first code-book member in the order of increasing
 *      reliability weight R(z) = sum of rho over the flipped positions, ties
 *      by Hamming weight and then positions lexicographically (the order
 *      every decoder of this library uses inside one weight).
 *
 * The search walks the subsets of {1..n} as a binary tree in lexicographic
 * order: node S = {j_1 < ... < j_t} has the child S + {j_t + 1} ("add") and
 * the next sibling S - {j_t} + {j_t + 1} ("replace"); every non-empty subset
 * is reached once from the root {1}.  Everything below a node keeps
 * j_1..j_{t-1} and adds positions >= j_t, so R(S) - rho_{j_t} + msuf_{j_t}
 * bounds the weight of the node and all it leads to from below; a pass with
 * bound Rhi enters only nodes whose bound is <= Rhi and tests those with
 * R <= Rhi (the weights rho need not increase with j).  The 32 lanes of the
 * warp each walk a part of the tree depth first (lane l starts with the sets
 * whose least position is l + 1), with their positions on a per-lane stack
 * in shared memory; a lane that runs out of work is given the "replace"
 * branch of a lane that is about to take its "add" branch; a lane at a leaf
 * also tests up to kLeafRun of the leaf's later siblings in the same step
 * while they are leaves too (the lanes stay in step: a longer inner run
 * would hold the other lanes).  When the warps of a CTA share a block, the
 * tree is cut into kClasses classes by the sets' second positions (modulo
 * kClasses; the singletons by their position), the warps take classes from
 * a counter, and each pass's node counts and least member are combined over
 * the warps.
 *
 * Passes run with growing bounds ("bands"): a pass that finds code-book
 * members lowers its bound to the lightest one found, and the least of
 * them in the order (weight, Hamming weight, positions) is the decoding; a
 * second pass over the nodes up to that weight counts the patterns that
 * come before it, which gives its query index.  A pass without a member
 * that already covers `cap` queries ends the block as abandoned.  Every
 * pass is a finite walk of a finite tree; each also stops after a fixed
 * number of steps (a guard, never reached by a correct walk) and marks the
 * block ORBG_BLOCK_RANGE, as does a search that would need weights beyond
 * 2^26 - 1.
 */
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "orbg_decode_block.cuh"
#include "orbg_fit.cuh"

namespace orbg_fitsearch {

using namespace orbg_dev;

constexpr int kWarps = 8;                   /* warps per CTA, one block each */
constexpr int kDepth = 31;                  /* largest pattern the stack holds */
constexpr uint32_t kRhoInf = 1u << 30;      /* weight of a position never reached */
constexpr int32_t kRmax = (1 << 26) - 1;    /* heaviest reliability weight searched */
constexpr int kLeafRun = 3;                /* leaf siblings tested per step besides the node */
/* nodes a one-warp pass may test before a CTA takes over (a quarter of the
 * cap if less): measured on BCH(127,113) and CA-Polar[256,234] (3 lines),
 * 2^16 sends so many BCH blocks to the CTA search (each restarting there)
 * that its step grows by a fifth; 2^18 costs BCH nothing and still takes
 * the long CA-Polar blocks off single warps */
constexpr uint32_t kSplit = 1u << 18;
constexpr int32_t kNoHit = 0x7FFFFFFF;
constexpr int kBlockRange = ORBG_BLOCK_RANGE; /* abandoned[] value: beyond the search range */

/* Shared memory of one warp (one block in flight). */
template <int W> struct FsSmem {
    typedef typename Syn<W>::T T;
    uint32_t *rho;   /* [258] rho_j, j = 1..n; rho[n + 1] = kRhoInf */
    uint32_t *msuf;  /* [258] suffix minima, msuf[n + 1] = kRhoInf */
    uint32_t *c0;    /* [258] first syndrome word of position j; c0[0] = 0 */
    T *h;            /* [258] whole syndrome of position j (W > 1) */
    float *L;        /* [256] ordered reliabilities */
    uint8_t *pi;     /* [256] received index of sorted position j - 1 */
    uint8_t *cw;     /* [256] staged codeword */
    uint8_t *stk;    /* [32][32] stk[d * 32 + lane]: j_{d+1} of the lane's node */
    uint8_t *hb;     /* [32][32] hb[i * 32 + lane]: the lane's best member so far */
    uint8_t *best;   /* [32] the block's decoding, positions ascending */
    int32_t *rec;    /* [24] the block's model record */
    int32_t *anch;   /* [9] anchors during the fit */
    __device__ __forceinline__ FsSmem(unsigned char *base)
    {
        unsigned char *p = base;
        rho = (uint32_t *)p;
        p += 258 * 4;
        msuf = (uint32_t *)p;
        p += 258 * 4;
        c0 = (uint32_t *)p;
        p += 258 * 4;
        p = (unsigned char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
        h = (T *)p;
        if (W > 1)
            p += 258 * sizeof(T);
        L = (float *)p;
        p += 256 * 4;
        pi = p;
        p += 256;
        cw = p;
        p += 256;
        stk = p;
        p += 32 * 32;
        hb = p;
        p += 32 * 32;
        best = p;
        p += 32;
        rec = (int32_t *)p;
        p += 24 * 4;
        anch = (int32_t *)p;
    }
};

template <int W>
__host__ __device__ constexpr uint32_t fs_warp_bytes()
{
    return (uint32_t)((3 * 258 * 4 + 15) / 16 * 16 + (W > 1 ? 258 * 4 * W : 0) + 256 * 4 + 256 +
                      256 + 32 * 32 + 32 * 32 + 32 + 24 * 4 + 9 * 4 + 15) /
           16 * 16;
}

/* ---------------------------------------------------------- the fit */

/* The largest chord gap over the indices of (lo, hi), the smaller index on
 * equal gaps (-1 if no gap is > 0), exactly as the one-lane loop of
 * fit_sorted finds it.  Each lane first computes its indices' gaps in
 * single precision: with M the largest |L| of the interval, a single-
 * precision gap is within 7 * 2^-24 M of the double-precision one (five
 * roundings, each of a value <= 2 M), so an index whose single-precision gap
 * is more than 2^-19 M below the largest cannot hold the largest double-
 * precision gap.  If exactly one index is left and its gap exceeds 2^-19 M,
 * its double-precision gap is positive and larger than every other one: it
 * is the answer, with no double-precision work; otherwise the remaining
 * candidates are evaluated in double precision (all of them when the curve
 * is not finite there). */
template <int W>
__device__ __forceinline__ int chord_argmax(const FsSmem<W> &sm, int lo, int hi, int lane)
{
    float M = 0.0f, g32max = 0.0f;
    for (int j = lo + lane; j <= hi; j += 32)
        M = fmaxf(M, sm.L[j - 1]);
    /* reliabilities are >= 0 (or +inf): their bit patterns order as they do */
    M = __uint_as_float(__reduce_max_sync(FULL_MASK, __float_as_uint(M)));
    const bool finite = isfinite(M);
    const float Llo = sm.L[lo - 1], rise = sm.L[hi - 1] - Llo, span = (float)(hi - lo);
    const float margin = ldexpf(M, -19);
    if (finite) {
        for (int j = lo + 1 + lane; j < hi; j += 32)
            g32max = fmaxf(g32max, fabsf(Llo + rise * (float)(j - lo) / span - sm.L[j - 1]));
        g32max = __uint_as_float(__reduce_max_sync(FULL_MASK, __float_as_uint(g32max)));
        const float cut = g32max - margin;
        uint32_t n_cand = 0;
        int cand = -1;
        for (int j = lo + 1 + lane; j < hi; j += 32)
            if (fabsf(Llo + rise * (float)(j - lo) / span - sm.L[j - 1]) >= cut) {
                n_cand++;
                cand = j;
            }
        if (__reduce_add_sync(FULL_MASK, n_cand) == 1u && g32max > margin)
            return __reduce_max_sync(FULL_MASK, (unsigned)(cand + 1)) - 1;
    }
    const float cut = g32max - margin;
    double gap = 0.0;
    int best = -1;
    for (int j = lo + 1 + lane; j < hi; j += 32) {
        if (finite && fabsf(Llo + rise * (float)(j - lo) / span - sm.L[j - 1]) < cut)
            continue;
        const double g = orbg_fit::chord_gap(sm.L, lo, hi, j);
        if (g > gap) {
            gap = g;
            best = j;
        }
    }
    /* gaps kept are >= 0 and not NaN: their bit patterns order as they do */
    unsigned long long gb = (unsigned long long)__double_as_longlong(gap);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long og = __shfl_xor_sync(FULL_MASK, gb, d);
        const int oj = __shfl_xor_sync(FULL_MASK, best, d);
        if (oj >= 0 && (best < 0 || og > gb || (og == gb && oj < best))) {
            gb = og;
            best = oj;
        }
    }
    return best;
}

/* Eq. Q and Eq. quant for the anchors sm.anch[0..na-1], one segment per
 * lane: the same double operations per segment as orbg_fit::quantise, and
 * the same results (the least slope is taken over the segments in any
 * order; a NaN first slope gives the basic model as there).  Writes sm.rec,
 * which holds the basic model on entry. */
template <int W>
__device__ __forceinline__ void quantise_lanes(const FsSmem<W> &sm, int na, int divisible,
                                               int lane)
{
    using namespace orbg_fit;
    const double kFitMax = 16777216.0; /* 2^24 */
    const int m = na - 1;
    const bool mine = lane < m;
    const int a0 = sm.anch[mine ? lane : 0], a1 = sm.anch[mine ? lane + 1 : 1];
    const double sl = mine ? dvd(sub(Lj(sm.L, a1), Lj(sm.L, a0)), (double)(a1 - a0)) : 0.0;
    const double s0 = __shfl_sync(FULL_MASK, sl, 0);
    double Q = mine ? sl : s0;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        Q = fmin(Q, __shfl_xor_sync(FULL_MASK, Q, d));
    if (s0 != s0)
        Q = s0; /* the first slope NaN: as the one-lane loop, no positive Q */
    if (!(Q > 0.0))
        return;
    const double rs = mine ? dvd(sl, Q) : 0.0;
    const double rl = mine ? dvd(Lj(sm.L, a0), Q) : 0.0;
    const bool bad = mine && (!(rs <= kFitMax) || !(rl <= kFitMax));
    if (__any_sync(FULL_MASK, bad))
        return;
    long long beta = 0, J = 0;
    if (mine) {
        beta = round_half_away(rs);
        J = round_half_away(rl);
    }
    const long long beta1 = __shfl_sync(FULL_MASK, beta, 0);
    if (lane == 0)
        J -= beta1;
    if (mine && divisible)
        J = round_half_away(dvd((double)J, (double)beta)) * beta;
    __syncwarp();
    if (lane == 0)
        sm.rec[0] = m;
    if (mine) {
        if (lane >= 1)
            sm.rec[lane] = a0;
        sm.rec[8 + lane] = (int32_t)J;
        sm.rec[16 + lane] = (int32_t)beta;
    }
    __syncwarp();
}

/* Sec. III-E on the ordered curve sm.L: anchors by the largest chord gap,
 * then Eq. Q / Eq. quant.  Writes sm.rec. */
template <int W>
__device__ void fit_block(const FsSmem<W> &sm, int n, int lines, int divisible, int lane)
{
    if (lane < ORBG_FIT_WORDS)
        sm.rec[lane] = 0;
    __syncwarp();
    if (lane == 0) {
        sm.rec[0] = 1;
        sm.rec[8] = 0;
        sm.rec[16] = 1;
        sm.anch[0] = 1;
        sm.anch[1] = n / 2;
    }
    __syncwarp();
    if (n < 4)
        return;
    int na = 2;
    while (na - 1 < lines) {
        const int best = chord_argmax<W>(sm, sm.anch[0], sm.anch[1], lane);
        if (best < 0)
            break;
        __syncwarp();
        if (lane == 0) {
            for (int k = na; k > 1; k--)
                sm.anch[k] = sm.anch[k - 1];
            sm.anch[1] = best;
        }
        __syncwarp();
        na++;
    }
    quantise_lanes<W>(sm, na, divisible, lane);
}

/* rho_j from the model record (Eq. relest_seg), clamped to kRhoInf, and the
 * suffix minima.  Lane l owns positions 8l + 1 .. 8l + 8. */
template <int W>
__device__ void position_weights(const FsSmem<W> &sm, int n, int lane)
{
    const int m = sm.rec[0];
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int j = 8 * lane + 1 + i;
        uint32_t r = kRhoInf;
        if (j <= n) {
            int seg = 0, Ilo = 0;
            for (int s = 1; s < m; s++)
                if (j > sm.rec[s]) {
                    seg = s;
                    Ilo = sm.rec[s];
                }
            const long long w =
                (long long)sm.rec[8 + seg] + (long long)sm.rec[16 + seg] * (long long)(j - Ilo);
            r = w < 0 ? 0u : w >= (long long)kRhoInf ? kRhoInf : (uint32_t)w;
            sm.rho[j] = r;
        }
        v[i] = r;
    }
#pragma unroll
    for (int i = 6; i >= 0; i--)
        v[i] = min(v[i], v[i + 1]);
    /* minimum over the lanes above: inclusive suffix scan, shifted by one */
    uint32_t incl = v[0];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_down_sync(FULL_MASK, incl, d);
        if (lane + d < 32)
            incl = min(incl, o);
    }
    uint32_t above = __shfl_down_sync(FULL_MASK, incl, 1);
    if (lane == 31)
        above = kRhoInf;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int j = 8 * lane + 1 + i;
        if (j <= n)
            sm.msuf[j] = min(v[i], above);
    }
    if (lane == 0) {
        sm.rho[n + 1] = kRhoInf;
        sm.msuf[n + 1] = kRhoInf;
    }
    __syncwarp();
}

/* ------------------------------------------------- the tree walk */

/* Is the lane's node (stack j_1..j_{t-1}, then jt) before the t-position
 * pattern other[i * ostride] in lexicographic order? */
__device__ __forceinline__ bool node_lex_less(const uint8_t *stk, int lane, int t, int jt,
                                              const uint8_t *other, int ostride)
{
    for (int i = 0; i < t; i++) {
        const int a = i < t - 1 ? (int)stk[i * 32 + lane] : jt;
        const int b = (int)other[i * ostride];
        if (a != b)
            return a < b;
    }
    return false;
}

/* Are the best members of lanes la and lb (t positions each) in
 * lexicographic order? */
__device__ __forceinline__ bool hb_lex_less(const uint8_t *hb, int la, int lb, int t)
{
    for (int i = 0; i < t; i++) {
        const int a = hb[i * 32 + la], b = hb[i * 32 + lb];
        if (a != b)
            return a < b;
    }
    return false;
}

/* Syndrome of the lane's node on all W words. */
template <int W>
__device__ __noinline__ bool node_is_member(const FsSmem<W> &sm, int lane, int t, int jt,
                                            typename Syn<W>::T s0)
{
    typename Syn<W>::T P = sx(s0, sm.h[jt]);
    for (int i = 0; i < t - 1; i++)
        P = sx(P, sm.h[sm.stk[i * 32 + lane]]);
    return sz(P);
}

/*
 * One pass over the nodes whose bound is <= Rhi.
 * RANK = false: tests every node with R <= Rhi; a lane keeps its least
 *   member (bR, bT, its positions in hb) and the bound drops to the warp's
 *   lightest member.  Returns the number of nodes tested (lane's share).
 * RANK = true: counts the nodes before the block's decoding (weight Rb,
 *   Hamming weight Tb, positions sm.best): lighter, or as heavy with fewer
 *   positions, or as heavy and as many positions and lexicographically
 *   smaller.  Returns the lane's share of that count.
 * *guard is set (warp-uniform) if the walk exceeds `steps` iterations.
 * P, w: the walk covers class w of P (P = 1, w = 0: the whole tree): the
 * sets {j} with j = w + 1 modulo P and the larger sets whose second position
 * is w + 1 modulo P.  It walks all the depth-1 nodes, and its steps to depth
 * 2 go to the next such position ("add") or P positions on ("replace"), so
 * the big subtrees of the least reliable positions are shared out evenly.
 */
template <int W, bool RANK, int P>
__device__ uint32_t tree_pass(const FsSmem<W> &sm, int n, typename Syn<W>::T s0, int32_t Rhi,
                              int32_t Rb, int Tb, int lane, uint32_t steps, int32_t *bR,
                              int *bT, bool *guard, int w)
{
    const uint32_t s0w = first_word(s0);
    bool active = false; /* an active lane's node is always untested yet */
    int t = 0, t0 = 0, jt = 0;
    uint32_t R = 0, rcur = 0, ccur = 0, syn = 0, don = 0, cnt = 0;
    /* every lane starts at once: lane l < L takes the sets whose least
     * position is l + 1 (the node {l + 1} and what its "add" branch leads to:
     * the "replace" branch at depth 1 is marked as given away), lane L the
     * sets whose least position is L + 1 or more (node {L + 1} with both
     * branches); L = min(n, 32) - 1 */
    const int last = min(n, 32) - 1;
    if (lane <= last) {
        jt = lane + 1;
        rcur = sm.rho[jt];
        ccur = sm.c0[jt];
        active = (lane < last ? rcur : sm.msuf[jt]) <= (uint32_t)Rhi;
        t = 1;
        t0 = 1;
        don = lane < last ? 1u << 1 : 0u;
        R = rcur;
        syn = s0w ^ ccur;
    }
    uint32_t it = 0;
    for (;;) {
        const uint32_t act = __ballot_sync(FULL_MASK, active);
        if (act == 0)
            break;
        if (++it > steps) {
            *guard = true;
            break;
        }
        const bool tested =
            active && R <= (uint32_t)Rhi && (P == 1 || t != 1 || (jt - 1) % P == w);
        if (RANK) {
            if (tested) {
                if (R < (uint32_t)Rb)
                    cnt++;
                else if (R == (uint32_t)Rb &&
                         (t < Tb || (t == Tb && node_lex_less(sm.stk, lane, t, jt, sm.best, 1))))
                    cnt++;
            }
        } else {
            cnt += tested ? 1u : 0u;
            const bool cand = tested && syn == 0u;
            if (__any_sync(FULL_MASK, cand)) {
                if (cand && (W == 1 || node_is_member<W>(sm, lane, t, jt, s0))) {
                    const bool better =
                        (int32_t)R < *bR ||
                        ((int32_t)R == *bR &&
                         (t < *bT ||
                          (t == *bT && node_lex_less(sm.stk, lane, t, jt, sm.hb + lane, 32))));
                    if (better) {
                        for (int i = 0; i < t - 1; i++)
                            sm.hb[i * 32 + lane] = sm.stk[i * 32 + lane];
                        sm.hb[(t - 1) * 32 + lane] = (uint8_t)jt;
                        *bR = (int32_t)R;
                        *bT = t;
                    }
                }
                /* nothing heavier than the lightest member found can come first */
                Rhi = min(Rhi, __reduce_min_sync(FULL_MASK, *bR));
            }
        }
        /* the "add" child's new position: one on (at depth 1, on to the
         * warp's class) */
        const int jn = P == 1 || t != 1 ? jt + 1 : jt + 1 + ((w - jt) % P + P) % P;
        const bool okn = active && jn <= n;
        const uint32_t ms = okn ? sm.msuf[jn] : kRhoInf;
        const bool addOK = okn && R + ms <= (uint32_t)Rhi;
        /* the "replace" branch's position: one on, or P on at depth 2 */
        const int rs = t == 2 ? P : 1;
        const int jr = jt + rs;
        const bool okr = active && jr <= n;
        const uint32_t msr = P == 1 ? ms : okr ? sm.msuf[jr] : kRhoInf;
        bool replOK = okr && R - rcur + msr <= (uint32_t)Rhi && !((don >> t) & 1u);
        /* lanes without work take the replace branch of lanes about to add */
        const uint32_t idle = ~act;
        const uint32_t donors = __ballot_sync(FULL_MASK, addOK && replOK);
        bool got = false;
        if (idle != 0u && donors != 0u) {
            const uint32_t below = (1u << lane) - 1u;
            int src = lane;
            if (!active) {
                /* the r-th idle lane takes the r-th donor's branch */
                uint32_t r = __popc(idle & below);
                if (r < (uint32_t)__popc(donors)) {
                    uint32_t m = donors;
                    for (; r > 0; r--)
                        m &= m - 1u;
                    src = __ffs(m) - 1;
                }
            }
            const bool give = addOK && replOK && __popc(donors & below) < __popc(idle);
            const int st = __shfl_sync(FULL_MASK, t, src);
            const int sj = __shfl_sync(FULL_MASK, jt, src);
            const uint32_t sR = __shfl_sync(FULL_MASK, R, src);
            const uint32_t ssyn = __shfl_sync(FULL_MASK, syn, src);
            const uint32_t src_r = __shfl_sync(FULL_MASK, rcur, src);
            const uint32_t src_c = __shfl_sync(FULL_MASK, ccur, src);
            if (src != lane) {
                const int sjr = sj + (st == 2 ? P : 1); /* the donor's replace position */
                const uint32_t rn = sm.rho[sjr], cn = sm.c0[sjr];
                for (int d = 0; d < st - 1; d++)
                    sm.stk[d * 32 + lane] = sm.stk[d * 32 + src];
                t = st;
                t0 = st;
                jt = sjr;
                R = sR - src_r + rn;
                syn = ssyn ^ src_c ^ cn;
                rcur = rn;
                ccur = cn;
                don = 0;
                active = true;
                got = true;
            }
            if (give) {
                don |= 1u << t;
                replOK = false;
            }
            __syncwarp();
        }
        if (active && !got) {
            int jm = addOK ? jn : jr; /* the position the move brings in */
            bool move = addOK || replOK;
            if (addOK && t >= kDepth) {
                *guard = true; /* deeper than the stack: cannot happen within 2^26 queries */
                active = false;
                move = false;
            } else if (addOK) {
                sm.stk[(t - 1) * 32 + lane] = (uint8_t)jt;
                t++;
            } else if (replOK && (P == 1 || t != 1)) {
                /* a leaf: test up to kLeafRun of its later siblings (same
                 * prefix, last position jm = jt + 1, ...) in this step while
                 * they are leaves too; stop at one that leads further or needs
                 * the full step, and move there (or past the tested ones) */
                const uint32_t Rp = R - rcur, sp = syn ^ ccur;
                move = false;
                bool stop = false;
#pragma unroll
                for (int u = 0; u < kLeafRun; u++) {
                    if (stop)
                        break;
                    if (jm > n || Rp + sm.msuf[jm] > (uint32_t)Rhi) {
                        stop = true; /* no later sibling is reachable */
                        break;
                    }
                    const uint32_t r = sm.rho[jm], Rs = Rp + r;
                    const bool inner = jm < n && Rs + sm.msuf[jm + 1] <= (uint32_t)Rhi;
                    const bool own = Rs <= (uint32_t)Rhi &&
                                     (RANK ? Rs == (uint32_t)Rb : (sp ^ sm.c0[jm]) == 0u);
                    if (inner || own) {
                        move = true;
                        stop = true;
                        break;
                    }
                    if (Rs <= (uint32_t)Rhi)
                        cnt += RANK ? (Rs < (uint32_t)Rb ? 1u : 0u) : 1u;
                    jm += rs;
                }
                if (!stop)
                    move = jm <= n && Rp + sm.msuf[jm] <= (uint32_t)Rhi;
                if (!move) {
                    /* the siblings are done: back up from the prefix */
                    R = Rp;
                    syn = sp;
                    rcur = 0u;
                    ccur = 0u;
                }
            }
            if (!move && active && !addOK) {
                /* back up until an ancestor's "replace" branch is open (it is
                 * taken at once), or the lane's part of the tree is done */
                for (;;) {
                    if (t <= t0) {
                        active = false;
                        break;
                    }
                    R -= rcur;
                    syn ^= ccur;
                    don &= ~(1u << t);
                    t--;
                    jt = sm.stk[(t - 1) * 32 + lane];
                    rcur = sm.rho[jt];
                    ccur = RANK ? 0u : sm.c0[jt];
                    jm = jt + (t == 2 ? P : 1);
                    if (jm <= n + 1 && R - rcur + sm.msuf[jm] <= (uint32_t)Rhi &&
                        !((don >> t) & 1u)) {
                        move = true;
                        break;
                    }
                }
            }
            if (move) {
                /* the rank pass needs no syndromes */
                const uint32_t rn = sm.rho[jm], cn = RANK ? 0u : sm.c0[jm];
                if (addOK) {
                    R += rn;
                    syn ^= cn;
                } else {
                    /* replace: the last position jt gives way to jm = jt + 1 */
                    R = R - rcur + rn;
                    syn ^= ccur ^ cn;
                }
                jt = jm;
                rcur = rn;
                ccur = cn;
            }
        }
    }
    *guard = __any_sync(FULL_MASK, *guard);
    return cnt;
}

/* Sum over the warp of per-lane counts below 2^32 (exact in 64 bits). */
__device__ __forceinline__ uint64_t warp_sum64(uint32_t v)
{
    const uint64_t hi = __reduce_add_sync(FULL_MASK, v >> 16);
    const uint64_t lo = __reduce_add_sync(FULL_MASK, v & 0xFFFFu);
    return (hi << 16) + lo;
}

/* ---------------------------------------------------------- one block */

/* Handover record of a block left to the search launch (ORBG_FIT_HAND_BYTES
 * bytes): its reliability order pi (n bytes), its model record (24 int32)
 * and its starting syndrome s0. */
constexpr int kHandRec = 256;
constexpr int kHandS0 = 352;
static_assert(kHandS0 + 16 <= ORBG_FIT_HAND_BYTES, "handover record too small");

/* Stage 1 of a block (the preparing launch): load, hard decision, s0; the
 * exact reliability order and the fit (steps 1-3).  A block that needs no
 * search (NaN, a hard decision that is a code word, cap 1) is finished and
 * written here; any other is appended to the open list with its handover
 * record. */
template <int K, int W>
__device__ void prepare_fitted_block(const OrbgDeviceCode &code, const float *__restrict__ llr,
                                     uint8_t *__restrict__ cw_out, uint32_t *__restrict__ q_out,
                                     uint8_t *__restrict__ ab_out, int32_t *__restrict__ rec_out,
                                     uint32_t cap, int lines, int divisible, const FsSmem<W> &sm,
                                     int lane, uint32_t b, uint32_t *__restrict__ open,
                                     unsigned long long *__restrict__ nopen,
                                     unsigned char *__restrict__ hand)
{
    typedef typename Syn<W>::T T;
    const int n = code.n;
    uint32_t key[K];
    bool nan;
    const T s0 = load_block<K, W>(code, llr, key, sm.cw, lane, &nan);
    uint32_t q = 0;
    int ab = 0;
    if (nan) {
        ab = ORBG_BLOCK_NAN;
        if (rec_out && lane < ORBG_FIT_WORDS)
            rec_out[lane] = 0;
    } else if (sz(s0) && rec_out == nullptr) {
        q = 1; /* the hard decision is a code word: query 1, whatever the model */
    } else {
        sort_block<K>(key, llr, n, lane);
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int e = lane * K + k;
            if (e < n) {
                const int idx = (int)key[k];
                sm.pi[e] = (uint8_t)idx;
                sm.L[e] = fabsf(__ldg(llr + idx));
            }
        }
        __syncwarp();
        fit_block<W>(sm, n, lines, divisible, lane);
        if (rec_out && lane < ORBG_FIT_WORDS)
            rec_out[lane] = sm.rec[lane];
        if (sz(s0)) {
            q = 1;
        } else if (cap <= 1) {
            q = cap;
            ab = ORBG_BLOCK_ABANDONED;
        } else {
            /* to the search launch */
            unsigned long long slot = 0;
            if (lane == 0)
                slot = atomicAdd(nopen, 1ull);
            slot = __shfl_sync(FULL_MASK, slot, 0);
            unsigned char *r = hand + slot * ORBG_FIT_HAND_BYTES;
            for (int e = lane; e < n; e += 32)
                r[e] = sm.pi[e];
            if (lane < ORBG_FIT_WORDS)
                reinterpret_cast<int32_t *>(r + kHandRec)[lane] = sm.rec[lane];
            if (lane == 0) {
                *reinterpret_cast<T *>(r + kHandS0) = s0;
                open[slot] = b;
            }
            __syncwarp();
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int i = k * 32 + lane;
        if (i < n)
            cw_out[i] = sm.cw[i];
    }
    if (lane == 0) {
        *q_out = q;
        *ab_out = (uint8_t)ab;
    }
    __syncwarp();
}
/* A block's state for the search, from its handover record and LLRs: the
 * order, the permuted columns, the hard decision and the model, then the
 * position weights.  Returns s0. */
template <int W>
__device__ typename Syn<W>::T load_record(const OrbgDeviceCode &code,
                                          const float *__restrict__ llr, const FsSmem<W> &sm,
                                          int lane, const unsigned char *__restrict__ r)
{
    typedef typename Syn<W>::T T;
    const int n = code.n;
    for (int e = lane; e < n; e += 32) {
        const int idx = (int)r[e];
        sm.pi[e] = (uint8_t)idx;
        const T col = load_col<W>(code.hcol, idx);
        sm.c0[e + 1] = first_word(col);
        if (W > 1)
            sm.h[e + 1] = col;
        sm.cw[e] = __ldg(llr + e) > 0.0f ? 1 : 0;
    }
    if (lane == 0) {
        sm.c0[0] = 0u;
        if (W > 1)
            sm.h[0] = szero<T>();
    }
    if (lane < ORBG_FIT_WORDS)
        sm.rec[lane] = reinterpret_cast<const int32_t *>(r + kHandRec)[lane];
    __syncwarp();
    position_weights<W>(sm, n, lane);
    return *reinterpret_cast<const T *>(r + kHandS0);
}

/* Classes of the tree a CTA's warps share out, pass by pass, from a counter:
 * class k holds the sets {j} with j = k + 1 and the larger sets whose second
 * position is k + 1 modulo kClasses (many more classes than warps, so the
 * warps end a pass close together). */
constexpr int kClasses = 64; /* measured on CA-Polar[256,234]: 32 95 ms, 64 87, 128 88 */

/* Exchange area of the warps of a CTA that search one block together. */
struct FsTeam {
    unsigned int next[2];           /* the next class of a search pass, of a rank pass */
    unsigned long long c[kWarps];   /* a pass's tested nodes, per warp */
    int32_t rb[kWarps];             /* its lightest member's weight (kNoHit: none) */
    int32_t tb[kWarps];             /* that member's size */
    int32_t guard[kWarps];
    uint8_t pos[kWarps][32];        /* that member's positions */
};

/* The warp's least member of a pass (weight Rb over the warp): its size,
 * and (lanes < size) its positions in *pos_out. */
template <int W>
__device__ __forceinline__ int warp_least_member(const FsSmem<W> &sm, int lane, int32_t bR,
                                                 int bT, int32_t Rb, uint8_t *pos_out)
{
    int cl = bR == Rb ? lane : -1;
    int cT = bR == Rb ? bT : 0x7FFFFFFF;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const int ol = __shfl_down_sync(FULL_MASK, cl, d);
        const int oT = __shfl_down_sync(FULL_MASK, cT, d);
        if (lane + d < 32 && ol >= 0 &&
            (cl < 0 || oT < cT || (oT == cT && hb_lex_less(sm.hb, ol, cl, oT)))) {
            cl = ol;
            cT = oT;
        }
    }
    cl = __shfl_sync(FULL_MASK, cl, 0);
    const int Tb = __shfl_sync(FULL_MASK, cT, 0);
    if (lane < Tb)
        pos_out[lane] = sm.hb[lane * 32 + cl];
    __syncwarp();
    return Tb;
}

/*
 * The banded search of one block (steps 5): by one warp (CTA = false), or
 * by the kWarps warps of a CTA (CTA = true), each taking classes of the
 * tree (kClasses) from a counter, each pass's counts, members and guard
 * combined through `team` (every warp takes the same decisions).
 * split > 0 (one warp): a pass without a member that tests more than
 * `split` nodes (and has not reached the cap) ends the walk with *handover
 * set, for the CTA search.  Sets *q, *ab, and *wbest (the decoding's size;
 * its positions in sm.best).
 */
template <int W, bool CTA>
__device__ void band_search(const FsSmem<W> &sm, int n, typename Syn<W>::T s0, uint32_t cap,
                            int lane, int warp, FsTeam *team, uint32_t split, uint32_t *q_out,
                            int *ab_out, int *wbest_out, bool *handover)
{
    constexpr int P = CTA ? kClasses : 1;
    uint32_t q = 0;
    int ab = 0, wbest = 0;
    *handover = false;
    /* first bound: the twelfth position's weight (about seventy patterns
     * for the basic order) */
    uint32_t r12 = lane < 12 && lane < n ? sm.rho[lane + 1] : 0u;
    r12 = __reduce_max_sync(FULL_MASK, r12);
    int32_t Rhi = (int32_t)min(max(r12, sm.msuf[1]), (uint32_t)kRmax);
    int32_t Rprev = (int32_t)sm.msuf[1] - 1;
    double Cprev = 1.0;
    const uint32_t steps = 64u * (min(cap, (uint32_t)ORBG_MAX_QUERY_CAP) + 4096u);
    for (;;) {
        int32_t bR = kNoHit;
        int bT = 0;
        bool guard = false;
        uint32_t c = 0;
        if (!CTA) {
            c = tree_pass<W, false, 1>(sm, n, s0, Rhi, 0, 0, lane, steps, &bR, &bT, &guard, 0);
        } else {
            for (;;) {
                unsigned int k = 0;
                if (lane == 0)
                    k = atomicAdd(&team->next[0], 1u);
                k = __shfl_sync(FULL_MASK, k, 0);
                if (k >= (unsigned)kClasses)
                    break;
                const int32_t Rk = min(Rhi, __reduce_min_sync(FULL_MASK, bR));
                c += tree_pass<W, false, P>(sm, n, s0, Rk, 0, 0, lane, steps, &bR, &bT, &guard,
                                            (int)k);
            }
        }
        uint64_t tested = warp_sum64(c);
        int32_t Rb = __reduce_min_sync(FULL_MASK, bR);
        int Tb = 0;
        if (!CTA) {
            if (Rb != kNoHit && !guard)
                Tb = warp_least_member<W>(sm, lane, bR, bT, Rb, sm.best);
        } else {
            if (Rb != kNoHit && !guard)
                Tb = warp_least_member<W>(sm, lane, bR, bT, Rb, team->pos[warp]);
            if (lane == 0) {
                team->c[warp] = tested;
                team->rb[warp] = Rb;
                team->tb[warp] = Tb;
                team->guard[warp] = guard ? 1 : 0;
            }
            __syncthreads();
            if (threadIdx.x == 0)
                team->next[0] = 0u; /* no warp takes a class again before the sync below */
            /* the team's totals and least member: weight, size, positions */
            tested = 0;
            guard = false;
            Rb = kNoHit;
            int win = -1;
            for (int v = 0; v < kWarps; v++) {
                tested += team->c[v];
                guard |= team->guard[v] != 0;
                const int32_t r = team->rb[v];
                if (r == kNoHit)
                    continue;
                bool better = win < 0 || r < Rb;
                if (!better && r == Rb) {
                    const int t = team->tb[v], tw = team->tb[win];
                    better = t < tw;
                    if (t == tw)
                        for (int i = 0; i < t; i++)
                            if (team->pos[v][i] != team->pos[win][i]) {
                                better = team->pos[v][i] < team->pos[win][i];
                                break;
                            }
                }
                if (better) {
                    win = v;
                    Rb = r;
                }
            }
            if (win >= 0) {
                Tb = team->tb[win];
                if (lane < Tb)
                    sm.best[lane] = team->pos[win][lane];
            }
            __syncthreads(); /* every warp has read the team's entries */
        }
        if (guard) {
            ab = kBlockRange;
            break;
        }
        const double C = 1.0 + (double)tested;
        if (Rb != kNoHit) {
            __syncwarp();
            uint32_t b = 0;
            if (!CTA) {
                b = tree_pass<W, true, 1>(sm, n, s0, Rb, Rb, Tb, lane, steps, &bR, &bT, &guard,
                                          0);
            } else {
                for (;;) {
                    unsigned int k = 0;
                    if (lane == 0)
                        k = atomicAdd(&team->next[1], 1u);
                    k = __shfl_sync(FULL_MASK, k, 0);
                    if (k >= (unsigned)kClasses)
                        break;
                    b += tree_pass<W, true, P>(sm, n, s0, Rb, Rb, Tb, lane, steps, &bR, &bT,
                                               &guard, (int)k);
                }
            }
            uint64_t before = warp_sum64(b);
            if (CTA) {
                if (lane == 0) {
                    team->c[warp] = before;
                    team->guard[warp] = guard ? 1 : 0;
                }
                __syncthreads();
                if (threadIdx.x == 0)
                    team->next[1] = 0u;
                before = 0;
                guard = false;
                for (int v = 0; v < kWarps; v++) {
                    before += team->c[v];
                    guard |= team->guard[v] != 0;
                }
                __syncthreads();
            }
            if (guard) {
                ab = kBlockRange;
                break;
            }
            const uint64_t rank = 2ull + before;
            if (rank <= cap) {
                q = (uint32_t)rank;
                wbest = Tb;
            } else {
                q = cap;
                ab = ORBG_BLOCK_ABANDONED;
            }
            break;
        }
        if (C >= (double)cap) {
            q = cap;
            ab = ORBG_BLOCK_ABANDONED;
            break;
        }
        if (!CTA && split > 0 && C > (double)split) {
            *handover = true;
            break;
        }
        if (Rhi >= kRmax) {
            ab = kBlockRange;
            break;
        }
        /* next bound: aim at about four times the patterns (at most a little
         * past the cap), from the growth over the last band */
        const double target = fmin(4.0 * C, 1.25 * (double)cap + 64.0);
        const double span = (double)(Rhi - Rprev);
        double delta = 2.0 * span;
        if (C > Cprev) {
            const double g = log(C / Cprev) / span;
            delta = log(target / C) / g;
        }
        delta = fmax(1.0, fmin(delta, 4.0 * span));
        Rprev = Rhi;
        Cprev = C;
        Rhi = (int32_t)fmin((double)Rhi + ceil(delta), (double)kRmax);
    }
    if (q == 0u && ab == 0)
        ab = kBlockRange;
    *q_out = q;
    *ab_out = ab;
    *wbest_out = wbest;
}

/* The outputs of a searched block: the decoding's flips on the hard
 * decision, the query count and the flag. */
template <int K, int W>
__device__ __forceinline__ void write_fitted(const FsSmem<W> &sm, int n, int lane, uint32_t q,
                                             int ab, int wbest, uint8_t *__restrict__ cw_out,
                                             uint32_t *__restrict__ q_out,
                                             uint8_t *__restrict__ ab_out)
{
    __syncwarp();
    if (lane < wbest)
        sm.cw[sm.pi[sm.best[lane] - 1]] ^= 1;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int i = k * 32 + lane;
        if (i < n)
            cw_out[i] = sm.cw[i];
    }
    if (lane == 0) {
        *q_out = ab == kBlockRange ? 0u : q;
        *ab_out = (uint8_t)ab;
    }
    __syncwarp();
}

/* The scratch of one call (orbg_fitsearch_scratch_bytes): counters, the
 * open list, the list of blocks for the CTA search, the handover records. */
struct FsScratch {
    unsigned long long *cnt; /* [0] stage-1 queue, [1] open blocks, [2] stage-2 queue,
                              * [3] stage-3 queue, [4] blocks for stage 3 */
    uint32_t *open;          /* block of each open slot */
    uint32_t *wide;          /* open slots left to stage 3 */
    unsigned char *hand;
    __host__ __device__ FsScratch(unsigned char *base, int64_t B)
    {
        const size_t list = (4 * (size_t)B + 15) & ~(size_t)15;
        cnt = reinterpret_cast<unsigned long long *>(base);
        open = reinterpret_cast<uint32_t *>(base + 64);
        wide = reinterpret_cast<uint32_t *>(base + 64 + list);
        hand = base + 64 + 2 * list;
    }
};

/* Stage 1, persistent: warps take blocks from an atomic counter. */
template <int K, int W>
__global__ void __launch_bounds__(kWarps * 32, 3) orbg_fitprep_kernel(
    const __grid_constant__ OrbgDeviceCode code, const float *__restrict__ llr, int64_t B,
    uint32_t cap, int lines, int divisible, uint8_t *__restrict__ cw,
    uint32_t *__restrict__ q, uint8_t *__restrict__ ab, int32_t *__restrict__ models,
    unsigned char *__restrict__ scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FsSmem<W> sm(smem + warp * fs_warp_bytes<W>());
    const FsScratch sc(scratch, B);
    const int64_t n = code.n;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0)
            b = atomicAdd(&sc.cnt[0], 1ull);
        b = __shfl_sync(FULL_MASK, b, 0);
        if (b >= (unsigned long long)B)
            break;
        prepare_fitted_block<K, W>(code, llr + (int64_t)b * n, cw + (int64_t)b * n, q + b, ab + b,
                                   models ? models + (int64_t)b * ORBG_FIT_WORDS : nullptr, cap,
                                   lines, divisible, sm, lane, (uint32_t)b, sc.open, &sc.cnt[1],
                                   sc.hand);
    }
}

/* Stage 2, persistent over the open list that stage 1 filled, one warp per
 * block; a block whose search grows past min(kSplit, cap / 4) nodes without
 * a member is left to stage 3. */
template <int K, int W>
__global__ void __launch_bounds__(kWarps * 32, 3) orbg_fitsearch_kernel(
    const __grid_constant__ OrbgDeviceCode code, const float *__restrict__ llr, int64_t B,
    uint32_t cap, uint8_t *__restrict__ cw, uint32_t *__restrict__ q,
    uint8_t *__restrict__ ab, unsigned char *__restrict__ scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FsSmem<W> sm(smem + warp * fs_warp_bytes<W>());
    const FsScratch sc(scratch, B);
    const unsigned long long nopen = sc.cnt[1];
    const int n = code.n;
    const uint32_t split = min(kSplit, cap / 4u);
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0)
            i = atomicAdd(&sc.cnt[2], 1ull);
        i = __shfl_sync(FULL_MASK, i, 0);
        if (i >= nopen)
            break;
        const int64_t b = sc.open[i];
        const auto s0 = load_record<W>(code, llr + b * n, sm, lane,
                                       sc.hand + i * ORBG_FIT_HAND_BYTES);
        uint32_t qb = 0;
        int abb = 0, wbest = 0;
        bool handover = false;
        band_search<W, false>(sm, n, s0, cap, lane, warp, nullptr, split, &qb, &abb, &wbest,
                              &handover);
        if (handover) {
            if (lane == 0)
                sc.wide[atomicAdd(&sc.cnt[4], 1ull)] = (uint32_t)i;
            __syncwarp();
            continue;
        }
        write_fitted<K, W>(sm, n, lane, qb, abb, wbest, cw + b * n, q + b, ab + b);
    }
}

/* Stage 3, persistent over the blocks stage 2 left: all warps of a CTA
 * search one block, each its own class of least positions. */
template <int K, int W>
__global__ void __launch_bounds__(kWarps * 32, 3) orbg_fitsearch_cta_kernel(
    const __grid_constant__ OrbgDeviceCode code, const float *__restrict__ llr, int64_t B,
    uint32_t cap, uint8_t *__restrict__ cw, uint32_t *__restrict__ q,
    uint8_t *__restrict__ ab, unsigned char *__restrict__ scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ FsTeam team;
    __shared__ unsigned long long s_i;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FsSmem<W> sm(smem + warp * fs_warp_bytes<W>());
    const FsScratch sc(scratch, B);
    const unsigned long long nwide = sc.cnt[4];
    const int n = code.n;
    for (;;) {
        if (threadIdx.x == 0) {
            s_i = atomicAdd(&sc.cnt[3], 1ull);
            team.next[0] = 0u;
            team.next[1] = 0u;
        }
        __syncthreads();
        const unsigned long long k = s_i;
        __syncthreads(); /* everyone has read s_i before it changes */
        if (k >= nwide)
            break; /* uniform */
        const uint32_t i = sc.wide[k];
        const int64_t b = sc.open[i];
        const auto s0 = load_record<W>(code, llr + b * n, sm, lane,
                                       sc.hand + (size_t)i * ORBG_FIT_HAND_BYTES);
        uint32_t qb = 0;
        int abb = 0, wbest = 0;
        bool handover = false;
        band_search<W, true>(sm, n, s0, cap, lane, warp, &team, 0u, &qb, &abb, &wbest,
                             &handover);
        if (warp == 0)
            write_fitted<K, W>(sm, n, lane, qb, abb, wbest, cw + b * n, q + b, ab + b);
    }
}

template <int K, int W>
int launch_fitsearch(const OrbgDeviceCode &code, const float *llr, int64_t B, uint32_t cap,
                     int lines, int divisible, uint8_t *cw, uint32_t *q, uint8_t *ab,
                     int32_t *models, unsigned char *scratch, void *stream)
{
    auto k1 = orbg_fitprep_kernel<K, W>;
    auto k2 = orbg_fitsearch_kernel<K, W>;
    auto k3 = orbg_fitsearch_cta_kernel<K, W>;
    const size_t smem = (size_t)fs_warp_bytes<W>() * kWarps;
    int g1 = 0, g2 = 0, g3 = 0;
    int rc = orbg_grid_for((const void *)k1, kWarps * 32, smem, 0, &g1);
    if (rc == 0)
        rc = orbg_grid_for((const void *)k2, kWarps * 32, smem, 0, &g2);
    if (rc == 0)
        rc = orbg_grid_for((const void *)k3, kWarps * 32, smem, 0, &g3);
    if (rc != 0)
        return rc;
    const int64_t need = (B + kWarps - 1) / kWarps;
    if (g1 > need)
        g1 = (int)need;
    if (g2 > need)
        g2 = (int)need;
    if (g3 > B)
        g3 = (int)B;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 64, st);
    if (e != cudaSuccess)
        return (int)e;
    k1<<<g1, kWarps * 32, smem, st>>>(code, llr, B, cap, lines, divisible, cw, q, ab, models,
                                      scratch);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return (int)e;
    k2<<<g2, kWarps * 32, smem, st>>>(code, llr, B, cap, cw, q, ab, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return (int)e;
    k3<<<g3, kWarps * 32, smem, st>>>(code, llr, B, cap, cw, q, ab, scratch);
    return (int)cudaGetLastError();
}

}  // namespace orbg_fitsearch
