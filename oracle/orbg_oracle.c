/*
 * orbg_oracle.c -- plain, single-threaded CPU oracle for basic ORBGRAND.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or helper with the CUDA
 * library; it is written straight from the paper:
 *
 *   Duffy, An, Medard, "Ordered Reliability Bits Guessing Random Additive
 *   Noise Decoding", arXiv 2202.13951.
 *
 * What it computes, step by step, in the paper's order and notation:
 *   1. Hard decision y_i = (sign(LLR_i)+1)/2 and reliability |LLR_i|
 *      (Sec. III-A).  Reading: y_i = 1 iff LLR_i > 0, so +-0 give 0.
 *   2. pi: bit positions sorted by increasing reliability (Sec. III-A);
 *      ties broken by the lower received index.
 *   3. GRAND loop (Algorithm 1): noise effects z are queried in increasing
 *      logistic weight w_L(z) = sum_i i z_i (Eq. lw), Hamming weight
 *      fractionated (Eq. fractionation), each (W, w) set enumerated as
 *      partitions u of W' = W - w(w+1)/2 into w parts in [0, n'=n-w]
 *      (Eq. intpart2) by the Landslide generator (Algorithm 2) with its
 *      Build-mountain routine (Sec. III-C), mapped back by v_i = i + u_i
 *      (Eq. vu) and through pi.  Reading of the arbitrary tie order: w
 *      ascending within a logistic weight, Landslide order within (W, w).
 *   4. Membership of y (+) z is tested by the syndrome H (y (+) z) = 0
 *      (Sec. I: a linear code is checked by a matrix multiply and compare),
 *      evaluated as H y (+) sum of the columns of H that z selects.
 *   5. The first query in the code-book is the decoding; after `cap`
 *      queries without one the decoder abandons (Sec. IV-A) and returns the
 *      hard decision with the abandon flag set.
 *
 * Full ORBGRAND with one line (Sec. III-D, Eq. relest_seg with m = 1,
 * I_1 = n): the sorted position j gets the integer reliability
 * J_0 + beta j, so pattern z has reliability weight
 * J_0 w_H(z) + beta w_L(z), and queries go in increasing reliability weight.
 * For a weight R and a Hamming weight w the logistic weight is fixed,
 * w_L = (R - J_0 w) / beta (Eq. wu_i), and the patterns are the same
 * Landslide sets as above.  Readings: J_0 >= 0 and beta >= 1 (the model's
 * values increase with the position); ties within a reliability weight in
 * the same canonical order as the basic decoder (w ascending, then the
 * Landslide order).  Basic ORBGRAND is the case J_0 = 0, beta = 1 (the
 * paper notes it is the special case of Eq. relest_seg).
 *
 * Piece-wise linear fitting and quantisation (Sec. III-E, Eq. Q and
 * Eq. quant) turn a block's ordered reliabilities into such a model:
 * orbg_oracle_fit, with the readings stated there.
 *
 * Parity pins (tests): brute force over all 2^n patterns for tiny codes,
 * the first queries listed in Sec. III-B, the Fig. 3 / Fig. 5 Landslide
 * examples, closed-form partition counts (for the reliability weight, the
 * coefficients of prod_i (1 + x^(J_0 + beta i))) and decoder invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_N 1024
#define ORC_MAX_WORDS 16 /* syndromes up to 1024 bits */

enum {
    ORC_OK = 0,
    ORC_EINVAL = -1,
    ORC_ENAN = -4,
    ORC_STOP = 1 /* internal: the visitor asked to stop */
};

/* ------------------------------------------------------------------ */
/* Landslide (Algorithm 2) with Build-mountain (Sec. III-C).            */
/* u is 1-based: u[0] is the dummy part used for the initial partition. */
/* ------------------------------------------------------------------ */

typedef int (*orc_visit_fn)(const int *u, int w, void *ctx);

/* Build-mountain from part k: fill u_{k+1..w} with u_k, then push the
 * remaining cells of W' into the right-most parts, each capped at n'. */
static void orc_build_mountain(int *u, int k, int w, int Wp, int np)
{
    int i, sum, Wpp, q, r, room;
    for (i = k + 1; i <= w; i++)
        u[i] = u[k];                      /* step 1 */
    sum = 0;
    for (i = 1; i <= w; i++)
        sum += u[i];
    Wpp = Wp - sum;                       /* step 2 */
    if (Wpp == 0)
        return;                           /* nothing left to place */
    room = np - u[k];                     /* > 0 whenever Wpp > 0 */
    q = Wpp / room;                       /* step 3 */
    r = Wpp % room;
    if (q != 0)
        for (i = w - q + 1; i <= w; i++)
            u[i] = np;                    /* step 4 */
    u[w - q] += r;                        /* step 5 */
}

/* Accumulated drop D(i) = sum_{j=i}^{w} d(j) with d(w) = 0 and
 * d(i) = u_{i+1} - u_i; it telescopes to u_w - u_i. */
static int orc_drop(const int *u, int i, int w)
{
    int j, D = 0;
    for (j = i; j < w; j++)
        D += u[j + 1] - u[j];
    return D;
}

/* Generate every partition of Wp into w non-decreasing parts in [0, np],
 * in Landslide order, calling visit on each.  Requires w >= 1 and
 * 0 <= Wp <= w * np. Returns ORC_STOP if the visitor stopped early. */
int orc_landslide(int Wp, int w, int np, orc_visit_fn visit, void *ctx)
{
    int u[ORC_MAX_N + 1];
    int k, rc;
    if (w < 1 || w > ORC_MAX_N || np < 0 || Wp < 0 || Wp > w * np)
        return ORC_EINVAL;
    memset(u, 0, sizeof(u));
    orc_build_mountain(u, 0, w, Wp, np);  /* dummy part u_0 = 0 */
    rc = visit(u, w, ctx);
    if (rc)
        return rc;
    while (orc_drop(u, 1, w) >= 2) {
        for (k = w; k >= 1; k--)          /* largest k with D(k) >= 2 */
            if (orc_drop(u, k, w) >= 2)
                break;
        u[k] += 1;
        orc_build_mountain(u, k, w, Wp, np);
        rc = visit(u, w, ctx);
        if (rc)
            return rc;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The query order: W ascending; within W, Hamming weight w ascending   */
/* (Eq. fractionation); within (W, w), Landslide order.                 */
/* Patterns are reported as v (1-based positions in the sorted order).  */
/* ------------------------------------------------------------------ */

typedef int (*orc_pattern_fn)(const int *v, int w, void *ctx);

typedef struct {
    orc_pattern_fn fn;
    void *ctx;
} orc_map_ctx;

static int orc_map_u_to_v(const int *u, int w, void *vctx)
{
    orc_map_ctx *m = (orc_map_ctx *)vctx;
    int v[ORC_MAX_N + 1];
    int i;
    for (i = 1; i <= w; i++)
        v[i] = i + u[i];                  /* Eq. vu */
    return m->fn(v + 1, w, m->ctx);
}

/* Walk the patterns of a length-n word in the order of increasing
 * reliability weight R = J0 w_H + beta w_L (Sec. III-D; basic ORBGRAND:
 * J0 = 0, beta = 1, where R is the logistic weight), stopping when the
 * visitor returns non-zero.  The zero pattern (R = 0) comes first. */
static int orc_walk_rw(int n, long J0, long beta, orc_pattern_fn fn, void *ctx)
{
    /* reliability weight of the all-ones pattern */
    long Rmax = J0 * n + beta * ((long)n * (n + 1) / 2);
    long R, L;
    int w, rc;
    orc_map_ctx m;
    m.fn = fn;
    m.ctx = ctx;
    rc = fn(NULL, 0, ctx);               /* R = 0: nothing flipped */
    if (rc)
        return rc;
    for (R = 1; R <= Rmax; R++) {
        for (w = 1; w <= n; w++) {
            if (R - J0 * w < 0)
                break;                    /* larger w only weigh more */
            if ((R - J0 * w) % beta)
                continue;                 /* no integer logistic weight */
            L = (R - J0 * w) / beta;      /* Eq. wu_i with m = 1 */
            /* smallest w_L of weight w is w(w+1)/2 (Eq. fractionation);
             * it grows with w while L shrinks */
            if (L < (long)w * (w + 1) / 2)
                break;
            {
                long Wp = L - (long)w * (w + 1) / 2;
                int np = n - w;
                if (Wp > (long)w * np)
                    continue;             /* no partition fits */
                rc = orc_landslide((int)Wp, w, np, orc_map_u_to_v, &m);
                if (rc)
                    return rc;
            }
        }
    }
    return ORC_OK;
}

/* The basic order: increasing logistic weight. */
static int orc_walk_patterns(int n, orc_pattern_fn fn, void *ctx)
{
    return orc_walk_rw(n, 0, 1, fn, ctx);
}

/* ------------------------------------------------------------------ */
/* Enumeration export, for pinning the order itself.                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int *out;        /* [count][n+1]: w, then v_1..v_w (rest zero) */
    int stride;
    long count, done;
} orc_enum_ctx;

static int orc_enum_visit(const int *v, int w, void *vctx)
{
    orc_enum_ctx *e = (orc_enum_ctx *)vctx;
    int *row, i;
    if (e->done >= e->count)
        return ORC_STOP;
    row = e->out + e->done * e->stride;
    memset(row, 0, sizeof(int) * (size_t)e->stride);
    row[0] = w;
    for (i = 0; i < w; i++)
        row[1 + i] = v[i];
    e->done++;
    return e->done >= e->count ? ORC_STOP : 0;
}

/* First `count` patterns for length n, rows of n+1 ints.  Returns the
 * number written (less than count once the 2^n patterns run out). */
long orbg_oracle_enumerate(int n, long count, int *out)
{
    orc_enum_ctx e;
    if (n < 1 || n > ORC_MAX_N || count < 0 || (count > 0 && !out))
        return ORC_EINVAL;
    if (count == 0)
        return 0;
    e.out = out;
    e.stride = n + 1;
    e.count = count;
    e.done = 0;
    orc_walk_patterns(n, orc_enum_visit, &e);
    return e.done;
}

/* The same for the one-line order of reliability weight J0 w_H + beta w_L. */
long orbg_oracle_enumerate_1line(int n, long J0, long beta, long count, int *out)
{
    orc_enum_ctx e;
    if (n < 1 || n > ORC_MAX_N || J0 < 0 || beta < 1 || count < 0 || (count > 0 && !out))
        return ORC_EINVAL;
    if (count == 0)
        return 0;
    e.out = out;
    e.stride = n + 1;
    e.count = count;
    e.done = 0;
    orc_walk_rw(n, J0, beta, orc_enum_visit, &e);
    return e.done;
}

typedef struct {
    int *out;
    int w;
    long cap, done;
} orc_ls_ctx;

static int orc_ls_visit(const int *u, int w, void *vctx)
{
    orc_ls_ctx *c = (orc_ls_ctx *)vctx;
    int i;
    if (c->done >= c->cap)
        return ORC_STOP;
    for (i = 0; i < w; i++)
        c->out[c->done * w + i] = u[i + 1];
    c->done++;
    return 0;
}

/* Landslide output for (W', w, n'), as rows of w parts u_1..u_w. */
long orbg_oracle_landslide(int Wp, int w, int np, long cap, int *out)
{
    orc_ls_ctx c;
    int rc;
    c.out = out;
    c.w = w;
    c.cap = cap;
    c.done = 0;
    rc = orc_landslide(Wp, w, np, orc_ls_visit, &c);
    if (rc < 0)
        return rc;
    return c.done;
}

typedef struct {
    long *counts;    /* [(Wmax+1) * (n+1)], index W*(n+1) + w */
    int n, Wmax;
} orc_count_ctx;

static int orc_count_visit(const int *v, int w, void *vctx)
{
    orc_count_ctx *c = (orc_count_ctx *)vctx;
    long W = 0;
    int i;
    for (i = 0; i < w; i++)
        W += v[i];                        /* w_L of the pattern (Eq. lw) */
    if (W > c->Wmax)
        return ORC_STOP;                  /* the order is by W: done */
    c->counts[W * (c->n + 1) + w] += 1;
    return 0;
}

/* Number of patterns of each (logistic weight W, Hamming weight w) met by
 * the query order, for W <= Wmax. */
int orbg_oracle_count_by_weight(int n, int Wmax, long *counts)
{
    orc_count_ctx c;
    if (n < 1 || n > ORC_MAX_N || Wmax < 0 || !counts)
        return ORC_EINVAL;
    memset(counts, 0, sizeof(long) * (size_t)(Wmax + 1) * (n + 1));
    c.counts = counts;
    c.n = n;
    c.Wmax = Wmax;
    orc_walk_patterns(n, orc_count_visit, &c);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The decoder (Algorithm 1 with the basic ORBGRAND generator).         */
/* ------------------------------------------------------------------ */

typedef struct {
    int n, r, words;
    const uint64_t *col;     /* col[j*words + x]: column j of H, bit i = H[i][j] */
    const int *pi;           /* pi[p] = received index of the p-th least reliable bit */
    uint64_t s0[ORC_MAX_WORDS];
    uint64_t cap, t, sum_w;
    int hit, hit_w;
    int hit_v[ORC_MAX_N];
} orc_dec_ctx;

static int orc_dec_visit(const int *v, int w, void *vctx)
{
    orc_dec_ctx *d = (orc_dec_ctx *)vctx;
    uint64_t s[ORC_MAX_WORDS];
    int i, x, zero;
    if (d->t >= d->cap)
        return ORC_STOP;                  /* abandon: cap queries made */
    d->t += 1;
    d->sum_w += (uint64_t)w;
    for (x = 0; x < d->words; x++)
        s[x] = d->s0[x];
    for (i = 0; i < w; i++) {
        const uint64_t *c = d->col + (size_t)d->pi[v[i] - 1] * d->words;
        for (x = 0; x < d->words; x++)
            s[x] ^= c[x];
    }
    zero = 1;
    for (x = 0; x < d->words; x++)
        if (s[x])
            zero = 0;
    if (!zero)
        return 0;
    d->hit = 1;
    d->hit_w = w;
    for (i = 0; i < w; i++)
        d->hit_v[i] = v[i];
    return ORC_STOP;
}

/* Sort order of Sec. III-A: increasing reliability |LLR|, lower received
 * index first among equal reliabilities.  A plain insertion sort. */
static void orc_sort_by_reliability(const float *llr, int n, int *pi)
{
    int i, j;
    for (i = 0; i < n; i++)
        pi[i] = i;
    for (i = 1; i < n; i++) {
        int key = pi[i];
        float rk = fabsf(llr[key]);
        j = i - 1;
        while (j >= 0) {
            float rj = fabsf(llr[pi[j]]);
            if (rj > rk || (rj == rk && pi[j] > key)) {
                pi[j + 1] = pi[j];
                j--;
            } else {
                break;
            }
        }
        pi[j + 1] = key;
    }
}

/*
 * Decode one received block.
 *   H       : r x n parity-check matrix, row-major bytes 0/1.
 *   llr     : n log-likelihood ratios, LLR = log f(Y|1)/f(Y|0).
 *   cap     : abandon after this many queries (>= 1).
 *   c_out   : n bytes, the decoding (or the hard decision if abandoned).
 *   q_out   : queries made: the index of the hit, or cap if abandoned.
 *   abandon : 1 if no code-book member was met within cap queries.
 *   sum_w   : sum over the queries made of their Hamming weights.
 *   hit_w / hit_v (optional): the winning pattern, positions 1-based in
 *             the sorted order.
 * Returns 0, or ORC_ENAN if an LLR is NaN, ORC_EINVAL on bad sizes.
 */
/* A query order: walks the patterns of length n, calling fn on each. */
typedef int (*orc_walker)(int n, const void *order, orc_pattern_fn fn, void *ctx);

typedef struct {
    long J0, beta;
} orc_line;

static int orc_walk_line(int n, const void *order, orc_pattern_fn fn, void *ctx)
{
    const orc_line *l = (const orc_line *)order;
    return orc_walk_rw(n, l->J0, l->beta, fn, ctx);
}

static int orc_decode_walk(const uint8_t *H, int n, int r, const float *llr, uint64_t cap,
                           orc_walker walk, const void *order, uint8_t *c_out,
                           uint64_t *q_out, int *abandon, uint64_t *sum_w, int *hit_w,
                           int *hit_v)
{
    static uint64_t col[ORC_MAX_N * ORC_MAX_WORDS];
    int pi[ORC_MAX_N];
    uint8_t y[ORC_MAX_N];
    orc_dec_ctx d;
    int i, j, words;

    if (n < 1 || n > ORC_MAX_N || r < 1 || r > 64 * ORC_MAX_WORDS || cap < 1)
        return ORC_EINVAL;
    for (i = 0; i < n; i++)
        if (isnan(llr[i]))
            return ORC_ENAN;
    words = (r + 63) / 64;
    memset(col, 0, sizeof(uint64_t) * (size_t)n * words);
    for (i = 0; i < r; i++)
        for (j = 0; j < n; j++)
            if (H[(size_t)i * n + j])
                col[(size_t)j * words + i / 64] |= (uint64_t)1 << (i % 64);

    for (i = 0; i < n; i++)
        y[i] = llr[i] > 0.0f ? 1 : 0;     /* (sign(LLR)+1)/2, zero -> 0 */
    orc_sort_by_reliability(llr, n, pi);

    memset(&d, 0, sizeof(d));
    d.n = n;
    d.r = r;
    d.words = words;
    d.col = col;
    d.pi = pi;
    d.cap = cap;
    for (i = 0; i < n; i++)               /* s0 = H y */
        if (y[i])
            for (j = 0; j < words; j++)
                d.s0[j] ^= col[(size_t)i * words + j];

    walk(n, order, orc_dec_visit, &d);

    for (i = 0; i < n; i++)
        c_out[i] = y[i];
    if (d.hit) {
        for (i = 0; i < d.hit_w; i++)
            c_out[pi[d.hit_v[i] - 1]] ^= 1;   /* y (-) z */
        *q_out = d.t;
        *abandon = 0;
    } else {
        *q_out = d.t;                      /* = cap, or 2^n if exhausted */
        *abandon = 1;
    }
    if (sum_w)
        *sum_w = d.sum_w;
    if (hit_w)
        *hit_w = d.hit ? d.hit_w : -1;
    if (hit_v && d.hit)
        for (i = 0; i < d.hit_w; i++)
            hit_v[i] = d.hit_v[i];
    return ORC_OK;
}

/* One block in the one-line order (J0 >= 0, beta >= 1). */
static int orc_decode_rw(const uint8_t *H, int n, int r, const float *llr, uint64_t cap,
                         long J0, long beta, uint8_t *c_out, uint64_t *q_out, int *abandon,
                         uint64_t *sum_w, int *hit_w, int *hit_v)
{
    orc_line l;
    if (J0 < 0 || beta < 1)
        return ORC_EINVAL;
    l.J0 = J0;
    l.beta = beta;
    return orc_decode_walk(H, n, r, llr, cap, orc_walk_line, &l, c_out, q_out, abandon, sum_w,
                           hit_w, hit_v);
}

/* Basic ORBGRAND (the order of increasing logistic weight). */
int orbg_oracle_decode(const uint8_t *H, int n, int r, const float *llr,
                       uint64_t cap, uint8_t *c_out, uint64_t *q_out,
                       int *abandon, uint64_t *sum_w, int *hit_w, int *hit_v)
{
    return orc_decode_rw(H, n, r, llr, cap, 0, 1, c_out, q_out, abandon, sum_w, hit_w, hit_v);
}

/* One-line full ORBGRAND with integer J0 >= 0, beta >= 1 (Sec. III-D). */
int orbg_oracle_decode_1line(const uint8_t *H, int n, int r, const float *llr, uint64_t cap,
                             long J0, long beta, uint8_t *c_out, uint64_t *q_out,
                             int *abandon, uint64_t *sum_w, int *hit_w, int *hit_v)
{
    return orc_decode_rw(H, n, r, llr, cap, J0, beta, c_out, q_out, abandon, sum_w, hit_w,
                         hit_v);
}

/* Batch forms: blocks decoded one after another, same H. */
int orbg_oracle_decode_batch_1line(const uint8_t *H, int n, int r, const float *llr, long B,
                                   uint64_t cap, long J0, long beta, uint8_t *c_out,
                                   uint64_t *q_out, uint8_t *abandon, uint64_t *sum_w)
{
    long b;
    for (b = 0; b < B; b++) {
        int ab = 0, rc;
        uint64_t sw = 0;
        rc = orc_decode_rw(H, n, r, llr + (size_t)b * n, cap, J0, beta,
                           c_out + (size_t)b * n, q_out + b, &ab, &sw, NULL, NULL);
        if (rc)
            return rc;
        abandon[b] = (uint8_t)ab;
        if (sum_w)
            sum_w[b] = sw;
    }
    return ORC_OK;
}

int orbg_oracle_decode_batch(const uint8_t *H, int n, int r, const float *llr,
                             long B, uint64_t cap, uint8_t *c_out,
                             uint64_t *q_out, uint8_t *abandon, uint64_t *sum_w)
{
    return orbg_oracle_decode_batch_1line(H, n, r, llr, B, cap, 0, 1, c_out, q_out, abandon,
                                          sum_w);
}

/* ------------------------------------------------------------------ */
/* Full ORBGRAND with m segments (Sec. III-D).                          */
/* ------------------------------------------------------------------ */

/*
 * The piece-wise linear model (Eq. relest_seg): anchors 0 = I_0 < I_1 <
 * ... < I_m = n; sorted position j in segment i (I_{i-1} < j <= I_i) counts
 * J_{i-1} + beta_i (j - I_{i-1}).  A pattern's reliability weight is the
 * sum over its flipped positions; queries go in increasing weight.  For a
 * weight R (the paper's W) the oracle follows the paper's construction:
 * every split R = W_1 + ... + W_m (Algorithm 3, nested sweeps of W_1 ..
 * W_{m-1}), each W_i checked against its valid partial Hamming weights
 * (Algorithm 4 with Eq. wi_cond, the bounds applying to the partial
 * logistic weight (W_i - w_i J_{i-1}) / beta_i, Eq. wu_i), each segment's
 * partial patterns from Landslide, and their Cartesian product
 * (Eq. cartP).  Readings: beta_i >= 1 and J_{i-1} >= -beta_i, so every
 * position weighs at least 0 (the fitted J_0 of Eq. quant can be as low as
 * -beta_1); the patterns of one weight are visited in the canonical order
 * of the other decoders (Hamming weight ascending, then positions
 * lexicographically), since the paper leaves the order inside a weight
 * free.
 */
#define ORC_MAX_SEG 8

typedef struct {
    int m;
    int I[ORC_MAX_SEG + 1];    /* anchors, I[0] = 0, I[m] = n */
    long J[ORC_MAX_SEG];       /* J_{i-1} of segment i, at index i-1 */
    long beta[ORC_MAX_SEG];    /* beta_i of segment i, at index i-1 */
} orc_model;

/* Patterns of one reliability weight, collected before they are ordered. */
typedef struct {
    int *pos;                  /* all positions, pattern after pattern */
    long *start;               /* start[k]: offset of pattern k in pos */
    int *len;                  /* Hamming weight of pattern k */
    long npat, cap_pat, npos, cap_pos;
} orc_bucket;

static int orc_bucket_add(orc_bucket *b, const int *v, int w)
{
    if (b->npat == b->cap_pat) {
        long c = b->cap_pat ? 2 * b->cap_pat : 1024;
        long *s2 = (long *)realloc(b->start, sizeof(long) * (size_t)c);
        int *l2 = (int *)realloc(b->len, sizeof(int) * (size_t)c);
        if (!s2 || !l2) {
            if (s2) b->start = s2;
            if (l2) b->len = l2;
            return ORC_EINVAL;
        }
        b->start = s2;
        b->len = l2;
        b->cap_pat = c;
    }
    if (b->npos + w > b->cap_pos) {
        long c = b->cap_pos ? 2 * b->cap_pos : 4096;
        int *p2;
        while (c < b->npos + w)
            c *= 2;
        p2 = (int *)realloc(b->pos, sizeof(int) * (size_t)c);
        if (!p2)
            return ORC_EINVAL;
        b->pos = p2;
        b->cap_pos = c;
    }
    b->start[b->npat] = b->npos;
    b->len[b->npat] = w;
    memcpy(b->pos + b->npos, v, sizeof(int) * (size_t)w);
    b->npos += w;
    b->npat += 1;
    return ORC_OK;
}

/* State of one weight's construction: the split, chosen Hamming weights,
 * and the partial patterns fixed so far (absolute positions, ascending). */
typedef struct {
    const orc_model *md;
    int n;
    long W[ORC_MAX_SEG];
    int w[ORC_MAX_SEG];
    int v[ORC_MAX_N];
    int nv;
    int seg;                   /* segment being filled */
    orc_bucket *bucket;
    int err;
} orc_seg_ctx;

static int orc_fill_segment(orc_seg_ctx *c);

/* Landslide visitor for segment c->seg: append its partial pattern and
 * go on with the next segment. */
static int orc_seg_visit(const int *u, int w, void *vctx)
{
    orc_seg_ctx *c = (orc_seg_ctx *)vctx;
    const int i = c->seg, base = c->md->I[i];
    int k, keep = c->nv, rc;
    for (k = 1; k <= w; k++)
        c->v[c->nv++] = base + k + u[k];     /* Eq. vu, shifted into segment i */
    c->seg = i + 1;
    rc = orc_fill_segment(c);
    c->seg = i;
    c->nv = keep;
    return rc;
}

/* Cartesian product over segments seg .. m-1 (Eq. cartP). */
static int orc_fill_segment(orc_seg_ctx *c)
{
    const orc_model *md = c->md;
    const int i = c->seg;
    long L;
    int ni, w;
    if (i == md->m)
        return orc_bucket_add(c->bucket, c->v, c->nv) ? (c->err = 1, ORC_STOP) : 0;
    w = c->w[i];
    if (w == 0)                              /* W_i = 0: nothing flipped here */
    {
        int rc;
        c->seg = i + 1;
        rc = orc_fill_segment(c);
        c->seg = i;
        return rc;
    }
    ni = md->I[i + 1] - md->I[i];
    L = (c->W[i] - (long)w * md->J[i]) / md->beta[i];   /* Eq. wu_i */
    return orc_landslide((int)(L - (long)w * (w + 1) / 2), w, ni - w, orc_seg_visit, c);
}

/* Algorithm 4: is w a valid partial Hamming weight for W_i in segment i
 * (Eq. wi_cond, bounds on the partial logistic weight)? */
static int orc_valid_w(const orc_model *md, int i, long Wi, int w)
{
    const int ni = md->I[i + 1] - md->I[i];
    long rem, L;
    if (w > ni)
        return 0;
    rem = Wi - (long)w * md->J[i];
    if (rem < 0 || rem % md->beta[i])
        return 0;
    L = rem / md->beta[i];
    return L >= (long)w * (w + 1) / 2 && L <= (long)(ni + 1) * w - (long)w * (w + 1) / 2;
}

/* For a complete split: every choice of valid partial Hamming weights. */
static int orc_choose_w(orc_seg_ctx *c, int i)
{
    const orc_model *md = c->md;
    int w, rc;
    if (i == md->m) {
        c->seg = 0;
        c->nv = 0;
        return orc_fill_segment(c);
    }
    if (c->W[i] == 0) {                      /* nothing flipped in segment i */
        c->w[i] = 0;
        rc = orc_choose_w(c, i + 1);
        if (rc)
            return rc;
    }
    for (w = 1; w <= md->I[i + 1] - md->I[i]; w++) {
        if (!orc_valid_w(md, i, c->W[i], w))
            continue;
        c->w[i] = w;
        rc = orc_choose_w(c, i + 1);
        if (rc)
            return rc;
    }
    return 0;
}

/* Algorithm 3: sweep W_1 .. W_{m-1} (W_m is the rest); a non-zero W_i
 * without a valid partial Hamming weight is skipped (Algorithm 4). */
static int orc_split(orc_seg_ctx *c, int i, long left)
{
    const orc_model *md = c->md;
    long Wi;
    int w, ok, rc;
    if (i == md->m - 1) {
        c->W[i] = left;
        Wi = left;
        ok = Wi == 0;
        for (w = 1; !ok && w <= md->I[i + 1] - md->I[i]; w++)
            ok = orc_valid_w(md, i, Wi, w);
        return ok ? orc_choose_w(c, 0) : 0;
    }
    for (Wi = 0; Wi <= left; Wi++) {
        ok = Wi == 0;
        for (w = 1; !ok && w <= md->I[i + 1] - md->I[i]; w++)
            ok = orc_valid_w(md, i, Wi, w);
        if (!ok)
            continue;
        c->W[i] = Wi;
        rc = orc_split(c, i + 1, left - Wi);
        if (rc)
            return rc;
    }
    return 0;
}

/* Canonical order inside one weight: Hamming weight, then positions. */
static const orc_bucket *orc_sort_bucket;
static int orc_cmp_pattern(const void *a, const void *b)
{
    const long ka = *(const long *)a, kb = *(const long *)b;
    const orc_bucket *bk = orc_sort_bucket;
    const int la = bk->len[ka], lb = bk->len[kb];
    const int *pa = bk->pos + bk->start[ka], *pb = bk->pos + bk->start[kb];
    int i;
    if (la != lb)
        return la < lb ? -1 : 1;
    for (i = 0; i < la; i++)
        if (pa[i] != pb[i])
            return pa[i] < pb[i] ? -1 : 1;
    return 0;
}

static int orc_check_model(const orc_model *md, int n)
{
    int i;
    if (md->m < 1 || md->m > ORC_MAX_SEG || md->I[0] != 0 || md->I[md->m] != n)
        return 0;
    for (i = 0; i < md->m; i++)
        if (md->I[i + 1] <= md->I[i] || md->beta[i] < 1 || md->J[i] < -md->beta[i])
            return 0;                        /* every position weight >= 0 */
    return 1;
}

/* Walk every pattern in increasing reliability weight under model md. */
static int orc_walk_model(int n, const orc_model *md, orc_pattern_fn fn, void *ctx)
{
    long Rmax = 0, R, k;
    int i, j, rc = 0;
    orc_bucket b;
    orc_seg_ctx c;
    long *order = NULL;
    for (i = 0; i < md->m; i++)
        for (j = md->I[i] + 1; j <= md->I[i + 1]; j++)
            Rmax += md->J[i] + md->beta[i] * (j - md->I[i]);
    memset(&b, 0, sizeof(b));
    /* R = 0 holds the empty pattern (all W_i = 0, nothing flipped) and,
     * when a segment starts at weight 0, the patterns of zero weight */
    for (R = 0; R <= Rmax && !rc; R++) {
        memset(&c, 0, sizeof(c));
        c.md = md;
        c.n = n;
        c.bucket = &b;
        b.npat = 0;
        b.npos = 0;
        orc_split(&c, 0, R);
        if (c.err) {
            rc = ORC_EINVAL;
            break;
        }
        if (b.npat == 0)
            continue;
        order = (long *)realloc(order, sizeof(long) * (size_t)b.npat);
        if (!order) {
            rc = ORC_EINVAL;
            break;
        }
        for (k = 0; k < b.npat; k++)
            order[k] = k;
        orc_sort_bucket = &b;
        qsort(order, (size_t)b.npat, sizeof(long), orc_cmp_pattern);
        for (k = 0; k < b.npat && !rc; k++)
            rc = fn(b.pos + b.start[order[k]], b.len[order[k]], ctx);
    }
    free(order);
    free(b.pos);
    free(b.start);
    free(b.len);
    return rc < 0 ? rc : ORC_OK;
}

static void orc_fill_model(orc_model *md, int m, const int *anchors, const long *J,
                           const long *beta, int n)
{
    int i;
    memset(md, 0, sizeof(*md));
    md->m = m;
    md->I[0] = 0;
    for (i = 1; i < m && i < ORC_MAX_SEG; i++)
        md->I[i] = anchors[i - 1];
    if (m >= 1 && m <= ORC_MAX_SEG)
        md->I[m] = n;
    for (i = 0; i < m && i < ORC_MAX_SEG; i++) {
        md->J[i] = J[i];
        md->beta[i] = beta[i];
    }
}

/*
 * m-segment full ORBGRAND (Sec. III-D).
 *   anchors: I_1 .. I_{m-1} (I_0 = 0 and I_m = n implied), increasing;
 *   J:       J_0 .. J_{m-1};  beta: beta_1 .. beta_m.
 * Other arguments as orbg_oracle_decode_batch / _enumerate.
 */
long orbg_oracle_enumerate_mline(int n, int m, const int *anchors, const long *J,
                                 const long *beta, long count, int *out)
{
    orc_model md;
    orc_enum_ctx e;
    if (n < 1 || n > ORC_MAX_N || count < 0 || (count > 0 && !out))
        return ORC_EINVAL;
    orc_fill_model(&md, m, anchors, J, beta, n);
    if (!orc_check_model(&md, n))
        return ORC_EINVAL;
    if (count == 0)
        return 0;
    e.out = out;
    e.stride = n + 1;
    e.count = count;
    e.done = 0;
    orc_walk_model(n, &md, orc_enum_visit, &e);
    return e.done;
}

static int orc_walk_model_fn(int n, const void *order, orc_pattern_fn fn, void *ctx)
{
    return orc_walk_model(n, (const orc_model *)order, fn, ctx);
}

int orbg_oracle_decode_batch_mline(const uint8_t *H, int n, int r, const float *llr, long B,
                                   uint64_t cap, int m, const int *anchors, const long *J,
                                   const long *beta, uint8_t *c_out, uint64_t *q_out,
                                   uint8_t *abandon, uint64_t *sum_w)
{
    orc_model md;
    long b;
    if (n < 1 || n > ORC_MAX_N)
        return ORC_EINVAL;
    orc_fill_model(&md, m, anchors, J, beta, n);
    if (!orc_check_model(&md, n))
        return ORC_EINVAL;
    for (b = 0; b < B; b++) {
        int ab = 0, rc;
        uint64_t sw = 0;
        rc = orc_decode_walk(H, n, r, llr + (size_t)b * n, cap, orc_walk_model_fn, &md,
                             c_out + (size_t)b * n, q_out + b, &ab, &sw, NULL, NULL);
        if (rc)
            return rc;
        abandon[b] = (uint8_t)ab;
        if (sum_w)
            sum_w[b] = sw;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Piece-wise linear fitting and quantisation (Sec. III-E).             */
/* ------------------------------------------------------------------ */

#define ORC_FIT_MAX 16777216.0 /* 2^24: largest quantised slope or offset */

static long orc_round(double x)              /* [ ]: half away from zero */
{
    return (long)(x < 0 ? -floor(-x + 0.5) : floor(x + 0.5));
}

/*
 * Fit `lines` (1..ORC_MAX_SEG) lines to the block's ordered reliability
 * curve L_1 <= ... <= L_n (|LLR| sorted as in Sec. III-A) and quantise
 * them (Eq. Q, Eq. quant).  Anchors start at the edge index 1 and the
 * centre floor(n/2); each further anchor goes into the first interval
 * (the high-curvature edge), at the largest vertical gap between that
 * interval's chord and the curve (smallest index on ties); the search
 * stops early when the interval has no inner index or no gap.  The line
 * ending at the centre is extended to n.  With the anchors a_0 = 1 < a_1
 * < ... < a_m = centre: I_i = a_i for 0 < i < m, I_m = n; slope s_1 =
 * (L_{a_1} - L_1)/(a_1 - 1), s_i = (L_{a_i} - L_{a_{i-1}})/(a_i - a_{i-1});
 * Q = min s_i; beta_i = [s_i / Q]; J_0 = [L_1 / Q] - beta_1;
 * J_i = [L_{I_i} / Q].  divisible != 0: J_{i-1} <- [J_{i-1} / beta_i] beta_i.
 * n < 4, Q <= 0 (a flat stretch), or a ratio s_i / Q or L_{I_i} / Q
 * (i < m) that is not finite or exceeds 2^24: the basic model, one line
 * with J_0 = 0, beta_1 = 1.  Outputs: *m, anchors I_1 .. I_{m-1}, J_0 ..
 * J_{m-1}, beta_1 .. beta_m.
 */
int orbg_oracle_fit(const float *llr, int n, int lines, int divisible, int *m_out,
                    int *anchors, long *J, long *beta)
{
    int pi[ORC_MAX_N];
    double L[ORC_MAX_N + 1];
    int a[ORC_MAX_SEG + 1], na, i, j, k;
    double s[ORC_MAX_SEG], Q;
    if (n < 1 || n > ORC_MAX_N || lines < 1 || lines > ORC_MAX_SEG || !m_out || !J || !beta)
        return ORC_EINVAL;
    for (i = 0; i < n; i++)
        if (isnan(llr[i]))
            return ORC_ENAN;
    orc_sort_by_reliability(llr, n, pi);
    for (j = 1; j <= n; j++)
        L[j] = fabs((double)llr[pi[j - 1]]);
    *m_out = 1;
    J[0] = 0;
    beta[0] = 1;
    if (n < 4)
        return ORC_OK;
    a[0] = 1;
    a[1] = n / 2;
    na = 2;
    while (na - 1 < lines) {                  /* one more line: split [a_0, a_1] */
        const int lo = a[0], hi = a[1];
        int best = -1;
        double gap = 0.0;
        for (j = lo + 1; j < hi; j++) {
            const double chord = L[lo] + (L[hi] - L[lo]) * (double)(j - lo) / (double)(hi - lo);
            const double g = fabs(chord - L[j]);
            if (g > gap) {
                gap = g;
                best = j;
            }
        }
        if (best < 0)
            break;                            /* no inner index or no gap */
        for (k = na; k > 1; k--)
            a[k] = a[k - 1];
        a[1] = best;
        na++;
    }
    {
        const int m = na - 1;
        s[0] = (L[a[1]] - L[1]) / (double)(a[1] - 1);
        for (i = 2; i <= m; i++)
            s[i - 1] = (L[a[i]] - L[a[i - 1]]) / (double)(a[i] - a[i - 1]);
        Q = s[0];
        for (i = 1; i < m; i++)
            if (s[i] < Q)
                Q = s[i];                     /* Eq. Q */
        if (!(Q > 0.0))
            return ORC_OK;                    /* a flat stretch: basic model */
        for (i = 0; i < m; i++)
            if (!(s[i] / Q <= ORC_FIT_MAX) || !(L[a[i]] / Q <= ORC_FIT_MAX))
                return ORC_OK;                /* out of range: basic model */
        for (i = 0; i < m; i++)
            beta[i] = orc_round(s[i] / Q);    /* Eq. quant */
        J[0] = orc_round(L[1] / Q) - beta[0];
        for (i = 1; i < m; i++)
            J[i] = orc_round(L[a[i]] / Q);
        if (divisible)
            for (i = 0; i < m; i++)
                J[i] = orc_round((double)J[i] / (double)beta[i]) * beta[i];
        for (i = 1; i < m; i++)
            if (anchors)
                anchors[i - 1] = a[i];
        *m_out = m;
    }
    return ORC_OK;
}

/*
 * Full ORBGRAND per block (the flow of Fig. flow_char): fit and quantise
 * each block's own model (orbg_oracle_fit), then query in increasing
 * reliability weight under it (orbg_oracle_decode_batch_mline's walk).
 * Outputs as orbg_oracle_decode_batch_1line.
 */
int orbg_oracle_decode_batch_fit(const uint8_t *H, int n, int r, const float *llr, long B,
                                 uint64_t cap, int lines, int divisible, uint8_t *c_out,
                                 uint64_t *q_out, uint8_t *abandon, uint64_t *sum_w)
{
    long b;
    if (n < 1 || n > ORC_MAX_N || lines < 1 || lines > ORC_MAX_SEG)
        return ORC_EINVAL;
    for (b = 0; b < B; b++) {
        const float *x = llr + (size_t)b * n;
        int m = 1, anchors[ORC_MAX_SEG], ab = 0, rc;
        long J[ORC_MAX_SEG], beta[ORC_MAX_SEG];
        uint64_t sw = 0;
        orc_model md;
        rc = orbg_oracle_fit(x, n, lines, divisible, &m, anchors, J, beta);
        if (rc)
            return rc;
        orc_fill_model(&md, m, anchors, J, beta, n);
        if (!orc_check_model(&md, n))
            return ORC_EINVAL;
        rc = orc_decode_walk(H, n, r, x, cap, orc_walk_model_fn, &md, c_out + (size_t)b * n,
                             q_out + b, &ab, &sw, NULL, NULL);
        if (rc)
            return rc;
        abandon[b] = (uint8_t)ab;
        if (sum_w)
            sum_w[b] = sw;
    }
    return ORC_OK;
}

/* The permutation of Sec. III-A alone, for tests. */
int orbg_oracle_sort(const float *llr, int n, int *pi)
{
    if (n < 1 || n > ORC_MAX_N)
        return ORC_EINVAL;
    orc_sort_by_reliability(llr, n, pi);
    return ORC_OK;
}
