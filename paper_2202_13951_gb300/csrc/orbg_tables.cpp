/*
 * orbg_tables.cpp -- host-side tables of the query order, and GF(2) helpers.
 *
 * The order is basic ORBGRAND's (Sec. III-B): logistic weight
 * W = sum_i v_i over the flipped sorted positions v (Eq. lw) ascending,
 * split by Hamming weight w (Eq. fractionation) ascending, and inside one
 * (W, w) the distinct-part partitions v_1 < ... < v_w <= n of W (Eq.
 * intpart) in lexicographic order, the order Algorithm 2 (Landslide)
 * generates.  This file enumerates that order directly, as lexicographic
 * prefixes followed by a run of pairs or of triples (see orbg_internal.h),
 * not with Landslide.  The one-line order of full ORBGRAND (Sec. III-D)
 * reorders the same (W, w) classes; the m-segment order (Eq. relest_seg)
 * is built pattern by pattern (orbg_build_tables_model).
 */
#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>

#include "orbg_internal.h"

namespace {

/* Pairs a < b <= n (1-based) with a + b = S and a >= lo: a in
 * [max(lo, S - n), (S - 1) / 2]. */
inline int pair_lo(int S, int lo, int n) { return std::max(lo, S - n); }
inline int pair_hi(int S) { return (S - 1) / 2; }

/* Triples c < a < b <= n with c + a + b = S3 and c >= lo: the c that admit a
 * pair form [max(lo, S3 - (2n - 1)), (S3 - 3) / 3]. */
inline int trip_c_lo(int S3, int lo, int n) { return std::max(lo, S3 - (2 * n - 1)); }
inline int trip_c_hi(int S3) { return (S3 - 3) / 3; }

/* Longest chunk a triple run starting at query t is cut into: short early
 * in the order (a warp step over 32 chunks should not overshoot a hit by
 * much) and long deep in it (the per-chunk setup is amortised). */
int chunk_len(uint64_t t)
{
    const uint64_t c = t / 512;
    return (int)(c < 8 ? 8 : c > 255 ? 255 : c);
}

struct Builder {
    int n;
    bool cta;                      /* build the CTA table (triple runs) */
    int s3max = 0;                 /* triple sums covered by X3 */
    const std::vector<uint32_t> *x3off = nullptr; /* first X3 index of each sum */
    uint64_t t = 1;                /* next query index */
    std::vector<OrbgRun> cls;      /* runs of the current (W, w) class */
    int pre[64];
    bool overflow = false;
    long J0 = 0, beta = 1;         /* the line: reliability J0 + beta j */

    OrbgRun blank(int kind, int npre) {
        OrbgRun r;
        std::memset(&r, 0, sizeof(r));
        r.tstart = (uint32_t)t;
        r.kind = (uint8_t)kind;
        r.npre = (uint8_t)npre;
        for (int i = 0; i < npre; i++) {
            overflow |= pre[i] > 255; /* a byte holds positions 1..255 */
            r.pre[i] = (uint8_t)pre[i]; /* 1-based; 0 marks an unused slot */
        }
        return r;
    }

    void emit(OrbgRun r, uint64_t count) {
        if (count > 0xFFFF || count == 0) {
            overflow |= count > 0xFFFF;
            return;
        }
        r.count = (uint16_t)count;
        cls.push_back(r);
        t += count;
    }

    void single(int np) { emit(blank(ORBG_RUN_SINGLE, np), 1); }

    /* pairs of sum S after a prefix of `depth` positions ending at q */
    void pairs(int depth, int q, int S) {
        const int lo = pair_lo(S, q + 1, n), hi = pair_hi(S);
        if (lo > hi)
            return;
        OrbgRun r = blank(ORBG_RUN_PAIRS, depth);
        r.aux = (uint32_t)S | ((uint32_t)lo << 8);
        emit(r, (uint64_t)(hi - lo + 1));
    }

    /* triples of sum S3 after a prefix ending at q: one X3 range, chunked */
    void triples(int depth, int q, int S3) {
        const int c_lo = trip_c_lo(S3, q + 1, n), c_hi = trip_c_hi(S3);
        if (c_lo > c_hi)
            return;
        /* X3 index of the first triple with c >= c_lo, and the range length */
        uint32_t x = (*x3off)[S3];
        for (int c = trip_c_lo(S3, 1, n); c < c_lo; c++)
            x += (uint32_t)(pair_hi(S3 - c) - pair_lo(S3 - c, c + 1, n) + 1);
        uint64_t total = 0;
        for (int c = c_lo; c <= c_hi; c++)
            total += (uint64_t)(pair_hi(S3 - c) - pair_lo(S3 - c, c + 1, n) + 1);
        while (total > 0) {
            const uint64_t len = std::min<uint64_t>(total, (uint64_t)chunk_len(t));
            OrbgRun r = blank(ORBG_RUN_TRIPLES, depth);
            r.aux = x;
            emit(r, len);
            x += (uint32_t)len;
            total -= len;
        }
    }

    /* Prefixes of `need` more positions, each >= lo, with `rem` left for
     * them and the final `tail` (2 = pair, 3 = triple) positions. */
    void prefixes(int depth, int need, int lo, int rem, int tail) {
        if (need == 0) {
            if (tail == 2)
                pairs(depth, lo - 1, rem);
            else
                triples(depth, lo - 1, rem);
            return;
        }
        const int m = need - 1 + tail; /* positions after v, all above it */
        for (int v = lo; v <= n; v++) {
            long min_rest = (long)m * v + (long)m * (m + 1) / 2;
            long max_rest = (long)m * n - (long)m * (m - 1) / 2;
            if (v + min_rest > rem)
                break;
            if (v + max_rest < rem)
                continue;
            pre[depth] = v;
            prefixes(depth + 1, need - 1, v + 1, rem - v, tail);
        }
    }

    void flush(std::vector<OrbgRun> *out) {
        /* longest runs first; equal lengths keep the query order */
        std::stable_sort(cls.begin(), cls.end(),
                         [](const OrbgRun &a, const OrbgRun &b) {
                             return a.count > b.count;
                         });
        out->insert(out->end(), cls.begin(), cls.end());
        cls.clear();
    }

    /* The whole order up to the class holding query `cap`: classes (W, w)
     * of logistic weight W and Hamming weight w in increasing reliability
     * weight R = J0 w + beta W (one-line full ORBGRAND, Sec. III-D; basic
     * ORBGRAND is J0 = 0, beta = 1, R = W), w ascending within R. */
    int build(uint64_t cap, std::vector<OrbgRun> *out, uint64_t *patterns, int *wdeep) {
        t = 1;
        single(0); /* R = 0: the zero pattern */
        flush(out);
        *wdeep = 0;
        const long Rlast = J0 * n + beta * ((long)n * (n + 1) / 2);
        for (long R = 1; R <= Rlast && t <= cap; R++) {
            for (int w = 1; w <= n; w++) {
                if (R - J0 * w < 0)
                    break;                 /* larger w only weigh more */
                if ((R - J0 * w) % beta)
                    continue;              /* no integer logistic weight */
                const long W = (R - J0 * w) / beta;
                if (W < (long)w * (w + 1) / 2)
                    break;                 /* below the lightest w-subset */
                if (W > (long)w * (w + 1) / 2 + (long)w * (n - w))
                    continue;              /* above the heaviest w-subset */
                if (W > ORBG_MAX_LOGISTIC)
                    return -2;
                if (w == 1) {
                    if (W <= n) {
                        pre[0] = (int)W;
                        single(1);
                    }
                } else if (cta && w >= 3) {
                    /* triple runs where the prefix leaves a sum inside X3,
                     * pair runs (prefix extended by c) where it does not */
                    if (w - 2 > ORBG_RUN_MAX_PRE)
                        return -2;
                    prefixes_split(0, w - 3, 1, (int)W);
                } else {
                    if (w - 2 > ORBG_RUN_MAX_PRE)
                        return -2;
                    prefixes(0, w - 2, 1, (int)W, 2);
                }
                flush(out);
                *wdeep = std::max(*wdeep, (int)W);
            }
        }
        *patterns = t - 1;
        return overflow ? -2 : 0;
    }

    /* CTA table, w >= 3: (w-3)-prefixes in lexicographic order; each one's
     * triples become an X3 range if their sum fits X3, else the prefix is
     * extended by every valid c (in order) and the pairs after it form
     * pair runs -- the same patterns in the same order. */
    void prefixes_split(int depth, int need, int lo, int rem) {
        if (need == 0) {
            if (rem <= s3max) {
                triples(depth, lo - 1, rem);
            } else {
                const int c_lo = trip_c_lo(rem, lo, n), c_hi = trip_c_hi(rem);
                for (int c = c_lo; c <= c_hi; c++) {
                    pre[depth] = c;
                    pairs(depth + 1, c, rem - c);
                }
            }
            return;
        }
        const int m = need - 1 + 3;
        for (int v = lo; v <= n; v++) {
            long min_rest = (long)m * v + (long)m * (m + 1) / 2;
            long max_rest = (long)m * n - (long)m * (m - 1) / 2;
            if (v + min_rest > rem)
                break;
            if (v + max_rest < rem)
                continue;
            pre[depth] = v;
            prefixes_split(depth + 1, need - 1, v + 1, rem - v);
        }
    }
};

/* reach[g]: the largest query index in groups 0..g; and the first group
 * holding a query beyond `nflat` */
void reaches(const std::vector<OrbgRun> &runs, uint32_t nflat, std::vector<uint32_t> *out,
             uint32_t *flat_group)
{
    const size_t nr = runs.size();
    const size_t ng = (nr + ORBG_GROUP - 1) / ORBG_GROUP;
    out->assign(ng, 0u);
    uint32_t reach = 0;
    *flat_group = (uint32_t)ng;
    for (size_t g = 0; g < ng; g++) {
        bool beyond = false;
        for (size_t i = g * ORBG_GROUP; i < std::min(nr, (g + 1) * ORBG_GROUP); i++) {
            const uint32_t last = runs[i].tstart + runs[i].count - 1u;
            reach = std::max(reach, last);
            beyond |= last > nflat;
        }
        (*out)[g] = reach;
        if (beyond && *flat_group == ng)
            *flat_group = (uint32_t)g;
    }
}

void floors(const std::vector<OrbgRun> &runs, std::vector<uint32_t> *out)
{
    const size_t nr = runs.size();
    const size_t ng = (nr + ORBG_GROUP - 1) / ORBG_GROUP;
    out->assign(ng, 0xFFFFFFFFu);
    uint32_t floor = 0xFFFFFFFFu;
    for (size_t g = ng; g-- > 0;) {
        for (size_t i = g * ORBG_GROUP; i < std::min(nr, (g + 1) * ORBG_GROUP); i++)
            floor = std::min(floor, runs[i].tstart);
        (*out)[g] = floor;
    }
}

/* Group floors and reaches, the flat table and the CTA table's triple
 * needs, from the two run tables (and X3) of `out`. */
void finish_tables(OrbgTables *out)
{
    const uint64_t patterns = out->patterns;
    const int s3max = out->s3max;
    floors(out->runs, &out->group_floor);
    floors(out->runs_cta, &out->group_floor_cta);
    /* flat table: the leading patterns of weight <= ORBG_FLAT_POS, at most
     * ORBG_FLAT_MAX of them, in query order */
    std::vector<std::vector<int>> first((size_t)std::min<uint64_t>(patterns, ORBG_FLAT_MAX));
    std::vector<int> v(64);
    for (const OrbgRun &r : out->runs)
        for (int j = 0; j < r.count; j++) {
            const uint64_t t = (uint64_t)r.tstart + (uint64_t)j;
            if (t <= first.size()) {
                const int w = orbg_run_pattern(r, j, out->trip.data(), v.data());
                first[t - 1].assign(v.begin(), v.begin() + w);
            }
        }
    uint32_t nflat = 0;
    while (nflat < first.size() && first[nflat].size() <= ORBG_FLAT_POS)
        nflat++;
    /* per step of 32 patterns: the ranks it needs in sorted order (its
     * largest position, non-decreasing over the steps; the table ends before
     * the first step needing more than ORBG_FLAT_RANKS) and its largest
     * Hamming weight */
    std::vector<uint8_t> need;
    {
        int mx = 0;
        uint32_t keep = 0;
        for (uint32_t base = 0; base < nflat; base += 32) {
            const uint32_t end = std::min<uint32_t>(nflat, base + 32);
            int wmax = 0;
            for (uint32_t t = base; t < end; t++) {
                wmax = std::max(wmax, (int)first[t].size());
                for (int p : first[t])
                    mx = std::max(mx, p);
            }
            if (mx > ORBG_FLAT_RANKS)
                break;
            need.push_back((uint8_t)(mx | wmax << 5));
            keep = end;
        }
        nflat = keep;
    }
    out->nflat = nflat;
    out->flat.assign((size_t)std::max<uint32_t>(nflat, 1) * 8, 0);
    for (uint32_t t = 0; t < nflat; t++) {
        uint8_t *e = &out->flat[(size_t)t * 8];
        for (size_t i = 0; i < first[t].size(); i++)
            e[i] = (uint8_t)first[t][i];
        e[7] = need[t / 32];
    }
    reaches(out->runs, nflat, &out->reach, &out->flat_group);
    reaches(out->runs_cta, nflat, &out->reach_cta, &out->flat_group_cta);
    /* largest triple sum read by the runs of groups <= g: an X3 index falls
     * in the sum whose range holds it */
    {
        const size_t nr = out->runs_cta.size();
        const size_t ng = (nr + ORBG_GROUP - 1) / ORBG_GROUP;
        out->s3_cta.assign(ng, 0);
        int s3 = 0;
        for (size_t g = 0; g < ng; g++) {
            for (size_t i = g * ORBG_GROUP; i < std::min(nr, (g + 1) * ORBG_GROUP); i++) {
                const OrbgRun &r = out->runs_cta[i];
                if (r.kind != ORBG_RUN_TRIPLES)
                    continue;
                const uint32_t last = r.aux + r.count - 1u;
                int S = 6;
                while (S < s3max && out->x3off[S + 1] <= last)
                    S++;
                s3 = std::max(s3, S);
            }
            out->s3_cta[g] = (uint8_t)s3;
        }
    }
}

}  // namespace

int orbg_build_tables(int n, uint64_t cap, OrbgTables *out, long J0, long beta)
{
    if (n < 1 || n > 256 || cap < 1 || J0 < 0 || beta < 1 || J0 > ORBG_MAX_LINE ||
        beta > ORBG_MAX_LINE)
        return -1;
    /* warp table */
    Builder bw;
    bw.n = n;
    bw.cta = false;
    bw.J0 = J0;
    bw.beta = beta;
    out->runs.clear();
    uint64_t patterns = 0;
    int wdeep = 0;
    int rc = bw.build(cap, &out->runs, &patterns, &wdeep);
    if (rc)
        return rc;
    out->patterns = patterns;
    out->wmax_logistic = wdeep;
    if (patterns >= 0xFFFFFFFFull)
        return -3;
    /* X3: every triple c < a < b <= n by sum (<= the table's depth, within
     * ORBG_X3_MAX entries), then c, then a */
    std::vector<uint32_t> x3off(ORBG_MAX_LOGISTIC + 2, 0);
    out->trip.clear();
    int s3max = 0;
    for (int S3 = 6; S3 <= wdeep; S3++) {
        size_t cnt = 0;
        for (int c = trip_c_lo(S3, 1, n); c <= trip_c_hi(S3); c++)
            cnt += (size_t)(pair_hi(S3 - c) - pair_lo(S3 - c, c + 1, n) + 1);
        if (out->trip.size() + cnt > ORBG_X3_MAX)
            break;
        x3off[S3] = (uint32_t)out->trip.size();
        for (int c = trip_c_lo(S3, 1, n); c <= trip_c_hi(S3); c++)
            for (int a = pair_lo(S3 - c, c + 1, n); a <= pair_hi(S3 - c); a++)
                out->trip.push_back((uint32_t)(c - 1) | ((uint32_t)(a - 1) << 8) |
                                    ((uint32_t)(S3 - c - a - 1) << 16));
        s3max = S3;
    }
    out->s3max = s3max;
    out->x3off.assign(x3off.begin(), x3off.begin() + (s3max + 2));
    out->x3off[s3max + 1] = (uint32_t)out->trip.size();
    /* CTA table */
    Builder bc;
    bc.n = n;
    bc.cta = true;
    bc.J0 = J0;
    bc.beta = beta;
    bc.s3max = s3max;
    bc.x3off = &x3off;
    out->runs_cta.clear();
    uint64_t patterns_c = 0;
    int wdeep_c = 0;
    rc = bc.build(cap, &out->runs_cta, &patterns_c, &wdeep_c);
    if (rc)
        return rc;
    if (patterns_c != patterns)
        return -5;
    finish_tables(out);
    return 0;
}

namespace {

/*
 * m-segment full ORBGRAND (Sec. III-D, Eq. relest_seg): position j of
 * segment i, I_{i-1} < j <= I_i, weighs rho_j = J_{i-1} + beta_i (j -
 * I_{i-1}) >= 0, and patterns come in increasing reliability weight (the
 * sum of rho over the flipped positions), then Hamming weight, then
 * positions lexicographically.
 *
 * Patterns of increasing weight come from a best-first walk over subsets
 * of the positions ranked by weight, x_0 <= x_1 <= ...: a subset whose
 * highest rank is k leads to the subset with rank k + 1 added and to the
 * one with rank k replaced by k + 1.  Every non-empty subset is reached
 * exactly once, from {0}, and never weighs less than the subset it comes
 * from, so a min-heap pops weights in order.  All subsets of one weight R
 * are collected, ordered by (w, positions) and cut into runs: consecutive
 * patterns (p, a, b), (p, a + 1, b - 1), ... with one prefix p become one
 * pair run, and consecutive (p, a, b), (p, a + da, b - db), ... (a pair
 * across two segments whose slopes balance, beta da = beta' db) one strided
 * pair run; the rest are single runs.
 */
struct ModelBuilder {
    Builder b;                           /* run records and class flush */
    std::vector<long> x;                 /* weights by rank, lightest first */
    std::vector<int> pos;                /* 1-based position of each rank */
    struct Node {
        int parent;                      /* the subset without `rank`, -1 = empty */
        int rank;
    };
    std::vector<Node> nodes;

    /* one weight's patterns, back to back: pattern q is pos_all[start[q] ..
     * start[q] + len[q]) ascending */
    std::vector<int> pos_all;
    std::vector<uint32_t> start;
    std::vector<uint16_t> len;
    std::vector<uint32_t> order;  /* pattern indices in (w, positions) order */

    int build(uint64_t cap, std::vector<OrbgRun> *out, uint64_t *patterns) {
        const int n = b.n;
        typedef std::pair<long, int> Item;   /* (weight, node) */
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
        nodes.clear();
        nodes.push_back(Node{-1, 0});
        heap.push(Item(x[0], 0));
        b.t = 1;
        long R = 0;
        bool first = true;
        while (b.t <= cap && (first || !heap.empty())) {
            pos_all.clear();
            start.clear();
            len.clear();
            if (first) {                 /* the empty pattern, weight 0 */
                start.push_back(0);
                len.push_back(0);
            } else {
                R = heap.top().first;
            }
            first = false;
            while (!heap.empty() && heap.top().first == R) {
                const int id = heap.top().second;
                heap.pop();
                const int k = nodes[id].rank;
                if (k + 1 < n) {
                    const int par = nodes[id].parent;
                    nodes.push_back(Node{id, k + 1});
                    heap.push(Item(R + x[k + 1], (int)nodes.size() - 1));
                    nodes.push_back(Node{par, k + 1});
                    heap.push(Item(R - x[k] + x[k + 1], (int)nodes.size() - 1));
                }
                const size_t s0 = pos_all.size();
                for (int q = id; q >= 0; q = nodes[q].parent)
                    pos_all.push_back(pos[nodes[q].rank]);
                std::sort(pos_all.begin() + (long)s0, pos_all.end());
                start.push_back((uint32_t)s0);
                len.push_back((uint16_t)(pos_all.size() - s0));
            }
            if (nodes.size() > (size_t)1 << 30 || pos_all.size() > 0xFFFFFFFFull)
                return -2;
            order.resize(start.size());
            for (size_t q = 0; q < order.size(); q++)
                order[q] = (uint32_t)q;
            std::sort(order.begin(), order.end(), [this](uint32_t p, uint32_t q) {
                if (len[p] != len[q])
                    return len[p] < len[q];
                const int *a = pos_all.data() + start[p], *c = pos_all.data() + start[q];
                return std::lexicographical_compare(a, a + len[p], c, c + len[q]);
            });
            if (emit_bucket(out))
                return -2;
        }
        *patterns = b.t - 1;
        return b.overflow ? -2 : 0;
    }

    const int *pat(size_t i) const { return pos_all.data() + start[order[i]]; }
    int wof(size_t i) const { return len[order[i]]; }

    /* Runs of one weight's patterns, class by class (one class per w). */
    int emit_bucket(std::vector<OrbgRun> *out) {
        const size_t np = order.size();
        size_t i = 0;
        while (i < np) {
            const int w = wof(i);
            size_t end = i;
            while (end < np && wof(end) == w)
                end++;
            if (w - 2 > ORBG_RUN_MAX_PRE)
                return -2;
            for (size_t s = i; s < end;) {
                const int *v = pat(s);
                size_t e = s + 1;
                if (w >= 2) {
                    const int a = v[w - 2], bb = v[w - 1];
                    /* the step from this pattern to the next, if it keeps the prefix */
                    int da = 1, db = 1;
                    if (e < end && std::equal(v, v + w - 2, pat(e))) {
                        da = pat(e)[w - 2] - a;
                        db = bb - pat(e)[w - 1];
                    }
                    if (da < 1 || db < 1 || da > 255 || db > 255)
                        da = db = 1;
                    while (e < end && std::equal(v, v + w - 2, pat(e)) &&
                           pat(e)[w - 2] == a + da * (int)(e - s) &&
                           pat(e)[w - 1] == bb - db * (int)(e - s))
                        e++;
                    if (da == 1 && db == 1 && a + bb <= 255) {
                        for (int q = 0; q < w - 2; q++)
                            b.pre[q] = v[q];
                        OrbgRun r = b.blank(ORBG_RUN_PAIRS, w - 2);
                        r.aux = (uint32_t)(a + bb) | ((uint32_t)a << 8);
                        b.emit(r, (uint64_t)(e - s));
                        s = e;
                        continue;
                    }
                    if (e - s >= 2 && bb <= 255) {
                        for (int q = 0; q < w - 2; q++)
                            b.pre[q] = v[q];
                        OrbgRun r = b.blank(ORBG_RUN_STRIDE, w - 2);
                        r.aux = (uint32_t)a | ((uint32_t)bb << 8) | ((uint32_t)da << 16) |
                                ((uint32_t)db << 24);
                        b.emit(r, (uint64_t)(e - s));
                        s = e;
                        continue;
                    }
                }
                if (w > ORBG_RUN_MAX_PRE)
                    return -2;
                for (size_t q = s; q < e; q++) {
                    for (int z = 0; z < w; z++)
                        b.pre[z] = pat(q)[z];
                    b.single(w);
                }
                s = e;
            }
            b.flush(out);
            i = end;
        }
        return 0;
    }
};

}  // namespace

int orbg_build_tables_model(int n, uint64_t cap, const OrbgModel &md, OrbgTables *out)
{
    if (n < 1 || n > 256 || cap < 1 || md.m < 1 || md.m > ORBG_MAX_SEG || md.I[0] != 0 ||
        md.I[md.m] != n)
        return -1;
    for (int i = 0; i < md.m; i++)
        if (md.I[i + 1] <= md.I[i] || md.beta[i] < 1 || md.beta[i] > ORBG_MAX_MODEL ||
            md.J[i] < -md.beta[i] || md.J[i] > ORBG_MAX_MODEL)
            return -1;
    ModelBuilder mb;
    mb.b.n = n;
    mb.b.cta = false;
    std::vector<std::pair<long, int>> w;
    for (int i = 0; i < md.m; i++)
        for (int j = md.I[i] + 1; j <= md.I[i + 1]; j++)
            w.push_back(std::make_pair(md.J[i] + md.beta[i] * (long)(j - md.I[i]), j));
    std::sort(w.begin(), w.end());
    for (const auto &e : w) {
        mb.x.push_back(e.first);
        mb.pos.push_back(e.second);
    }
    out->runs.clear();
    uint64_t patterns = 0;
    const int rc = mb.build(cap, &out->runs, &patterns);
    if (rc)
        return rc;
    if (patterns >= 0xFFFFFFFFull)
        return -3;
    out->patterns = patterns;
    out->wmax_logistic = 0;
    /* no triple runs: the CTA table is the warp table, X3 is empty */
    out->runs_cta = out->runs;
    out->trip.clear();
    out->s3max = 0;
    out->x3off.assign(2, 0u);
    finish_tables(out);
    return 0;
}

/* Expands run r's j-th pattern into v (1-based sorted positions, ascending);
 * returns its Hamming weight.  trip is the table's X3 triple list. */
int orbg_run_pattern(const OrbgRun &r, int j, const uint32_t *trip, int *v)
{
    int w = 0;
    for (int i = 0; i < r.npre; i++)
        v[w++] = r.pre[i];
    if (r.kind == ORBG_RUN_PAIRS) {
        const int S = (int)(r.aux & 0xFFu), a = (int)(r.aux >> 8) + j;
        v[w++] = a;
        v[w++] = S - a;
    } else if (r.kind == ORBG_RUN_STRIDE) {
        v[w++] = (int)(r.aux & 0xFFu) + j * (int)((r.aux >> 16) & 0xFFu);
        v[w++] = (int)((r.aux >> 8) & 0xFFu) - j * (int)(r.aux >> 24);
    } else if (r.kind == ORBG_RUN_TRIPLES) {
        const uint32_t t = trip[r.aux + (uint32_t)j];
        v[w++] = (int)(t & 0xFFu) + 1;
        v[w++] = (int)((t >> 8) & 0xFFu) + 1;
        v[w++] = (int)((t >> 16) & 0xFFu) + 1;
    }
    return w;
}

/* ------------------------------------------------------------- GF(2) -- */

namespace {

struct BitMat {
    int rows, cols, words;
    std::vector<uint64_t> a;
    BitMat(const uint8_t *M, int r, int c) : rows(r), cols(c), words((c + 63) / 64),
                                             a((size_t)r * ((c + 63) / 64), 0) {
        for (int i = 0; i < r; i++)
            for (int j = 0; j < c; j++)
                if (M[(size_t)i * c + j])
                    a[(size_t)i * words + j / 64] |= 1ull << (j % 64);
    }
    bool get(int i, int j) const { return (a[(size_t)i * words + j / 64] >> (j % 64)) & 1; }
    void swap_rows(int i, int k) {
        for (int w = 0; w < words; w++)
            std::swap(a[(size_t)i * words + w], a[(size_t)k * words + w]);
    }
    void add_row(int dst, int src) {
        for (int w = 0; w < words; w++)
            a[(size_t)dst * words + w] ^= a[(size_t)src * words + w];
    }
    /* reduced row echelon form; returns pivot columns */
    std::vector<int> rref() {
        std::vector<int> piv;
        int r = 0;
        for (int c = 0; c < cols && r < rows; c++) {
            int p = -1;
            for (int i = r; i < rows; i++)
                if (get(i, c)) { p = i; break; }
            if (p < 0)
                continue;
            swap_rows(r, p);
            for (int i = 0; i < rows; i++)
                if (i != r && get(i, c))
                    add_row(i, r);
            piv.push_back(c);
            r++;
        }
        return piv;
    }
};

}  // namespace

int orbg_gf2_rank(const uint8_t *M, int rows, int cols)
{
    BitMat m(M, rows, cols);
    return (int)m.rref().size();
}

int orbg_gf2_nullspace(const uint8_t *M, int rows, int cols,
                       std::vector<uint8_t> *basis, int *dim)
{
    BitMat m(M, rows, cols);
    std::vector<int> piv = m.rref();
    std::vector<char> is_piv(cols, 0);
    for (int c : piv)
        is_piv[c] = 1;
    basis->clear();
    int d = 0;
    for (int f = 0; f < cols; f++) {
        if (is_piv[f])
            continue;
        std::vector<uint8_t> x(cols, 0);
        x[f] = 1;
        for (size_t i = 0; i < piv.size(); i++)
            x[piv[i]] = m.get((int)i, f) ? 1 : 0;
        basis->insert(basis->end(), x.begin(), x.end());
        d++;
    }
    *dim = d;
    return 0;
}
