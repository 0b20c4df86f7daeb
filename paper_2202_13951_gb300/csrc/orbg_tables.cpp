/*
 * orbg_tables.cpp -- host-side tables of the query order, and GF(2) helpers.
 *
 * The order is basic ORBGRAND's (Sec. III-B): logistic weight
 * W = sum_i v_i over the flipped sorted positions v (Eq. lw) ascending,
 * split by Hamming weight w (Eq. fractionation) ascending, and inside one
 * (W, w) the distinct-part partitions v_1 < ... < v_w <= n of W (Eq.
 * intpart) in lexicographic order, the order Algorithm 2 (Landslide)
 * generates.  This file enumerates that order directly as lexicographic
 * prefixes plus a final pair (see orbg_internal.h), not with Landslide.
 */
#include <algorithm>
#include <cstring>
#include <vector>

#include "orbg_internal.h"

namespace {

struct Builder {
    int n;
    uint64_t t;                    /* next query index */
    std::vector<OrbgRun> cls;      /* runs of the current (W, w) class */
    int pre[64];

    void emit_single(const int *p, int np) {
        OrbgRun r;
        std::memset(&r, 0, sizeof(r));
        r.tstart = (uint32_t)t;
        r.pair_sum = (uint16_t)(2 * n);   /* a0 = b0 = n: the zero column */
        r.a0 = (uint16_t)n;
        r.len = 1;
        r.npre = (uint8_t)np;
        for (int i = 0; i < np; i++)
            r.pre[i] = (uint8_t)(p[i] - 1);
        cls.push_back(r);
        t += 1;
    }

    /* Prefixes of `need` more positions, each > lo-1, with `rem` left for
     * them and the final pair; `depth` positions already in pre[]. */
    void prefixes(int depth, int need, int lo, int rem) {
        if (need == 0) {
            /* pair a < b, a >= lo, b <= n, a + b = rem */
            int S = rem;
            int a_lo = std::max(lo, S - n);
            int a_hi = (S - 1) / 2;
            if (a_lo > a_hi)
                return;
            OrbgRun r;
            std::memset(&r, 0, sizeof(r));
            r.tstart = (uint32_t)t;
            r.pair_sum = (uint16_t)(S - 2);
            r.a0 = (uint16_t)(a_lo - 1);
            r.len = (uint8_t)(a_hi - a_lo + 1);
            r.npre = (uint8_t)depth;
            for (int i = 0; i < depth; i++)
                r.pre[i] = (uint8_t)(pre[i] - 1);
            cls.push_back(r);
            t += (uint64_t)(a_hi - a_lo + 1);
            return;
        }
        /* after choosing v, need-1 more prefix positions and the pair, all
         * distinct and above v: m = need + 1 positions */
        const int m = need + 1;
        for (int v = lo; v <= n; v++) {
            long min_rest = (long)m * v + (long)m * (m + 1) / 2;
            long max_rest = (long)m * n - (long)m * (m - 1) / 2;
            if (v + min_rest > rem)
                break;
            if (v + max_rest < rem)
                continue;
            pre[depth] = v;
            prefixes(depth + 1, need - 1, v + 1, rem - v);
        }
    }

    void flush(OrbgTables *out) {
        /* longest runs first; equal lengths keep the query order */
        std::stable_sort(cls.begin(), cls.end(),
                         [](const OrbgRun &a, const OrbgRun &b) {
                             return a.len > b.len;
                         });
        out->runs.insert(out->runs.end(), cls.begin(), cls.end());
        cls.clear();
    }
};

}  // namespace

int orbg_build_tables(int n, uint64_t cap, OrbgTables *out)
{
    if (n < 1 || n > 256 || cap < 1)
        return -1;
    out->runs.clear();
    out->group_floor.clear();
    Builder b;
    b.n = n;
    b.t = 1;
    /* W = 0: the zero pattern */
    b.emit_single(nullptr, 0);
    b.flush(out);
    long Wlast = (long)n * (n + 1) / 2;
    int wdeep = 0;
    for (long W = 1; W <= Wlast && b.t <= cap; W++) {
        for (int w = 1; (long)w * (w + 1) / 2 <= W && w <= n; w++) {
            if (w - 2 > ORBG_RUN_MAX_PRE)
                return -2;
            if (w == 1) {
                if (W <= n) {
                    int p = (int)W;
                    b.emit_single(&p, 1);
                }
            } else {
                b.prefixes(0, w - 2, 1, (int)W);
            }
            b.flush(out);
        }
        wdeep = (int)W;
    }
    out->patterns = b.t - 1;
    out->wmax_logistic = wdeep;
    if (out->patterns >= 0xFFFFFFFFull)
        return -3;
    /* pad to whole groups with runs that start after every real one */
    size_t nr = out->runs.size();
    size_t ng = (nr + ORBG_GROUP - 1) / ORBG_GROUP;
    out->group_floor.assign(ng, 0xFFFFFFFFu);
    uint32_t floor = 0xFFFFFFFFu;
    for (size_t g = ng; g-- > 0;) {
        for (size_t i = g * ORBG_GROUP; i < std::min(nr, (g + 1) * ORBG_GROUP); i++)
            floor = std::min(floor, out->runs[i].tstart);
        out->group_floor[g] = floor;
    }
    return 0;
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
