"""Pins of the CPU oracle against things other than itself.

Each function takes an ``oracle.Oracle`` and raises AssertionError on a
mismatch.  tests/test_oracle_pins.py runs them on the real oracle;
tests/test_oracle_mutations.py runs them on copies with planted mistakes,
each of which must fail at least one pin.

Sources of truth, none of them the oracle's own code:
  * the paper's worked examples (tests/golden/, each line cited);
  * closed forms: the generating function prod_i (1 + q^i) for the number
    of patterns per logistic weight (Eq. znwl), the Gaussian binomial for
    partitions into at most w parts <= n' (Eq. intpart2), textbook values
    of the distinct-part partition numbers;
  * brute force over all 2^n patterns (tests/brute_force.py);
  * decoder invariants (noiseless input, H c = 0, basis, scaling,
    permutation equivariance).
"""
import functools
import itertools
import os

import numpy as np

import brute_force
from paper_2202_13951_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            rows[k.strip()] = v.strip()
    return rows


# ------------------------------------------------------------ closed forms

def distinct_part_counts(n, Wmax):
    """Coefficients of prod_{i=1}^{n} (1 + q^i) up to q^Wmax."""
    poly = [1] + [0] * Wmax
    for i in range(1, n + 1):
        for W in range(Wmax, i - 1, -1):
            poly[W] += poly[W - i]
    return poly


@functools.lru_cache(maxsize=None)
def gaussian_binomial(m, k):
    """Coefficients of the q-binomial [m choose k]_q (a polynomial in q)."""
    if k < 0 or k > m:
        return [0]
    table = {}

    def rec(mm, kk):
        if kk == 0 or kk == mm:
            return [1]
        key = (mm, kk)
        if key in table:
            return table[key]
        a = rec(mm - 1, kk - 1)
        b = rec(mm - 1, kk)
        out = [0] * max(len(a), len(b) + kk)
        for i, x in enumerate(a):
            out[i] += x
        for i, x in enumerate(b):
            out[i + kk] += x
        table[key] = out
        return out

    return tuple(rec(m, k))


# ------------------------------------------------------------------ pins

def pin_first_queries(orc):
    """Sec. III-B: queries 1..3 are {}, {1}, {2}; queries 4-5 are {3} and
    {1,2} (tie arbitrary in the paper; this library's reading puts the lower
    Hamming weight first)."""
    g = _golden("sec3b_first_queries.txt")
    for n in (3, 8, 64, 256):
        got = orc.enumerate_patterns(n, 5)
        assert got[0] == () and g["1"] == "-"
        assert got[1] == tuple(int(x) for x in g["2"].split())
        assert got[2] == tuple(int(x) for x in g["3"].split())
        pair = [tuple(int(x) for x in p.split()) for p in g["4-5"].split("|")]
        assert set(got[3:5]) == set(pair)
        assert got[3] == (3,) and got[4] == (1, 2)   # w ascending reading


def pin_fig3(orc):
    """Fig. 3: Landslide(W'=8, w=4, n'=4) gives steps (a)..(h)."""
    g = _golden("fig3_landslide.txt")
    rows = orc.landslide(8, 4, 4)
    assert len(rows) == int(g["count"])
    assert rows[0] == tuple(int(x) for x in g["a"].split())
    assert rows[4] == tuple(int(x) for x in g["e"].split())
    assert rows[-1] == tuple(int(x) for x in g["h"].split())
    # every partition of 8 into 4 non-decreasing parts <= 4, each once
    brute = sorted(u for u in _nondecreasing(4, 8, 4))
    assert sorted(rows) == brute


def _nondecreasing(w, total, cap, lo=0):
    if w == 0:
        if total == 0:
            yield ()
        return
    for x in range(lo, cap + 1):
        if x * w > total:
            break
        for rest in _nondecreasing(w - 1, total - x, cap, x):
            yield (x,) + rest


def pin_fig5(orc):
    """Fig. 5: (W=18, w=4, n=8) is (W'=8, w=4, n'=4) shifted by 1,2,3,4, and
    it is exactly the 4-subsets of {1..8} summing to 18."""
    g = _golden("fig5_mapping.txt")
    W, w, n = int(g["W"]), int(g["w"]), int(g["n"])
    off = [int(x) for x in g["offsets"].split()]
    us = orc.landslide(W - w * (w + 1) // 2, w, n - w)
    vs = [tuple(u[i] + off[i] for i in range(w)) for u in us]
    brute = [c for c in itertools.combinations(range(1, n + 1), w)
             if sum(c) == W]
    assert sorted(vs) == sorted(brute)
    # and the decoder's order visits exactly these, in this order
    allp = orc.enumerate_patterns(n, 1 << n)
    cls = [p for p in allp if len(p) == w and sum(p) == W]
    assert cls == vs


def pin_counts_closed_form(orc):
    """Patterns per logistic weight = coefficients of prod (1+q^i) (Eq.
    znwl); per (W, w) = Gaussian binomial [n'+w choose w]_q at q^W'
    (Eq. intpart2); textbook distinct-part partition numbers."""
    textbook = [1, 1, 1, 2, 2, 3, 4, 5, 6, 8, 10, 12]  # A000009, W = 0..11
    cnt = orc.count_by_weight(40, 11)
    assert list(cnt.sum(axis=1)) == textbook
    for n, Wmax in ((7, 28), (16, 60), (64, 70), (128, 50), (256, 40)):
        cnt = orc.count_by_weight(n, Wmax)
        assert list(cnt.sum(axis=1)) == distinct_part_counts(n, Wmax)[:Wmax + 1]
        for W in range(Wmax + 1):
            for w in range(1, n + 1):
                Wp = W - w * (w + 1) // 2
                if Wp < 0:
                    assert cnt[W, w] == 0
                    continue
                gb = gaussian_binomial(n, w)  # [(n-w)+w choose w]_q
                expect = gb[Wp] if Wp < len(gb) else 0
                assert cnt[W, w] == expect, (n, W, w, cnt[W, w], expect)


def pin_cumulative_counts(orc):
    """Patterns with W <= 82 (the depth a 1e6 query cap reaches)."""
    for n in (64, 128):
        cnt = orc.count_by_weight(n, 82)
        assert int(cnt.sum()) == sum(distinct_part_counts(n, 82))


def pin_order_brute(orc):
    """The whole order for n <= 10 equals sorting all subsets by
    (W, w, lexicographic)."""
    for n in (1, 2, 5, 7, 10):
        got = orc.enumerate_patterns(n, 1 << n)
        assert got == list(brute_force.query_order(n))


def _tiny_inputs(code, rng, blocks):
    """Random LLRs with ties, signed zeros and infinities mixed in."""
    out = []
    for b in range(blocks):
        llr = rng.normal(0.0, 2.0, code.n).astype(np.float32)
        kind = b % 5
        if kind == 1:   # quantised: many ties
            llr = np.round(llr).astype(np.float32)
        elif kind == 2:  # signed zeros and infinities
            llr[rng.integers(0, code.n, 2)] = 0.0
            llr[rng.integers(0, code.n, 1)] = -0.0
            llr[rng.integers(0, code.n, 1)] = np.inf
        elif kind == 3:  # all equal magnitude: hard GRAND order
            llr = np.where(rng.random(code.n) < 0.5, -1.0, 1.0).astype(np.float32)
        out.append(llr)
    return out


def pin_brute_decode(orc, blocks=60):
    """Oracle = brute force on the (7,4) Hamming code and a seeded random
    (16,11) code, at every cap for n=7 and at boundary caps for n=16."""
    rng = np.random.default_rng(7)
    ham = workloads.hamming74()
    for llr in _tiny_inputs(ham, rng, blocks):
        for cap in range(1, 129):
            c0, q0, a0 = brute_force.decode(ham.H, llr, cap)
            c1, q1, a1, _, _ = orc.decode(ham.H, llr, cap)
            assert (c0 == c1).all() and q0 == q1 and a0 == a1, (llr, cap)
    code = workloads.rlc(16, 11, seed=16)
    for llr in _tiny_inputs(code, rng, blocks):
        _, qh, _ = brute_force.decode(code.H, llr, 1 << 16)
        for cap in sorted({1, 2, 3, max(1, qh - 1), qh, qh + 1, 1 << 16}):
            c0, q0, a0 = brute_force.decode(code.H, llr, cap)
            c1, q1, a1, _, _ = orc.decode(code.H, llr, cap)
            assert (c0 == c1).all() and q0 == q1 and a0 == a1, (llr, cap)


def pin_invariants(orc):
    """Noiseless input decodes at query 1; H c = 0 whenever not abandoned;
    decoding does not depend on the basis of H, on a positive scaling of the
    LLRs, and commutes with a joint permutation of coordinates."""
    rng = np.random.default_rng(11)
    code = workloads.rlc(48, 38, seed=3)
    llr, cw = workloads.awgn_llr(code, 40, 4.0, seed=5)
    # noiseless: LLR signs agree with the codeword
    clean = np.where(cw == 1, 3.0, -3.0).astype(np.float32)
    clean *= rng.uniform(0.5, 2.0, clean.shape).astype(np.float32)
    for b in range(10):
        c, q, a, _, _ = orc.decode(code.H, clean[b], 1000)
        assert q == 1 and a == 0 and (c == cw[b]).all()
    # other basis: H' = A H with A invertible over GF(2)
    while True:
        A = rng.integers(0, 2, (code.r, code.r)).astype(np.uint8)
        if workloads.gf2_rank(A) == code.r:
            break
    H2 = ((A.astype(np.int64) @ code.H.astype(np.int64)) % 2).astype(np.uint8)
    perm = rng.permutation(code.n)
    for b in range(llr.shape[0]):
        c, q, a, _, _ = orc.decode(code.H, llr[b], 20000)
        if not a:
            assert not ((code.H.astype(np.int64) @ c) % 2).any()
        c2, q2, a2, _, _ = orc.decode(H2, llr[b], 20000)
        assert (c == c2).all() and q == q2 and a == a2
        c3, q3, a3, _, _ = orc.decode(code.H, llr[b] * np.float32(4.0), 20000)
        assert (c == c3).all() and q == q3 and a == a3
        mags = np.abs(llr[b])
        if np.unique(mags).shape[0] == code.n:
            c4, q4, a4, _, _ = orc.decode(code.H[:, perm], llr[b][perm], 20000)
            assert (c4 == c[perm]).all() and q4 == q and a4 == a


def pin_cap_boundary(orc):
    """A hit exactly at query cap is a decoding; one query less abandons and
    returns the hard decision with q = cap."""
    code = workloads.rlc(32, 24, seed=9)
    llr, _ = workloads.awgn_llr(code, 30, 3.0, seed=10)
    seen = 0
    for b in range(llr.shape[0]):
        c, q, a, _, _ = orc.decode(code.H, llr[b], 100000)
        if a or q < 3:
            continue
        seen += 1
        c1, q1, a1, _, _ = orc.decode(code.H, llr[b], q)
        assert a1 == 0 and q1 == q and (c1 == c).all()
        c2, q2, a2, _, _ = orc.decode(code.H, llr[b], q - 1)
        assert a2 == 1 and q2 == q - 1
        assert (c2 == (llr[b] > 0)).all()
    assert seen > 5


# ---------------------------------------------- one-line full ORBGRAND

# (J0, beta) pairs: basic, intercepts below, at and far above one slope,
# slopes above one, and intercepts not divisible by the slope
LINES = [(0, 1), (1, 1), (3, 1), (20, 1), (0, 2), (5, 2), (2, 3), (7, 4)]


def pin_1line_order_brute(orc):
    """The whole one-line order for n <= 10 equals sorting all subsets by
    (J0 w + beta w_L, w, lexicographic) (Sec. III-D, Eq. relest_seg, m = 1)."""
    for n in (1, 3, 6, 9, 10):
        for J0, beta in LINES:
            got = orc.enumerate_patterns_1line(n, 1 << n, J0, beta)
            assert got == list(brute_force.query_order_1line(n, J0, beta)), (n, J0, beta)


def _rw_series(n, J0, beta, Rmax):
    """Coefficients of prod_{i=1}^{n} (1 + x^(J0 + beta i)) up to x^Rmax: the
    number of patterns of each reliability weight."""
    c = [0] * (Rmax + 1)
    c[0] = 1
    for i in range(1, n + 1):
        e = J0 + beta * i
        for R in range(Rmax, e - 1, -1):
            c[R] += c[R - e]
    return c


def pin_1line_generating_function(orc):
    """For n = 40 and 64, the oracle's first patterns carry non-decreasing
    reliability weights whose counts per weight are the coefficients of
    prod_i (1 + x^(J0 + beta i))."""
    for n, J0, beta, Rmax in ((40, 4, 2, 90), (64, 0, 1, 40), (64, 3, 1, 60),
                              (40, 2, 3, 80)):
        want = _rw_series(n, J0, beta, Rmax)
        total = sum(want)
        pats = orc.enumerate_patterns_1line(n, total, J0, beta)
        assert len(pats) == total
        rw = [J0 * len(v) + beta * sum(v) for v in pats]
        assert rw == sorted(rw) and rw[-1] <= Rmax
        hist = [0] * (Rmax + 1)
        for R in rw:
            hist[R] += 1
        assert hist == want, (n, J0, beta)


def pin_1line_is_basic_at_origin(orc):
    """J0 = 0, beta = 1 is basic ORBGRAND (the paper's special case of
    Eq. relest_seg): same order, same decodings."""
    assert orc.enumerate_patterns_1line(64, 20000, 0, 1) == orc.enumerate_patterns(64, 20000)
    code = workloads.rlc(48, 38, seed=3)
    llr, _ = workloads.awgn_llr(code, 60, 3.0, seed=6)
    a = orc.decode_batch(code.H, llr, 20000)
    b = orc.decode_batch_1line(code.H, llr, 20000, 0, 1)
    for x, y in zip(a, b):
        assert (x == y).all()


def pin_1line_brute_decode(orc, blocks=40):
    """One-line oracle = brute force on the (7,4) Hamming code at every cap
    and on a seeded random (12,8) code at boundary caps, for every line."""
    rng = np.random.default_rng(17)
    ham = workloads.hamming74()
    code = workloads.rlc(12, 8, seed=12)
    for J0, beta in LINES:
        for llr in _tiny_inputs(ham, rng, blocks // 4):
            for cap in range(1, 129, 7):
                c0, q0, a0 = brute_force.decode_1line(ham.H, llr, cap, J0, beta)
                c1, q1, a1, _, _ = orc.decode_1line(ham.H, llr, cap, J0, beta)
                assert (c0 == c1).all() and q0 == q1 and a0 == a1, (J0, beta, llr, cap)
        for llr in _tiny_inputs(code, rng, blocks // 4):
            _, qh, _ = brute_force.decode_1line(code.H, llr, 1 << 12, J0, beta)
            for cap in sorted({1, 2, max(1, qh - 1), qh, qh + 1, 1 << 12}):
                c0, q0, a0 = brute_force.decode_1line(code.H, llr, cap, J0, beta)
                c1, q1, a1, _, _ = orc.decode_1line(code.H, llr, cap, J0, beta)
                assert (c0 == c1).all() and q0 == q1 and a0 == a1, (J0, beta, llr, cap)


def pin_1line_invariants(orc):
    """Noiseless input decodes at query 1 for any line; H c = 0 whenever not
    abandoned."""
    rng = np.random.default_rng(19)
    code = workloads.rlc(40, 30, seed=4)
    llr, cw = workloads.awgn_llr(code, 20, 3.5, seed=8)
    clean = np.where(cw == 1, 2.0, -2.0).astype(np.float32)
    clean *= rng.uniform(0.5, 2.0, clean.shape).astype(np.float32)
    for J0, beta in ((3, 1), (5, 2)):
        for b in range(5):
            c, q, a, _, _ = orc.decode_1line(code.H, clean[b], 1000, J0, beta)
            assert q == 1 and a == 0 and (c == cw[b]).all()
        for b in range(llr.shape[0]):
            c, q, a, _, _ = orc.decode_1line(code.H, llr[b], 20000, J0, beta)
            if not a:
                assert not ((code.H.astype(np.int64) @ c) % 2).any()


# ------------------------------------------- m-segment full ORBGRAND

# (anchors, J, beta) for n = 10 (anchors inside 1..9); includes one
# segment, zero intercepts, J divisible and not divisible by beta
MODELS10 = [((), (0,), (1,)), ((), (4,), (3,)), ((3,), (0, 4), (1, 2)),
            ((2, 6), (0, 3, 6), (1, 1, 2)), ((4, 7), (1, 6, 9), (2, 3, 1)),
            ((1, 2, 5), (0, 2, 5, 9), (1, 2, 1, 3)),
            # a first segment starting at weight 0 (J_0 = -beta_1, as Eq. quant
            # gives when the least reliable bit rounds to 0)
            ((3,), (-2, 3), (2, 1)), ((), (-1,), (1,))]


def pin_mline_order_brute(orc):
    """The whole m-segment order for n = 10 equals sorting all subsets by
    (sum of the model's reliabilities, w, lexicographic) (Sec. III-D)."""
    for model in MODELS10:
        got = orc.enumerate_patterns_mline(10, 1 << 10, model)
        assert got == list(brute_force.query_order_model(10, model)), model


def pin_mline_generating_function(orc):
    """For n = 30, the first patterns' reliability weights are
    non-decreasing and their counts per weight are the coefficients of
    prod_j (1 + x^rho_j)."""
    n, Rmax = 30, 45
    for model in (((10, 20), (0, 4, 9), (1, 1, 2)), ((12,), (2, 7), (1, 3))):
        rho = brute_force.model_weights(n, model)
        c = [0] * (Rmax + 1)
        c[0] = 1
        for e in rho:
            for R in range(Rmax, e - 1, -1):
                c[R] += c[R - e]
        total = sum(c)
        pats = orc.enumerate_patterns_mline(n, total, model)
        rw = [sum(rho[p - 1] for p in v) for v in pats]
        assert len(pats) == total and rw == sorted(rw) and rw[-1] <= Rmax
        hist = [0] * (Rmax + 1)
        for R in rw:
            hist[R] += 1
        assert hist == c, model


def pin_mline_one_segment_is_one_line(orc):
    """One segment is the one-line order (Eq. relest_seg with m = 1)."""
    for J0, beta in ((0, 1), (3, 1), (5, 2)):
        assert (orc.enumerate_patterns_mline(40, 5000, ((), (J0,), (beta,))) ==
                orc.enumerate_patterns_1line(40, 5000, J0, beta))
    code = workloads.rlc(24, 16, seed=5)
    llr, _ = workloads.awgn_llr(code, 30, 2.5, seed=9)
    a = orc.decode_batch_1line(code.H, llr, 3000, 3, 1)
    b = orc.decode_batch_mline(code.H, llr, 3000, ((), (3,), (1,)))
    for x, y in zip(a, b):
        assert (x == y).all()


def pin_mline_brute_decode(orc, blocks=30):
    """m-segment oracle = brute force on a seeded random (10,6) code."""
    rng = np.random.default_rng(23)
    code = workloads.rlc(10, 6, seed=10)
    for model in MODELS10[2:]:
        llrs = np.stack(_tiny_inputs(code, rng, blocks))
        for cap in (1, 3, 17, 1 << 10):
            c1, q1, a1, _ = orc.decode_batch_mline(code.H, llrs, cap, model)
            for b in range(blocks):
                c0, q0, a0 = brute_force.decode_model(code.H, llrs[b], cap, model)
                assert (c0 == c1[b]).all() and q0 == q1[b] and a0 == a1[b], (model, cap)


# ------------------------------------------- piece-wise fitting (Sec. III-E)

# Closed forms for the ordered reliabilities L_j = j^2 (Eq. Q, Eq. quant),
# worked by hand.  The vertical gap between the chord over [lo, hi] and the
# parabola is (j - lo)(hi - j), largest at the midpoint; an odd lo + hi ties
# two indices and the smaller is taken.  Keys (n, lines); values are the
# models (anchors, J, beta) without and with J_{i-1} divisible by beta_i.
#   n = 64, centre 32: anchors 16 (tie 16/17), then 8 (tie 8/9), 4 (tie
#   4/5), 2 (tie 2/3), then [1, 2] has no inner index.  Four lines: slopes
#   15/3, 48/4, 192/8, 768/16 = 5, 12, 24, 48, Q = 5, beta = [1, 2.4, 4.8,
#   9.6] = (1, 2, 5, 10), J_0 = [1/5] - 1, J = [16/5], [64/5], [256/5];
#   divisible: [3/2]*2 = 4, [13/5]*5 = 15, [51/10]*10 = 50.
#   n = 12, centre 6: anchors 3 (tie 3/4), 2.  Three lines: slopes 3, 5, 9,
#   Q = 3, beta = (1, [5/3], 3), J = ([1/3] - 1, [4/3], [9/3]); divisible
#   J_1 = [1/2]*2 = 2 (half away from zero).
#   n = 13: the centre is floor(13/2) = 6, so the fit equals n = 12's.
PARABOLA_FITS = {
    (64, 1): (((), (-1,), (1,)), ((), (-1,), (1,))),
    (64, 2): (((16,), (-1, 15), (1, 3)), ((16,), (-1, 15), (1, 3))),
    (64, 3): (((8, 16), (-1, 7, 28), (1, 3, 5)), ((8, 16), (-1, 6, 30), (1, 3, 5))),
    (64, 4): (((4, 8, 16), (-1, 3, 13, 51), (1, 2, 5, 10)),
              ((4, 8, 16), (-1, 4, 15, 50), (1, 2, 5, 10))),
    (64, 5): (((2, 4, 8, 16), (-1, 1, 5, 21, 85), (1, 2, 4, 8, 16)),
              ((2, 4, 8, 16), (-1, 2, 4, 24, 80), (1, 2, 4, 8, 16))),
    (64, 6): (((2, 4, 8, 16), (-1, 1, 5, 21, 85), (1, 2, 4, 8, 16)),
              ((2, 4, 8, 16), (-1, 2, 4, 24, 80), (1, 2, 4, 8, 16))),
    (12, 1): (((), (-1,), (1,)), ((), (-1,), (1,))),
    (12, 2): (((3,), (-1, 2), (1, 2)), ((3,), (-1, 2), (1, 2))),
    (12, 3): (((2, 3), (-1, 1, 3), (1, 2, 3)), ((2, 3), (-1, 2, 3), (1, 2, 3))),
    (12, 4): (((2, 3), (-1, 1, 3), (1, 2, 3)), ((2, 3), (-1, 2, 3), (1, 2, 3))),
    (13, 2): (((3,), (-1, 2), (1, 2)), ((3,), (-1, 2), (1, 2))),
}


def _disguise(L, rng, scale=1.0):
    """Received LLRs whose sorted magnitudes are L * scale: a random order
    and random signs (the fit sees only the ordered reliabilities)."""
    x = np.asarray(L, np.float64) * scale
    x = x[rng.permutation(len(x))] * rng.choice((-1.0, 1.0), len(x))
    return x.astype(np.float32)


def pin_fit_parabola(orc):
    """Anchor search, Eq. Q and Eq. quant on L_j = j^2 against the hand-worked
    closed forms, in any received order and sign, at power-of-two scales."""
    rng = np.random.default_rng(29)
    for (n, lines), (plain, div) in PARABOLA_FITS.items():
        L = [j * j for j in range(1, n + 1)]
        for scale in (1.0, 0.125, 32.0):
            llr = _disguise(L, rng, scale)
            assert orc.fit(llr, lines) == plain, (n, lines, scale)
            assert orc.fit(llr, lines, divisible=True) == div, (n, lines, scale)


def pin_fit_piecewise_exact(orc):
    """A convex piece-wise linear curve with its kinks below the centre and
    a straight tail is fitted exactly: the anchors are the kinks and
    Q * rho_j = L_j at every j (Eq. relest_seg, Eq. quant with no rounding)."""
    rng = np.random.default_rng(31)
    # (n, lines, kinks, slopes, L_1, expected model), slopes a multiple of 2
    cases = [(40, 2, (6,), (2, 6), 6, ((6,), (2, 8), (1, 3))),
             (40, 3, (6,), (2, 6), 6, ((6,), (2, 8), (1, 3))),
             (40, 3, (3, 10), (2, 4, 8), 2, ((3, 10), (0, 3, 17), (1, 2, 4))),
             (64, 4, (3, 10), (2, 4, 8), 2, ((3, 10), (0, 3, 17), (1, 2, 4)))]
    for n, lines, kinks, slopes, L1, want in cases:
        L, seg = [L1], 0
        for j in range(2, n + 1):
            if seg < len(kinks) and j > kinks[seg]:
                seg += 1
            L.append(L[-1] + slopes[seg])
        model = orc.fit(_disguise(L, rng), lines)
        assert model == want, (n, lines, model)
        Q = min(slopes)
        assert [Q * r for r in brute_force.model_weights(n, model)] == L
    # the three-line case with J_{i-1} divisible by beta_i: [3/2]*2, [17/4]*4
    L = [2 * j if j <= 3 else 6 + 4 * (j - 3) if j <= 10 else 34 + 8 * (j - 10)
         for j in range(1, 41)]
    assert orc.fit(_disguise(L, rng), 3, divisible=True) == ((3, 10), (0, 4, 16), (1, 2, 4))


def pin_fit_invariants(orc):
    """On AWGN blocks: at most `lines` segments, anchors strictly inside
    (1, floor(n/2)) and nested as lines grow, beta >= 1 with the smallest
    slope quantised to 1 (Eq. Q), every position weight >= 0, J_{i-1} a
    multiple of beta_i in the divisible variant within beta_i / 2 of the
    plain J, the same model for any order, sign or power-of-two scale of
    the LLRs, and a model the m-segment order accepts."""
    rng = np.random.default_rng(37)
    code = workloads.rlc(64, 48, seed=6)
    for snr in (1.0, 4.0, 7.0):
        llr, _ = workloads.awgn_llr(code, 12, snr, seed=int(snr) + 40)
        for b in range(llr.shape[0]):
            x = llr[b]
            prev = ()
            for lines in range(1, 7):
                anchors, J, beta = model = orc.fit(x, lines)
                m = len(J)
                assert 1 <= m <= lines and len(beta) == m and len(anchors) == m - 1
                assert all(1 < a < 32 for a in anchors)
                assert list(anchors) == sorted(set(anchors))
                assert set(prev) <= set(anchors)
                prev = anchors
                assert min(beta) == 1 and all(bb >= 1 for bb in beta)
                assert min(brute_force.model_weights(64, model)) >= 0
                _, Jd, bd = orc.fit(x, lines, divisible=True)
                assert bd == beta
                assert all(Jd[i] % beta[i] == 0 and 2 * abs(Jd[i] - J[i]) <= beta[i]
                           for i in range(m))
                y = (x * np.float32(4.0))[rng.permutation(64)]
                y *= rng.choice((-1.0, 1.0), 64).astype(np.float32)
                assert orc.fit(y, lines) == model
                assert len(orc.enumerate_patterns_mline(64, 50, model)) == 50


def pin_fit_degenerate(orc):
    """Curves Eq. Q and Eq. quant cannot quantise give the basic model
    (J_0 = 0, beta_1 = 1): fewer than four positions, a flat curve (Q = 0),
    infinite reliabilities at the anchors, and a ratio beyond 2^24."""
    basic = ((), (0,), (1,))
    for n in (1, 2, 3):
        assert orc.fit(np.arange(1, n + 1, dtype=np.float32), 3) == basic
    assert orc.fit(np.full(40, 1.5, np.float32), 3) == basic
    assert orc.fit(np.full(40, np.inf, np.float32), 2) == basic
    # slope 1e-20 up to the kink at 5, then 1e20: the second slope is 1e40 Q
    steep = np.array([1e-20 * j if j <= 5 else 5e-20 + 1e20 * (j - 5) for j in range(1, 41)],
                     np.float32)
    for lines in (2, 3):
        assert orc.fit(steep, lines) == basic
        assert orc.fit(steep, lines, divisible=True) == basic


def pin_fit_brute_decode(orc, blocks=24):
    """Full ORBGRAND with per-block fitting (Sec. III-E, then the m-segment
    order) = brute force under the closed-form model, on blocks whose
    ordered reliabilities are j^2 (n = 12, seeded random (12, 6) code)."""
    rng = np.random.default_rng(41)
    code = workloads.rlc(12, 6, seed=11)
    L = [j * j for j in range(1, 13)]
    llrs = np.stack([_disguise(L, rng, 0.25) for _ in range(blocks)])
    for lines in (1, 2, 3):
        for divisible in (False, True):
            model = PARABOLA_FITS[(12, lines)][int(divisible)]
            for cap in (1, 5, 40, 1 << 12):
                c1, q1, a1, _ = orc.decode_batch_fit(code.H, llrs, cap, lines, divisible)
                for b in range(blocks):
                    c0, q0, a0 = brute_force.decode_model(code.H, llrs[b], cap, model)
                    assert (c0 == c1[b]).all() and q0 == q1[b] and a0 == a1[b], (lines, cap)
    # AWGN blocks: each block is decoded under its own fitted model
    code = workloads.rlc(24, 16, seed=5)
    llr, _ = workloads.awgn_llr(code, 16, 4.0, seed=12)
    c1, q1, a1, _ = orc.decode_batch_fit(code.H, llr, 3000, 3)
    for b in range(llr.shape[0]):
        c0, q0, a0, _ = orc.decode_batch_mline(code.H, llr[b:b + 1], 3000, orc.fit(llr[b], 3))
        assert (c0[0] == c1[b]).all() and q0[0] == q1[b] and a0[0] == a1[b]


FAST_PINS = [pin_first_queries, pin_fig3, pin_fig5, pin_order_brute,
             pin_counts_closed_form, pin_brute_decode, pin_invariants,
             pin_cap_boundary, pin_1line_order_brute, pin_1line_generating_function,
             pin_1line_is_basic_at_origin, pin_1line_brute_decode, pin_1line_invariants,
             pin_mline_order_brute, pin_mline_generating_function,
             pin_mline_one_segment_is_one_line, pin_mline_brute_decode, pin_fit_parabola,
             pin_fit_piecewise_exact, pin_fit_invariants, pin_fit_degenerate,
             pin_fit_brute_decode]


def run_all(orc, pins=None):
    for p in pins or FAST_PINS:
        p(orc)
