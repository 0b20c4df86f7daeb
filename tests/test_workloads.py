"""Input generators: code constructions and the channel convention."""
import math

import numpy as np

from paper_2202_13951_gb300 import workloads


def _golden(name):
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rows[k.strip()] = v.strip()
    return rows


def test_codes_are_consistent():
    for code in (workloads.hamming74(), workloads.config1_code(),
                 workloads.config2_code(), workloads.config3_code(),
                 *workloads.config4_codes()):
        G = code.G.astype(np.int64)
        H = code.H.astype(np.int64)
        assert G.shape == (code.k, code.n) and H.shape == (code.r, code.n)
        assert not ((G @ H.T) % 2).any()
        assert workloads.gf2_rank(code.G) == code.k
        assert workloads.gf2_rank(code.H) == code.r


def test_bch_generator_degree_and_distance():
    """BCH(127,113), t = 2: g(x) = lcm(m_1, m_3) has degree 14, and the code
    corrects 2 errors, so no codeword of weight <= 4 exists (checked on all
    weight-1..2 column sums of H being non-zero and distinct)."""
    code = workloads.config2_code()
    H = code.H.astype(np.int64)
    cols = [tuple(H[:, j]) for j in range(code.n)]
    assert all(any(c) for c in cols)
    assert len(set(cols)) == code.n  # no weight-2 codeword
    sums = set()
    for i in range(code.n):
        for j in range(i + 1, code.n):
            s = tuple((H[:, i] + H[:, j]) % 2)
            sums.add(s)
    # weight-3/4 absence is equivalent to all pair sums distinct and not a column
    assert len(sums) == code.n * (code.n - 1) // 2
    assert not (sums & set(cols))


def test_crc11_polynomial():
    # x^11 + x^10 + x^9 + x^5 + 1
    assert workloads.CRC11_POLY == 0b111000100001
    msg = [1, 0, 1, 1, 0, 0, 1]
    crc = workloads.crc_bits(msg)
    # appending the CRC gives a multiple of g(x)
    reg = 0
    for b in msg + crc:
        reg = (reg << 1) | b
        if reg >> 11:
            reg ^= workloads.CRC11_POLY
    assert reg == 0


def test_snr_convention():
    """Sec. IV-A: 9.8 dB SNR <=> hard flip probability 1e-3, with
    SNR = 1/sigma^2.  The generator's Eb/N0 is set so that
    2 R Eb/N0 = 10^0.98 and the empirical flip rate is checked."""
    g = _golden("sec4a_snr.txt")
    snr = 10 ** (float(g["snr_db"]) / 10)
    p = 0.5 * math.erfc(math.sqrt(snr) / math.sqrt(2))
    assert abs(p - float(g["p"])) / float(g["p"]) < 0.05
    code = workloads.rlc(100, 80, seed=1)
    R = code.k / code.n
    ebn0_db = 10 * math.log10(snr / (2 * R))
    llr, cw = workloads.awgn_llr(code, 20000, ebn0_db, seed=3)
    flips = ((llr > 0).astype(np.uint8) != cw).mean()
    assert abs(flips - 1e-3) / 1e-3 < 0.1, flips


def test_seeded_and_deterministic():
    code = workloads.config1_code()
    a, _ = workloads.awgn_llr(code, 50, 5.0, seed=101)
    b, _ = workloads.awgn_llr(code, 50, 5.0, seed=101)
    assert a.dtype == np.float32 and (a == b).all()


def test_primitive_polynomials():
    """Primitivity by the order of x: the textbook primitive polynomials the
    BCH codes are built on pass; an irreducible non-primitive one
    (x^4 + x^3 + x^2 + x + 1, order 5) and reducible ones fail; the smallest
    primitive polynomial of degree 22 is the trinomial x^22 + x + 1."""
    assert workloads.is_primitive_poly(0b10001001)      # x^7 + x^3 + 1
    assert workloads.is_primitive_poly(0b100011101)     # x^8 + x^4 + x^3 + x^2 + 1
    assert workloads.is_primitive_poly(0b10011)         # x^4 + x + 1
    assert not workloads.is_primitive_poly(0b11111)     # order 5
    assert not workloads.is_primitive_poly(0b101)       # (x + 1)^2
    assert not workloads.is_primitive_poly(0b10010)     # divisible by x
    # brute force for small degrees: x has order 2^d - 1 modulo p
    for d in range(2, 9):
        for p in range((1 << d) | 1, 1 << (d + 1), 2):
            r, order = 1, None
            for e in range(1, 1 << d):
                r <<= 1
                if r >> d:
                    r ^= p
                if r == 1:
                    order = e
                    break
            assert workloads.is_primitive_poly(p) == (order == (1 << d) - 1), bin(p)
    assert workloads.smallest_primitive_poly(22) == (1 << 22) | 0b11


def test_paper256_codes():
    """The [256, 234]-class codes of Sec. IV: sizes, G H^T = 0, full rank;
    BCH[255, 231] corrects 3 errors (all patterns of weight <= 3 have
    distinct syndromes), CRC[256, 234] corrects 1 (distinct non-zero
    columns: a shortened Hamming code), CA-Polar[256, 234] codewords carry
    frozen zeros and a valid CRC-11 on their 245 positions."""
    codes = workloads.paper256_codes()
    assert [(c.n, c.k) for c in codes] == [(256, 234), (256, 234), (256, 234), (255, 231)]
    for code in codes:
        G = code.G.astype(np.int64)
        H = code.H.astype(np.int64)
        assert not ((G @ H.T) % 2).any()
        assert workloads.gf2_rank(code.G) == code.k
        assert workloads.gf2_rank(code.H) == code.r
    polar, crc, _, bch = codes
    # BCH: syndromes of weight 0..3 patterns all distinct
    Hb = bch.H.astype(np.int64)
    col = (Hb * (1 << np.arange(bch.r))[:, None]).sum(axis=0)
    i, j = np.triu_indices(bch.n, 1)
    pair = col[i] ^ col[j]
    trip = (pair[None, :] ^ col[:, None])[(np.arange(bch.n)[:, None] < i[None, :])]
    syn = np.concatenate([[0], col, pair, trip])
    assert np.unique(syn).size == syn.size == 1 + 255 + 32385 + 2731135
    # CRC: distinct non-zero columns
    Hc = crc.H.astype(np.int64)
    colc = (Hc * (1 << np.arange(crc.r))[:, None]).sum(axis=0)
    assert (colc != 0).all() and np.unique(colc).size == crc.n
    # CA-Polar: F^(x)8 is its own inverse over GF(2); u = x F has zeros off
    # the 245 chosen positions, and its message bits end in their CRC-11
    pos = workloads.bhattacharyya_positions(256, 245, 3.0, 234 / 256)
    rng = np.random.default_rng(7)
    msg = rng.integers(0, 2, (5, 234)).astype(np.uint8)
    x = workloads.encode(polar.G, msg)
    u = workloads.polar_transform(x)
    frozen = np.setdiff1d(np.arange(256), pos)
    assert not u[:, frozen].any()
    for b in range(5):
        info = [int(v) for v in u[b, pos]]
        assert info[234:] == workloads.crc_bits(info[:234])


def test_paper256_inputs():
    """Mixed paper-shaped batch: deterministic, every code present, blocks
    back to back."""
    codes, cid, llr, off, cw, eb = workloads.paper256_inputs(B=4000, seed=5)
    codes2, cid2, llr2, *_ = workloads.paper256_inputs(B=4000, seed=5)
    assert np.array_equal(cid, cid2) and np.array_equal(llr, llr2)
    assert set(np.unique(cid)) == {0, 1, 2, 3}
    ns = np.array([c.n for c in codes])[cid]
    assert off[0] == 0 and (np.diff(off) == ns[:-1]).all()
    assert llr.shape[0] == off[-1] + ns[-1] and (eb >= 4.0).all() and (eb <= 7.0).all()
