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
