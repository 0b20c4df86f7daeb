"""Seeded synthetic inputs: code constructions and the BPSK/AWGN channel.

This module holds none of the decoder's arithmetic (no sorting, no
pattern order, no syndrome search).  It only builds codes and noisy
observations, with NumPy ``default_rng(seed)`` (PCG64), so that the CUDA
path and the CPU oracle decode byte-identical inputs.

Channel (Sec. III-A): a codeword c is modulated to 2c - 1, Gaussian noise
N(0, sigma^2) is added, and the decoder receives LLR = 2 Y / sigma^2, the
log-likelihood ratio log f(Y|1)/f(Y|0) of that channel, rounded to FP32.
Eb/N0 maps to sigma by sigma^2 = 1 / (2 R 10^(EbN0/10)) with R = k/n the
code's true rate.  (Sec. IV-A quotes 9.8 dB for a hard flip probability of
1e-3, i.e. SNR = 1/sigma^2; tests pin that convention.)

Codes (all given as a generator matrix G, k x n, and a parity-check matrix
H, (n-k) x n, with G H^T = 0 over GF(2)):
  * Hamming (7,4)
  * random linear codes G = [I | P], P i.i.d. Bernoulli(1/2) from a seed,
    H = [P^T | I]
  * binary BCH(127,113), t = 2: g(x) = lcm(m_1, m_3) over GF(2^7) built on
    x^7 + x^3 + 1
  * CA-Polar(128, K=105): F^(x)7 in natural order, K positions chosen by the
    Bhattacharyya recursion at a design Eb/N0, 94 message bits followed by an
    11-bit CRC with g(x) = x^11 + x^10 + x^9 + x^5 + 1 (linear dimension 94)
  * the [256, 234] family of Sec. IV (22 parity bits): CA-Polar[256, 234]
    (K = 245 positions: 234 message bits and the same 11-bit CRC),
    CRC[256, 234] (a shortened cyclic code whose degree-22 generator is the
    smallest primitive polynomial of that degree), RLC[256, 234], and
    BCH[255, 231], t = 3, over GF(2^8) built on x^8 + x^4 + x^3 + x^2 + 1
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Code:
    name: str
    n: int
    k: int
    G: np.ndarray  # k x n uint8
    H: np.ndarray  # (n-k) x n uint8

    @property
    def r(self):
        return self.n - self.k


def _check(G, H):
    assert ((G.astype(np.int64) @ H.T.astype(np.int64)) % 2 == 0).all()


def gf2_rank(M):
    """Rank over GF(2) (plain elimination)."""
    A = (np.asarray(M, dtype=np.uint8) & 1).copy()
    rows, cols = A.shape
    rank = 0
    for c in range(cols):
        piv = None
        for i in range(rank, rows):
            if A[i, c]:
                piv = i
                break
        if piv is None:
            continue
        A[[rank, piv]] = A[[piv, rank]]
        for i in range(rows):
            if i != rank and A[i, c]:
                A[i] ^= A[rank]
        rank += 1
        if rank == rows:
            break
    return rank


def gf2_nullspace(M):
    """Basis (rows) of {x : M x = 0} over GF(2)."""
    A = (np.asarray(M, dtype=np.uint8) & 1).copy()
    rows, cols = A.shape
    pivots = []
    r = 0
    for c in range(cols):
        piv = None
        for i in range(r, rows):
            if A[i, c]:
                piv = i
                break
        if piv is None:
            continue
        A[[r, piv]] = A[[piv, r]]
        for i in range(rows):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        pivots.append(c)
        r += 1
        if r == rows:
            break
    free = [c for c in range(cols) if c not in set(pivots)]
    basis = []
    for f in free:
        x = np.zeros(cols, np.uint8)
        x[f] = 1
        for i, pc in enumerate(pivots):
            x[pc] = A[i, f]
        basis.append(x)
    return np.array(basis, dtype=np.uint8).reshape(len(basis), cols)


def hamming74() -> Code:
    H = np.array([[1, 0, 1, 0, 1, 0, 1],
                  [0, 1, 1, 0, 0, 1, 1],
                  [0, 0, 0, 1, 1, 1, 1]], np.uint8)
    G = gf2_nullspace(H)
    _check(G, H)
    return Code("hamming(7,4)", 7, 4, G, H)


def rlc(n: int, k: int, seed: int) -> Code:
    """Random linear code, systematic G = [I_k | P], H = [P^T | I_{n-k}]."""
    rng = np.random.default_rng(seed)
    P = rng.integers(0, 2, size=(k, n - k), dtype=np.uint8)
    G = np.concatenate([np.eye(k, dtype=np.uint8), P], axis=1)
    H = np.concatenate([P.T.copy(), np.eye(n - k, dtype=np.uint8)], axis=1)
    _check(G, H)
    return Code("rlc(%d,%d,seed=%d)" % (n, k, seed), n, k, G, H)


# --------------------------------------------------------------- BCH ----

def _poly_mul2(a, b):
    """Product of GF(2) polynomials given as int bit masks."""
    out = 0
    while b:
        if b & 1:
            out ^= a
        a <<= 1
        b >>= 1
    return out


def _poly_mod2(a, m):
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _minimal_poly(beta_exp, m, prim):
    """Minimal polynomial over GF(2) of alpha^beta_exp in GF(2^m)."""
    nn = (1 << m) - 1
    # exp / log tables of GF(2^m)
    exp = [0] * (2 * nn)
    x = 1
    for i in range(nn):
        exp[i] = x
        x <<= 1
        if x >> m:
            x ^= prim
    for i in range(nn, 2 * nn):
        exp[i] = exp[i - nn]
    log = {exp[i]: i for i in range(nn)}
    coset = []
    e = beta_exp % nn
    while e not in coset:
        coset.append(e)
        e = (2 * e) % nn
    # product of (X + alpha^e) with GF(2^m) coefficients
    poly = [1]  # coefficients, lowest degree first, field elements as ints

    def fmul(a, b):
        if a == 0 or b == 0:
            return 0
        return exp[log[a] + log[b]]

    for e in coset:
        root = exp[e]
        newp = [0] * (len(poly) + 1)
        for i, c in enumerate(poly):
            newp[i + 1] ^= c
            newp[i] ^= fmul(c, root)
        poly = newp
    assert all(c in (0, 1) for c in poly)
    return sum(c << i for i, c in enumerate(poly))


def _poly_powmod2(e, m):
    """x^e mod m(x) over GF(2), square and multiply."""
    result, base = 1, _poly_mod2(0b10, m)
    while e:
        if e & 1:
            result = _poly_mod2(_poly_mul2(result, base), m)
        base = _poly_mod2(_poly_mul2(base, base), m)
        e >>= 1
    return result


def _prime_factors(v):
    out, f = [], 2
    while f * f <= v:
        if v % f == 0:
            out.append(f)
            while v % f == 0:
                v //= f
        f += 1
    if v > 1:
        out.append(v)
    return out


def is_primitive_poly(p):
    """p(x) of degree d over GF(2) is primitive iff x has order 2^d - 1
    modulo p: x^(2^d - 1) = 1 and x^((2^d - 1)/q) != 1 for every prime q
    dividing 2^d - 1 (p irreducible follows)."""
    d = p.bit_length() - 1
    if d < 1 or not p & 1:
        return False
    order = (1 << d) - 1
    if _poly_powmod2(order, p) != 1:
        return False
    return all(_poly_powmod2(order // q, p) != 1 for q in _prime_factors(order))


def smallest_primitive_poly(d):
    """The numerically smallest primitive polynomial of degree d."""
    for p in range((1 << d) | 1, 1 << (d + 1), 2):
        if is_primitive_poly(p):
            return p
    raise ValueError(d)


def cyclic_code(name, n, k, g):
    """The (shortened) cyclic code of generator g(x), deg g = n - k: the
    multiples m(x) g(x) of degree < n."""
    deg = g.bit_length() - 1
    assert deg == n - k, (deg, n - k)
    gb = np.array([(g >> i) & 1 for i in range(deg + 1)], np.uint8)
    G = np.zeros((k, n), np.uint8)
    for i in range(k):
        G[i, i:i + deg + 1] = gb
    H = gf2_nullspace(G)
    assert H.shape == (n - k, n)
    _check(G, H)
    return Code(name, n, k, G, H)


def crc_code(n: int = 256, k: int = 234) -> Code:
    """CRC[n, k]: codewords m(x) x^(n-k) + (m(x) x^(n-k) mod g(x)), i.e. the
    multiples of g(x); g is the smallest primitive polynomial of degree
    n - k (the paper does not print its generator)."""
    return cyclic_code("crc(%d,%d)" % (n, k), n, k, smallest_primitive_poly(n - k))


def bch(n: int = 127, k: int = 113, m: int = 7, prim: int = 0b10001001,
        t: int = 2) -> Code:
    """Binary narrow-sense BCH code, g(x) = lcm(m_1, m_3, ..., m_{2t-1})."""
    g = 1
    seen = []
    for j in range(1, 2 * t, 2):
        mp = _minimal_poly(j, m, prim)
        if mp not in seen:
            seen.append(mp)
            g = _poly_mul2(g, mp)
    assert _poly_mod2((1 << n) | 1, g) == 0  # g divides x^n + 1
    return cyclic_code("bch(%d,%d)" % (n, k), n, k, g)


# ----------------------------------------------------------- CA-Polar ----

CRC11_POLY = (1 << 11) | (1 << 10) | (1 << 9) | (1 << 5) | 1


def crc_bits(msg_bits, poly=CRC11_POLY):
    """Remainder of m(x) x^deg mod g(x), MSB first, zero initial state."""
    deg = poly.bit_length() - 1
    reg = 0
    for b in list(msg_bits) + [0] * deg:
        reg = (reg << 1) | int(b)
        if reg >> deg:
            reg ^= poly
    return [(reg >> (deg - 1 - i)) & 1 for i in range(deg)]


def polar_transform(u):
    """x = u F^(x)m in natural order, F = [[1,0],[1,1]]."""
    x = np.array(u, dtype=np.uint8).copy()
    N = x.shape[-1]
    h = 1
    while h < N:
        for i in range(0, N, 2 * h):
            x[..., i:i + h] ^= x[..., i + h:i + 2 * h]
        h *= 2
    return x


def bhattacharyya_positions(N, K, design_ebn0_db, rate):
    """K most reliable synthetic channels of F^(x)m, natural order:
    z0 = exp(-R Eb/N0); z <- concat(2z - z^2, z^2) per level."""
    z = np.array([math.exp(-rate * 10 ** (design_ebn0_db / 10.0))])
    while z.shape[0] < N:
        z = np.concatenate([2 * z - z * z, z * z])
    order = sorted(range(N), key=lambda i: (z[i], i))
    return sorted(order[:K])


def ca_polar(N: int = 128, K: int = 105, crc_poly: int = CRC11_POLY,
             design_ebn0_db: float = 3.0) -> Code:
    ncrc = crc_poly.bit_length() - 1
    kmsg = K - ncrc
    rate = kmsg / N
    pos = bhattacharyya_positions(N, K, design_ebn0_db, rate)
    G = np.zeros((kmsg, N), np.uint8)
    for i in range(kmsg):
        msg = [0] * kmsg
        msg[i] = 1
        u = np.zeros(N, np.uint8)
        u[pos] = np.array(msg + crc_bits(msg, crc_poly), np.uint8)
        G[i] = polar_transform(u)
    assert gf2_rank(G) == kmsg
    H = gf2_nullspace(G)
    assert H.shape == (N - kmsg, N)
    _check(G, H)
    return Code("ca-polar(%d,%d[K=%d])" % (N, kmsg, K), N, kmsg, G, H)


# ------------------------------------------------------------- channel ----

def sigma_for(ebn0_db, rate):
    return math.sqrt(1.0 / (2.0 * rate * 10 ** (ebn0_db / 10.0)))


def encode(G, info):
    """c = m G over GF(2).  The product is taken in float32, which is exact
    here (every sum is an integer <= k <= 256), then reduced mod 2."""
    prod = info.astype(np.float32) @ G.astype(np.float32)
    return (prod.astype(np.int64) % 2).astype(np.uint8)


def awgn_llr(code: Code, B: int, ebn0_db, seed: int, zero_info=False):
    """B blocks through BPSK/AWGN.  ebn0_db is a scalar or a per-block array.
    Returns (llr float32 [B][n], transmitted codewords uint8 [B][n]).
    Draw order: info bits (B x k) then noise (B x n), one generator."""
    rng = np.random.default_rng(seed)
    if zero_info:
        info = np.zeros((B, code.k), np.uint8)
        rng.integers(0, 2, size=(B, code.k), dtype=np.uint8)  # keep draw order
    else:
        info = rng.integers(0, 2, size=(B, code.k), dtype=np.uint8)
    cw = encode(code.G, info)
    ebn0 = np.broadcast_to(np.asarray(ebn0_db, dtype=np.float64), (B,))
    sigma = np.sqrt(1.0 / (2.0 * (code.k / code.n) * 10 ** (ebn0 / 10.0)))
    noise = rng.standard_normal(size=(B, code.n))
    y = (2.0 * cw.astype(np.float64) - 1.0) + sigma[:, None] * noise
    llr = (2.0 * y / (sigma[:, None] ** 2)).astype(np.float32)
    return llr, cw


# ------------------------------------------------- the benchmark configs ----

def config1_code():
    return rlc(64, 51, seed=1)


def config2_code():
    return bch()


def config3_code():
    return ca_polar()


def config4_codes():
    return [rlc(64, 51, 41), rlc(128, 112, 42), rlc(256, 240, 43),
            rlc(256, 232, 44)]


def config1_inputs(B=10_000):
    """RLC(64,51) at 5 dB: all-zero information (seed 101) and random
    information (seed 102), B blocks each."""
    code = config1_code()
    l0, c0 = awgn_llr(code, B, 5.0, 101, zero_info=True)
    l1, c1 = awgn_llr(code, B, 5.0, 102)
    return code, np.concatenate([l0, l1]), np.concatenate([c0, c1])


def config2_inputs(B_per_point=100_000, points=(4.0, 5.0, 6.0, 7.0),
                   seeds=(201, 202, 203, 204)):
    code = config2_code()
    ls, cs = [], []
    for e, s in zip(points, seeds):
        l, c = awgn_llr(code, B_per_point, e, s)
        ls.append(l)
        cs.append(c)
    return code, np.concatenate(ls), np.concatenate(cs)


def config3_inputs(B_per_point=100_000, points=(3.0, 4.0, 5.0, 6.0),
                   seeds=(301, 302, 303, 304)):
    code = config3_code()
    ls, cs = [], []
    for e, s in zip(points, seeds):
        l, c = awgn_llr(code, B_per_point, e, s)
        ls.append(l)
        cs.append(c)
    return code, np.concatenate(ls), np.concatenate(cs)


def config4_inputs(B=1_000_000, seed=401):
    """Mixed batch: code id uniform per block, Eb/N0 uniform in [4, 7] dB.
    Returns (codes, code_id[B], llr list per block as a flat float32 array,
    llr_offset[B], codewords flat, ebn0[B])."""
    return mixed_inputs(config4_codes(), B, seed)


def capolar256_code():
    """CA-Polar[256, 234] of Sec. IV (K = 245 polar positions: 234 message
    bits and the CRC-11), as in paper256_codes."""
    return ca_polar(256, 245)


def paper256_codes():
    """The [256, 234]-class codes of Sec. IV's first comparison."""
    return [ca_polar(256, 245), crc_code(256, 234), rlc(256, 234, seed=61),
            bch(255, 231, m=8, prim=0b100011101, t=3)]


def paper256_inputs(B=400_000, seed=601):
    """The paper-shaped mixed batch: the four [256, 234]-class codes, code
    uniform per block, Eb/N0 uniform in [4, 7] dB (as config4_inputs)."""
    return mixed_inputs(paper256_codes(), B, seed)


def mixed_inputs(codes, B, seed, ebn0_lo=4.0, ebn0_hi=7.0):
    """Blocks of several codes: code id uniform per block, Eb/N0 uniform in
    [ebn0_lo, ebn0_hi] dB; blocks laid out back to back.  Returns (codes,
    code_id[B], llr flat float32, llr_offset[B], codewords flat, ebn0[B])."""
    rng = np.random.default_rng(seed)
    cid = rng.integers(0, len(codes), size=B).astype(np.int32)
    ebn0 = rng.uniform(ebn0_lo, ebn0_hi, size=B)
    ns = np.array([c.n for c in codes], np.int64)
    lens = ns[cid]
    off = np.zeros(B, np.int64)
    off[1:] = np.cumsum(lens)[:-1]
    llr = np.zeros(int(lens.sum()), np.float32)
    cw = np.zeros(int(lens.sum()), np.uint8)
    for j, code in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        l, c = awgn_llr(code, idx.shape[0], ebn0[idx], seed * 10 + j)
        pos = off[idx][:, None] + np.arange(code.n)[None, :]
        llr[pos] = l
        cw[pos] = c
    return codes, cid, llr, off, cw, ebn0


def config5_codes():
    """The serving mix: BCH(127,113), CA-Polar(128,94[K=105]), RLC(128,112)."""
    return [bch(), ca_polar(), rlc(128, 112, seed=42)]


def serving_trace(rate_blocks_s=2e6, seconds=10.0, max_size=4096, ebn0=(3.0, 7.0),
                  seed=501, codes=None):
    """Poisson request stream: request sizes U{1..max_size} blocks, code
    uniform over `codes`, Eb/N0 uniform in `ebn0` per request; arrivals with
    exponential gaps at rate_blocks_s / E[size] requests per second, over
    `seconds`.  Returns a dict of arrays (arrival_s, code, B, ebn0,
    llr_off, blk_off) plus llr_all (float32) and cw_all (transmitted)."""
    codes = codes if codes is not None else config5_codes()
    rng = np.random.default_rng(seed)
    mean_size = (1 + max_size) / 2.0
    req_rate = rate_blocks_s / mean_size
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / req_rate)
        if t >= seconds:
            break
        arrivals.append(t)
    m = len(arrivals)
    size = rng.integers(1, max_size + 1, size=m).astype(np.int64)
    code = rng.integers(0, len(codes), size=m).astype(np.int32)
    eb = rng.uniform(ebn0[0], ebn0[1], size=m)
    ns = np.array([c.n for c in codes], np.int64)
    elems = size * ns[code]
    llr_off = np.zeros(m, np.int64)
    llr_off[1:] = np.cumsum(elems)[:-1]
    blk_off = np.zeros(m, np.int64)
    blk_off[1:] = np.cumsum(size)[:-1]
    llr_all = np.zeros(int(elems.sum()), np.float32)
    cw_all = np.zeros(int(elems.sum()), np.uint8)
    for j, cd in enumerate(codes):
        reqs = np.nonzero(code == j)[0]
        if reqs.size == 0:
            continue
        per_block_eb = np.repeat(eb[reqs], size[reqs])
        l, c = awgn_llr(cd, int(size[reqs].sum()), per_block_eb, seed * 10 + j)
        pos = 0
        for r in reqs:
            k = int(size[r])
            llr_all[llr_off[r]:llr_off[r] + k * cd.n] = l[pos:pos + k].ravel()
            cw_all[llr_off[r]:llr_off[r] + k * cd.n] = c[pos:pos + k].ravel()
            pos += k
    return {"arrival_s": np.array(arrivals, np.float64), "code": code, "B": size,
            "ebn0": eb, "llr_off": llr_off, "blk_off": blk_off, "llr_all": llr_all,
            "cw_all": cw_all, "codes": codes}


def serving_pool(codes=None, pool_blocks=1 << 19, ebn0=(3.0, 7.0), seed=511):
    """Blocks for long serving traces: per code, pool_blocks blocks whose
    Eb/N0 rises linearly from ebn0[0] to ebn0[1] over the pool's rows.
    Returns (codes, llr flat float32, pool_off[code] (element offset of the
    code's first row), cw flat)."""
    codes = codes if codes is not None else config5_codes()
    eb = np.linspace(ebn0[0], ebn0[1], pool_blocks)
    ns = np.array([c.n for c in codes], np.int64)
    pool_off = np.concatenate([[0], np.cumsum(ns * pool_blocks)[:-1]]).astype(np.int64)
    llr = np.zeros(int((ns * pool_blocks).sum()), np.float32)
    cw = np.zeros(llr.shape[0], np.uint8)
    for j, cd in enumerate(codes):
        l, c = awgn_llr(cd, pool_blocks, eb, seed * 10 + j)
        llr[pool_off[j]:pool_off[j] + cd.n * pool_blocks] = l.ravel()
        cw[pool_off[j]:pool_off[j] + cd.n * pool_blocks] = c.ravel()
    return codes, llr, pool_off, cw


def pooled_serving_trace(pool, pool_blocks, rate_blocks_s=2e6, seconds=10.0, max_size=4096,
                         ebn0=(3.0, 7.0), seed=501):
    """A Poisson request stream as serving_trace (sizes U{1..max_size}, code
    uniform, Eb/N0 uniform per request, exponential gaps) whose blocks are
    rows of a serving_pool: request r reads the B_r consecutive rows of its
    code's pool that start where the pool's Eb/N0 equals the request's, so
    a long trace needs no new blocks.  Requests may share rows (their
    codeword outputs then land on the same bytes: the decoder is
    deterministic, so they agree).  Returns the dict of serving_trace,
    with llr_all the pool's array and `pool_row[r]` the first row."""
    codes, llr, pool_off, cw = pool
    rng = np.random.default_rng(seed)
    mean_size = (1 + max_size) / 2.0
    req_rate = rate_blocks_s / mean_size
    m_est = int(req_rate * seconds * 1.2) + 16
    gaps = rng.exponential(1.0 / req_rate, size=m_est)
    arrivals = np.cumsum(gaps)
    while arrivals[-1] < seconds:
        more = np.cumsum(rng.exponential(1.0 / req_rate, size=m_est)) + arrivals[-1]
        arrivals = np.concatenate([arrivals, more])
    arrivals = arrivals[arrivals < seconds]
    m = arrivals.shape[0]
    size = rng.integers(1, max_size + 1, size=m).astype(np.int64)
    code = rng.integers(0, len(codes), size=m).astype(np.int32)
    eb = rng.uniform(ebn0[0], ebn0[1], size=m)
    ns = np.array([c.n for c in codes], np.int64)
    frac = (eb - ebn0[0]) / (ebn0[1] - ebn0[0])
    row = np.round(frac * (pool_blocks - size)).astype(np.int64)
    llr_off = pool_off[code] + row * ns[code]
    blk_off = np.zeros(m, np.int64)
    blk_off[1:] = np.cumsum(size)[:-1]
    return {"arrival_s": arrivals.astype(np.float64), "code": code, "B": size, "ebn0": eb,
            "llr_off": llr_off, "blk_off": blk_off, "llr_all": llr, "cw_all": cw,
            "codes": codes, "pool_row": row}
