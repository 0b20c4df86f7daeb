"""Brute-force basic and one-line full ORBGRAND for tiny codes (n <= 16): a
third, independent implementation used to pin the oracle.

It lists all 2^n noise patterns, sorts them by (logistic weight, Hamming
weight, positions lexicographically) -- the canonical reading of the
paper's arbitrary tie order -- and decodes by testing H c = 0 directly
(the plain definition of code-book membership), with no syndrome
bookkeeping and no partition generator.
"""
import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def query_order(n):
    """All subsets of {1..n} in the canonical query order."""
    pats = []
    for mask in range(1 << n):
        v = tuple(i + 1 for i in range(n) if (mask >> i) & 1)
        pats.append((sum(v), len(v), v))
    pats.sort()
    return tuple(p[2] for p in pats)


def reliability_order(llr):
    """Received indices sorted by increasing |LLR| (FP32), lower index first
    among equal reliabilities."""
    rel = np.abs(np.asarray(llr, dtype=np.float32))
    return sorted(range(len(rel)), key=lambda i: (float(rel[i]), i))


def decode(H, llr, cap):
    """Returns (codeword, queries, abandoned)."""
    H = np.asarray(H, dtype=np.int64)
    llr = np.asarray(llr, dtype=np.float32)
    n = llr.shape[0]
    y = (llr > 0).astype(np.uint8)
    pi = reliability_order(llr)
    for t, v in enumerate(query_order(n), start=1):
        if t > cap:
            return y.copy(), cap, 1
        c = y.copy()
        for p in v:
            c[pi[p - 1]] ^= 1
        if not ((H @ c.astype(np.int64)) % 2).any():
            return c, t, 0
    return y.copy(), len(query_order(n)), 1


@functools.lru_cache(maxsize=None)
def query_order_1line(n, J0, beta):
    """All subsets of {1..n} sorted by (reliability weight J0 |v| + beta sum(v),
    Hamming weight, positions lexicographically): one-line full ORBGRAND
    (Sec. III-D: sorted position j is worth J0 + beta j) with the same
    canonical tie order."""
    pats = []
    for mask in range(1 << n):
        v = tuple(i + 1 for i in range(n) if (mask >> i) & 1)
        pats.append((J0 * len(v) + beta * sum(v), len(v), v))
    pats.sort()
    return tuple(p[2] for p in pats)


def decode_1line(H, llr, cap, J0, beta):
    """decode() in the one-line order.  Returns (codeword, queries, abandoned)."""
    H = np.asarray(H, dtype=np.int64)
    llr = np.asarray(llr, dtype=np.float32)
    n = llr.shape[0]
    y = (llr > 0).astype(np.uint8)
    pi = reliability_order(llr)
    order = query_order_1line(n, J0, beta)
    for t, v in enumerate(order, start=1):
        if t > cap:
            return y.copy(), cap, 1
        c = y.copy()
        for p in v:
            c[pi[p - 1]] ^= 1
        if not ((H @ c.astype(np.int64)) % 2).any():
            return c, t, 0
    return y.copy(), len(order), 1


def model_weights(n, model):
    """rho_j for sorted positions j = 1..n under the piece-wise linear model
    (anchors I_1..I_{m-1}, J_0..J_{m-1}, beta_1..beta_m) of Eq. relest_seg."""
    anchors, J, beta = model
    I = [0] + list(anchors) + [n]
    rho = []
    for i in range(len(J)):
        for j in range(I[i] + 1, I[i + 1] + 1):
            rho.append(J[i] + beta[i] * (j - I[i]))
    return rho


@functools.lru_cache(maxsize=None)
def query_order_model(n, model):
    """All subsets of {1..n} sorted by (sum of rho over the subset, Hamming
    weight, positions lexicographically): m-segment full ORBGRAND with the
    canonical tie order."""
    rho = model_weights(n, model)
    pats = []
    for mask in range(1 << n):
        v = tuple(i + 1 for i in range(n) if (mask >> i) & 1)
        pats.append((sum(rho[p - 1] for p in v), len(v), v))
    pats.sort()
    return tuple(p[2] for p in pats)


def decode_model(H, llr, cap, model):
    """decode() in the m-segment order.  Returns (codeword, queries, abandoned)."""
    H = np.asarray(H, dtype=np.int64)
    llr = np.asarray(llr, dtype=np.float32)
    n = llr.shape[0]
    y = (llr > 0).astype(np.uint8)
    pi = reliability_order(llr)
    order = query_order_model(n, model)
    for t, v in enumerate(order, start=1):
        if t > cap:
            return y.copy(), cap, 1
        c = y.copy()
        for p in v:
            c[pi[p - 1]] ^= 1
        if not ((H @ c.astype(np.int64)) % 2).any():
            return c, t, 0
    return y.copy(), len(order), 1
