"""Oracle outputs of the benchmark configurations, computed once and kept.

TEST INFRASTRUCTURE ONLY: like the rest of oracle/, nothing on the product
path may import or run this.  It decodes every block of a configuration
with the CPU oracle (orbg_oracle.c, basic ORBGRAND: Algorithm 1 with the
Landslide generator of Algorithm 2), sharded over the host cores in
spawned single-threaded processes, and stores codeword bytes, query
counts, abandon flags and the oracle's sum of the queries' Hamming weights
per block in an .npz file named for the configuration and its seeds.  The
inputs come from paper_2202_13951_gb300.workloads, the seeded generators
both sides share (they hold none of the decoder's arithmetic).

    python -m oracle.cache --config 2 [--procs N] [--dir oracle/_cache]

A cached file records the SHA-256 of orbg_oracle.c it was made with;
load() ignores files made with another oracle.
"""
import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)
DEFAULT_DIR = os.path.join(_HERE, "_cache")

# configuration -> (query cap, seeds, what)
CONFIGS = {
    1: (100_000, (101, 102), "rlc(64,51), 2 x 10,000 blocks at 5 dB (all-zero, random info)"),
    2: (1_000_000, (201, 202, 203, 204), "bch(127,113), 4 x 100,000 blocks at 4-7 dB"),
    3: (1_000_000, (301, 302, 303, 304), "ca-polar(128,94[K=105]), 4 x 100,000 blocks at 3-6 dB"),
    4: (1_000_000, (401,), "mixed rlc(64,51),(128,112),(256,240),(256,232), 1,000,000 blocks"),
}


def oracle_digest():
    with open(os.path.join(_HERE, "orbg_oracle.c"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def inputs(config):
    """(codes, code_id[B], llr flat, llr_offset[B]) of a configuration."""
    from paper_2202_13951_gb300 import workloads
    if config == 4:
        codes, cid, llr, off, _, _ = workloads.config4_inputs()
        return codes, cid, llr, off
    if config == 1:
        code, llr, _ = workloads.config1_inputs()
    elif config == 2:
        code, llr, _ = workloads.config2_inputs()
    elif config == 3:
        code, llr, _ = workloads.config3_inputs()
    else:
        raise ValueError("no configuration %r" % config)
    B = llr.shape[0]
    return ([code], np.zeros(B, np.int32), np.ascontiguousarray(llr).ravel(),
            np.arange(B, dtype=np.int64) * code.n)


def _work(args):
    idx, H, rows, cap = args
    import oracle
    cw, q, ab, sw = oracle.decode_batch(H, rows, cap)
    return idx, cw, q, ab, sw


def path_for(config, directory=DEFAULT_DIR):
    cap, seeds, _ = CONFIGS[config]
    return os.path.join(directory, "config%d_seeds%s_cap%d.npz"
                        % (config, "-".join(str(s) for s in seeds), cap))


def compute(config, procs=None, directory=DEFAULT_DIR, chunk=500):
    """Decode every block of `config` with the oracle; store and return the
    arrays (cw flat as the inputs, q, ab, sw per block)."""
    import oracle
    oracle.build_oracle()
    cap = CONFIGS[config][0]
    codes, cid, llr, off = inputs(config)
    B = cid.shape[0]
    n_of = np.array([c.n for c in codes], np.int64)[cid]
    cw = np.zeros(llr.shape[0], np.uint8)
    q = np.zeros(B, np.uint64)
    ab = np.zeros(B, np.uint8)
    sw = np.zeros(B, np.uint64)
    tasks = []
    for j, code in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        for c in range(0, idx.size, chunk):
            sel = idx[c:c + chunk]
            rows = np.stack([llr[off[b]:off[b] + code.n] for b in sel])
            tasks.append((sel, code.H, rows, cap))
    procs = procs or os.cpu_count() or 1
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        for sel, c_, q_, a_, s_ in pool.imap_unordered(_work, tasks):
            for k, b in enumerate(sel):
                cw[off[b]:off[b] + n_of[b]] = c_[k]
            q[sel], ab[sel], sw[sel] = q_, a_, s_
    os.makedirs(directory, exist_ok=True)
    out = path_for(config, directory)
    tmp = out + ".%d.tmp.npz" % os.getpid()
    np.savez(tmp, cw=cw, q=q, ab=ab, sw=sw, digest=np.array(oracle_digest()))
    os.replace(tmp, out)
    return {"config": config, "blocks": B, "seconds": time.time() - t0, "procs": procs,
            "path": out}


def load(config, directory=DEFAULT_DIR):
    """The cached outputs of `config` (dict of arrays), or None when absent
    or made with another version of the oracle."""
    p = path_for(config, directory)
    if not os.path.exists(p):
        return None
    d = np.load(p)
    if str(d["digest"]) != oracle_digest():
        return None
    return {k: d[k] for k in ("cw", "q", "ab", "sw")}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", type=int, action="append", required=True,
                    choices=sorted(CONFIGS))
    ap.add_argument("--procs", type=int, default=0)
    ap.add_argument("--dir", default=DEFAULT_DIR)
    a = ap.parse_args()
    for c in a.config:
        print(compute(c, a.procs or None, a.dir), flush=True)


if __name__ == "__main__":
    main()
