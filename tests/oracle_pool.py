"""The oracle over all host cores for the larger GPU parity samples:
blocks are split into chunks decoded by spawned single-threaded oracle
processes (spawned, not forked, because the test process already holds a
CUDA context)."""
import multiprocessing as mp
import os

import numpy as np


def _decode(args):
    H, rows, cap = args
    import oracle
    return oracle.decode_batch(H, rows, cap)


def decode_batch(H, llr, cap, chunk=64):
    """oracle.decode_batch(H, llr, cap) computed on all host cores."""
    if llr.shape[0] <= chunk:
        return _decode((H, llr, cap))
    parts = [(H, llr[i:i + chunk], cap) for i in range(0, llr.shape[0], chunk)]
    with mp.get_context("spawn").Pool(min(len(parts), os.cpu_count() or 1)) as pool:
        res = pool.map(_decode, parts)
    return tuple(np.concatenate([r[k] for r in res]) for k in range(4))
