"""Continuous-batching decode server: replay a Poisson request trace through
orbg_server (include/orbg.h) and report latency and throughput.

    python -m paper_2202_13951_gb300.serve [--rate 2e6] [--seconds 2]
        [--budget-mb 2048] [--streams 4] [--max-batch 262144]

Prints one JSON line: offered and achieved blocks/s, p50/p99/max request
latency (submit to results on the host), batches formed and the most
batches in flight at once.
"""
import argparse
import json
import time

import numpy as np

from . import build, orbg, workloads


def run(rate=2e6, seconds=2.0, budget_mb=2048, streams=4, max_batch=1 << 18, cap=10 ** 6,
        seed=501, tuning=None, trace=None):
    build.build()
    orbg.load_library()
    t0 = time.time()
    tr = trace or workloads.serving_trace(rate_blocks_s=rate, seconds=seconds, seed=seed)
    gen_s = time.time() - t0
    codes = [orbg.Code(c.H, max_query_cap=cap) for c in tr["codes"]]
    cs = orbg.CodeSet(codes)
    if tuning:
        orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(*tuning))
    srv = orbg.orbg_server_create(cs.handle, budget_mb << 20, cap, streams, max_batch)
    m = tr["arrival_s"].shape[0]
    nblocks = int(tr["B"].sum())
    cw = np.zeros(tr["llr_all"].shape[0], np.uint8)
    q = np.zeros(nblocks, np.uint32)
    ab = np.zeros(nblocks, np.uint8)
    lat = np.zeros(m, np.float64)
    try:
        wall = orbg.orbg_server_replay(srv, tr["arrival_s"], tr["code"], tr["B"], tr["llr_off"],
                                       tr["blk_off"], tr["llr_all"], cw, q, ab, lat)
        stats = orbg.orbg_server_stats_get(srv)
    finally:
        orbg.orbg_server_destroy(srv)
    span = float(tr["arrival_s"][-1]) if m else 0.0
    res = {
        "workload": "serving: BCH(127,113), CA-Polar(128,94[K=105]), RLC(128,112); Poisson "
                    "arrivals, sizes U{1..4096}, Eb/N0 U[3,7] dB per request, cap %d" % cap,
        "offered_blocks_s": rate, "arrival_span_s": span, "requests": m, "blocks": nblocks,
        "achieved_blocks_s": nblocks / wall if wall > 0 else None, "wall_s": wall,
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                       "p99": 1e3 * float(np.percentile(lat, 99)),
                       "max": 1e3 * float(lat.max()), "mean": 1e3 * float(lat.mean())},
        "abandon_rate": float(ab.mean()), "mean_queries": float(q.mean()),
        "server": stats, "budget_mb": budget_mb, "streams": streams,
        "max_batch_blocks": max_batch, "trace_gen_s": gen_s,
    }
    return res, (cw, q, ab, lat), tr


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--rate", type=float, default=2e6)
    p.add_argument("--seconds", type=float, default=2.0)
    p.add_argument("--budget-mb", type=int, default=2048)
    p.add_argument("--streams", type=int, default=4)
    p.add_argument("--max-batch", type=int, default=1 << 18)
    p.add_argument("--seed", type=int, default=501)
    a = p.parse_args()
    res, _, _ = run(a.rate, a.seconds, a.budget_mb, a.streams, a.max_batch, seed=a.seed)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
