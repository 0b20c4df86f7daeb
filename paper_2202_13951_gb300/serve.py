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


def measure(seconds=10.0, rate=2e6, budget_mb=2048, streams=4, max_batch=1 << 18,
            cap=10 ** 6, pool_blocks=1 << 18, probe_seconds=1.0, seed=501):
    """The serving measurement of the benchmark: Poisson traces over a
    serving_pool (BCH, CA-Polar, RLC(128,112); Eb/N0 U[3,7] dB per request;
    sizes U{1..4096}): a short trace offered far above capacity (its
    achieved rate is the capacity), then `seconds` of arrivals at half that
    capacity and at `rate`.  Every request's queries and abandon flags, and
    the codewords, are compared with one batched decode of the whole pool
    (each block alone, outside any mix)."""
    build.build()
    orbg.load_library()
    import torch
    t0 = time.time()
    pool = workloads.serving_pool(pool_blocks=pool_blocks, seed=seed + 10)
    codes_h, llr, pool_off, _ = pool
    gen_s = time.time() - t0
    # the whole pool decoded once, batched (the reference for every request)
    codes = [orbg.Code(c.H, max_query_cap=cap) for c in codes_h]
    cs = orbg.CodeSet(codes)
    ns = np.array([c.n for c in codes_h], np.int64)
    cid = np.repeat(np.arange(len(codes_h), dtype=np.int32), pool_blocks)
    off = np.concatenate([pool_off[j] + np.arange(pool_blocks, dtype=np.int64) * ns[j]
                          for j in range(len(codes_h))])
    dev = torch.device("cuda")
    cw_d, q_d, ab_d = orbg.decode_batched(cs, torch.from_numpy(llr).to(dev), cap,
                                          code_id=torch.from_numpy(cid).to(dev),
                                          llr_offset=torch.from_numpy(off).to(dev),
                                          cw_offset=torch.from_numpy(off).to(dev),
                                          n_total=llr.shape[0])
    torch.cuda.synchronize()
    want_cw = cw_d.cpu().numpy()
    want_q = q_d.cpu().numpy().astype(np.int64).reshape(len(codes_h), pool_blocks)
    want_ab = ab_d.cpu().numpy().reshape(len(codes_h), pool_blocks)
    del cw_d, q_d, ab_d
    cs.close()
    for c in codes:
        c.close()

    def one(rate_b, secs, sd):
        tr = workloads.pooled_serving_trace(pool, pool_blocks, rate_blocks_s=rate_b,
                                            seconds=secs, seed=sd)
        res, (cw, q, ab, lat), _ = run(rate_b, secs, budget_mb, streams, max_batch, cap,
                                       trace=tr)
        bad = 0
        for r in range(tr["B"].shape[0]):
            j, k, row, bo = int(tr["code"][r]), int(tr["B"][r]), int(tr["pool_row"][r]), \
                int(tr["blk_off"][r])
            bad += int(not (np.array_equal(q[bo:bo + k].astype(np.int64),
                                           want_q[j, row:row + k]) and
                            np.array_equal(ab[bo:bo + k], want_ab[j, row:row + k])))
        touched = np.zeros(llr.shape[0], bool)
        for r in range(tr["B"].shape[0]):
            j = int(tr["code"][r])
            lo = int(tr["llr_off"][r])
            touched[lo:lo + int(tr["B"][r]) * int(ns[j])] = True
        cw_ok = bool(np.array_equal(cw[touched], want_cw[touched]))
        res["same_as_alone"] = {"requests": int(tr["B"].shape[0]),
                                "requests_differing": bad, "codewords_equal": cw_ok,
                                "what": "each request's queries, abandon flags and codewords "
                                        "equal one batched decode of the pool (each block "
                                        "alone, outside the mix)"}
        res["offered_blocks_s"] = rate_b
        res.pop("trace_gen_s", None)
        return res

    probe = one(2e7, probe_seconds, seed + 1)
    capacity = probe["achieved_blocks_s"] or rate
    half = one(0.5 * capacity, seconds, seed + 2)
    at_rate = one(rate, seconds, seed)
    return {"workload": at_rate["workload"] + "; blocks are rows of a pool of %d blocks per "
            "code whose Eb/N0 spans [3,7] dB, a request reading the rows at its own Eb/N0"
            % pool_blocks,
            "capacity_probe": probe, "half_capacity": half, "offered": at_rate,
            "pool_gen_s": gen_s}


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--rate", type=float, default=2e6)
    p.add_argument("--seconds", type=float, default=2.0)
    p.add_argument("--budget-mb", type=int, default=2048)
    p.add_argument("--streams", type=int, default=4)
    p.add_argument("--max-batch", type=int, default=1 << 18)
    p.add_argument("--seed", type=int, default=501)
    p.add_argument("--measure", action="store_true",
                   help="the benchmark's measurement: capacity, half capacity and --rate, "
                        "on pooled traces of --seconds, each checked against the blocks "
                        "decoded alone")
    a = p.parse_args()
    if a.measure:
        print(json.dumps(measure(a.seconds, a.rate, a.budget_mb, a.streams, a.max_batch,
                                 seed=a.seed)))
        return
    res, _, _ = run(a.rate, a.seconds, a.budget_mb, a.streams, a.max_batch, seed=a.seed)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
