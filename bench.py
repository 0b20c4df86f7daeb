#!/usr/bin/env python3
"""Throughput of the GB300 basic-ORBGRAND decoder.

One step = one batched persistent launch (orbg_decode_batched) over the
whole mixed workload: 1,000,000 blocks, each of a random linear code drawn
uniformly from (64,51), (128,112), (256,240) and (256,232), at Eb/N0
uniform in [4, 7] dB, query cap 1e6 -- every block sorted, searched and
written back.  Inputs (576 MB, larger than the 129 MB L2) are resident in
HBM when the timed region starts; the code tables stay resident.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU: each rank decodes its own
workload (seeds offset by rank), there is no data-path collective (blocks
are independent), and the timing is the max over ranks (weak scaling).
``--impl reference`` times the CPU oracle on the host cores instead, on a
bounded sample of the same workload.

Prints one JSON line (rank 0).  Besides the timing it carries ``parity``:
the GPU outputs of the timed step compared bit for bit with the oracle on
a stratified sample of the blocks (the whole workload where that is cheap).
At N = 1 on the default workload the line also carries ``forms`` (the
BCH(127,113) workload through the plain single launch and the batched form,
same inputs, same BLER), ``serving`` (the continuous-batching server on a
Poisson trace) and ``extra_workloads`` (full ORBGRAND orders, Sec. III-D and
III-E, and the paper-shaped [256,234] workload), each measured in its own
process after the headline (``--no-extra`` skips them).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("decoded blocks/s and syndrome queries/s (bit-exact vs oracle) "
          "+ p99 latency")
# name -> (description, code constructor name, Eb/N0 points, seeds)
WORKLOADS = {
    "bch": ("bch(127,113) 4x%d blocks at Eb/N0 4,5,6,7 dB, query cap 1e6",
            "config2_code", (4.0, 5.0, 6.0, 7.0), (201, 202, 203, 204)),
    "capolar": ("ca-polar(128,94[K=105]) 4x%d blocks at Eb/N0 3,4,5,6 dB, query cap 1e6",
                "config3_code", (3.0, 4.0, 5.0, 6.0), (301, 302, 303, 304)),
    "rlc64": ("rlc(64,51) 2x%d blocks at Eb/N0 5 dB (all-zero and random information), "
              "query cap 1e5", "config1_code", (5.0, 5.0), (101, 102)),
    "mixed": ("mixed rlc(64,51),(128,112),(256,240),(256,232), code uniform per block, "
              "%d blocks at Eb/N0 U[4,7] dB, query cap 1e6, one launch, autotuned",
              None, (), (401,)),
    "capolar256": ("ca-polar(256,234[K=245]) 4x%d blocks at Eb/N0 5,5.1,5.2,5.3 dB, "
                   "query cap 5e6", "capolar256_code", (5.0, 5.1, 5.2, 5.3),
                   (701, 702, 703, 704)),
    "paper256": ("paper-shaped [256,234] family: ca-polar(256,234[K=245]), crc(256,234), "
                 "rlc(256,234), bch(255,231), code uniform per block, %d blocks at Eb/N0 "
                 "U[4,7] dB, query cap 5e6, one launch, autotuned",
                 None, (), (601,)),
}
# multi-code workloads: generator of (codes, code_id, llr, llr_offset, codewords, ebn0)
# and blocks per step as a multiple of --blocks-per-point
MIXED = {"mixed": ("config4_inputs", 10), "paper256": ("paper256_inputs", 4)}
POINTS = (4.0, 5.0, 6.0, 7.0)
SEEDS = (201, 202, 203, 204)
B_PER_POINT = 100_000
WORKLOAD = WORKLOADS["bch"][0] % B_PER_POINT
CAP = 1_000_000
CAPS = {"rlc64": 100_000, "paper256": 5_000_000, "capolar256": 5_000_000}


# ------------------------------------------------------------------ utils

def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--line", default="",
                   help="J0,beta: decode one-line full ORBGRAND (Sec. III-D) instead of basic")
    p.add_argument("--model", default="",
                   help="I_1,..;J_0,..;beta_1,..: decode m-segment full ORBGRAND (Sec. III-D, "
                        "Eq. relest_seg) under this model instead of basic")
    p.add_argument("--fitted", action="store_true",
                   help="decode one-line full ORBGRAND with a line fitted per block "
                        "(Sec. III-E; orbg_fitted_decode) instead of basic")
    p.add_argument("--fitted-lines", type=int, default=0,
                   help="decode full ORBGRAND with a model of this many lines fitted per "
                        "block, each block searched in its own order (Sec. III-E, III-D; "
                        "orbg_decode_fitted)")
    p.add_argument("--divisible", action="store_true",
                   help="with --fitted-lines: Eq. quant's J-divisible quantisation")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the secondary measurements (full ORBGRAND orders, the "
                        "paper-shaped workload) that follow the headline one")
    p.add_argument("--no-graph", action="store_true",
                   help="time direct calls instead of replays of a captured CUDA graph")
    p.add_argument("--ref-sample", type=int, default=8000,
                   help="blocks per reference step (CPU oracle)")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="mixed",
                   help="mixed: the headline configuration (1,000,000 blocks of four "
                        "random codes); bch, capolar, rlc64: the single-code "
                        "configurations; paper256: the paper-shaped [256,234] family")
    p.add_argument("--no-parity", action="store_true",
                   help="skip the oracle comparison of the timed step's outputs")
    p.add_argument("--parity-budget", type=float, default=60.0,
                   help="seconds of host-core time (wall) the oracle comparison may take")
    p.add_argument("--parity-per-code", type=int, default=20000,
                   help="blocks of each code the oracle comparison aims to check")
    p.add_argument("--no-serving", action="store_true",
                   help="skip the serving measurement of the default run")
    p.add_argument("--serving-seconds", type=float, default=10.0,
                   help="seconds of Poisson arrivals in the serving measurement")
    p.add_argument("--blocks-per-point", type=int, default=B_PER_POINT)
    p.add_argument("--points", default="",
                   help="Eb/N0 points (dB, comma-separated) in place of a single-code "
                        "workload's own; seeds follow the workload's first seed")
    p.add_argument("--form", choices=("batched", "plain"), default="batched",
                   help="batched: orbg_decode_batched (two persistent launches); plain: "
                        "orbg_decode (one warp per block, one launch)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the library's default tuning")
    p.add_argument("--shape", default="",
                   help="warps_per_cta,ctas_per_sm,blocks_per_grab,warp_budget,heavy_warps "
                        "for the batched launch (orbg_tuning)")
    p.add_argument("--cap", type=int, default=0,
                   help="query cap of the codes and calls (0 = the workload's own); a low "
                        "cap stops every search there, which times the fixed work a block "
                        "costs (loading, query 1, writing)")
    args = p.parse_args(argv)
    select_workload(args.workload, args.blocks_per_point)
    if args.points:
        set_points(tuple(float(x) for x in args.points.split(",")))
    global LINE, MODEL, FITTED, WORKLOAD, CAP
    if args.cap < 0:
        raise SystemExit("--cap must be positive")
    if args.cap:
        CAP = int(args.cap)
        head, tail = WORKLOAD.split("query cap ", 1)
        rest = tail.split(",", 1)
        WORKLOAD = head + "query cap %d" % CAP + ("," + rest[1] if len(rest) > 1 else "")
    if sum(map(bool, (args.line, args.model, args.fitted, args.fitted_lines))) > 1:
        raise SystemExit("give one of --line, --model, --fitted, --fitted-lines")
    FITTED = bool(args.fitted)
    if FITTED:
        WORKLOAD += ", one-line full ORBGRAND with a line fitted per block"
    if args.fitted_lines:
        FITTED = (int(args.fitted_lines), bool(args.divisible))
        WORKLOAD += (", full ORBGRAND with a %d-line model fitted per block%s"
                     % (FITTED[0], " (J divisible by beta)" if FITTED[1] else ""))
    if args.line:
        LINE = tuple(int(x) for x in args.line.split(","))
        WORKLOAD += ", one-line full ORBGRAND J0=%d beta=%d" % LINE
    if args.model:
        parts = [tuple(int(x) for x in f.split(",") if x.strip()) for f in args.model.split(";")]
        if len(parts) != 3 or len(parts[1]) != len(parts[2]) or len(parts[0]) + 1 != len(parts[1]):
            raise SystemExit("--model wants I_1..I_{m-1};J_0..J_{m-1};beta_1..beta_m")
        MODEL = tuple(parts)
        WORKLOAD += ", %d-segment full ORBGRAND %s" % (len(MODEL[1]), describe_model(MODEL))
    return args


def describe_model(model):
    return "I=%s J=%s beta=%s" % tuple(",".join(str(x) for x in f) or "-" for f in model)


def select_workload(name, b_per_point):
    global WORKLOAD, POINTS, SEEDS, B_PER_POINT, CODE_FN, WORKLOAD_NAME, CAP
    desc, CODE_FN, POINTS, SEEDS = WORKLOADS[name]
    WORKLOAD_NAME = name
    CAP = CAPS.get(name, 1_000_000)
    if name == "rlc64" and b_per_point == 100_000:
        b_per_point = 10_000  # the configuration's 2 x 10,000 blocks
    B_PER_POINT = b_per_point
    WORKLOAD = desc % (b_per_point * MIXED[name][1] if name in MIXED else b_per_point)


def set_points(points):
    """Another set of Eb/N0 points for a single-code workload."""
    global POINTS, SEEDS, WORKLOAD
    if WORKLOAD_NAME in MIXED:
        raise SystemExit("--points applies to single-code workloads")
    base = SEEDS[0]
    POINTS = tuple(points)
    SEEDS = tuple(base + 17 * i for i in range(len(POINTS)))
    head = WORKLOAD.split(" blocks at Eb/N0 ")[0].rsplit(" ", 1)[0]
    tail = WORKLOAD.split(" dB", 1)[1]
    WORKLOAD = "%s %dx%d blocks at Eb/N0 %s dB%s" % (
        head, len(POINTS), B_PER_POINT, ",".join("%g" % e for e in POINTS), tail)


WORKLOAD_NAME = "bch"
LINE = None  # (J0, beta) for one-line full ORBGRAND, None for basic
MODEL = None  # (anchors, J, beta) for m-segment full ORBGRAND, None for basic
# False; True: one-line full ORBGRAND with a line fitted per block through
# per-line tables (orbg_fitted_decode); (lines, divisible): a model of that
# many lines fitted per block, each block searched in its own order
# (orbg_decode_fitted)
FITTED = False
# Full ORBGRAND models for the secondary measurements on the BCH workload: the
# one- and three-line fits (Sec. III-E, Eq. Q, Eq. quant) of the mean ordered
# |LLR| curve of 10,000 of its blocks at 5.5 dB (seed 7); a CPU test recomputes
# them with the oracle.
EXTRA_LINE = (5, 1)
EXTRA_MODEL = ((7, 17), (3, 37, 58), (5, 2, 1))


CODE_FN = "config2_code"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def rank_seeds(rank):
    """Each rank decodes its own workload: seeds offset by 1000 * rank."""
    return tuple(s + 1000 * rank for s in SEEDS)


def make_inputs(rank=0, with_codewords=False):
    from paper_2202_13951_gb300 import workloads
    code = getattr(workloads, CODE_FN)()
    ls, cs = [], []
    for i, (e, s) in enumerate(zip(POINTS, rank_seeds(rank))):
        zero = WORKLOAD_NAME == "rlc64" and i == 0  # config 1: all-zero information half
        l, c = workloads.awgn_llr(code, B_PER_POINT, e, s, zero_info=zero)
        ls.append(l)
        cs.append(c)
    llr = np.ascontiguousarray(np.concatenate(ls))
    if with_codewords:
        return code, llr, np.concatenate(cs)
    return code, llr


def max_over_ranks(value, world, device=None):
    """Max of a float over ranks (identity when world == 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def position_weights(n, line=None, model=None):
    """rho_j for the sorted positions j = 1..n: j for basic ORBGRAND, J0 + beta j
    for a line, J_{i-1} + beta_i (j - I_{i-1}) on segment i of a model
    (Eq. relest_seg)."""
    if model is not None:
        anchors, J, beta = model
        I = [0] + list(anchors) + [n]
        return [J[i] + beta[i] * (j - I[i]) for i in range(len(J))
                for j in range(I[i] + 1, I[i + 1] + 1)]
    J0, beta = line if line else (0, 1)
    return [J0 + beta * j for j in range(1, n + 1)]


def class_weight_prefix(n, max_queries, line=None, model=None):
    """Cumulative Hamming weight over the query order, by class: the order
    visits classes (R, w) -- the w-subsets of the positions whose weights
    rho_j sum to R -- in increasing R, w ascending within it (basic
    ORBGRAND: rho_j = j, so R is the logistic weight).  Returns (class_end[],
    class_w[]) up to max_queries, so sum_{t<=q} w_t follows from q alone."""
    rho = position_weights(n, line, model)
    sat = 1 << 61
    Rmax = 64
    while True:
        # N[w][R]: w-subsets of weight R (saturating counts)
        N = np.zeros((n + 1, Rmax + 1), np.int64)
        N[0, 0] = 1
        for r in rho:
            if r <= Rmax:
                N[1:, r:] += N[:-1, :Rmax + 1 - r]
                np.minimum(N, sat, out=N)
        if N.astype(np.float64).sum() >= max_queries or Rmax >= sum(rho):
            break
        Rmax *= 2
    w_idx = np.nonzero(N.T)          # classes in R order, w ascending within R
    counts = N.T[w_idx]
    cut = int(np.searchsorted(np.cumsum(counts.astype(np.float64)), max_queries)) + 1
    ends = np.cumsum(counts[:cut])
    return ends.astype(np.int64), w_idx[1][:cut].astype(np.int64)


def sum_weights(q, class_end, class_w):
    """sum over blocks of sum_{t=1}^{q_b} w_t, from the class structure."""
    q = np.asarray(q, np.int64)
    full = np.concatenate([[0], np.cumsum((class_end - np.concatenate([[0], class_end[:-1]]))
                                          * class_w)])
    idx = np.searchsorted(class_end, q, side="left")  # class holding query q
    start = np.concatenate([[0], class_end])[idx]
    return int((full[idx] + (q - start) * class_w[idx]).sum())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)

    def summary(self, t0, t1):
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((ts, parts))
        inside = [p for ts, p in rows if t0 <= ts <= t1]
        window = "timed"
        if not inside:
            inside = [p for _, p in rows]
            window = "whole run (timed region shorter than the sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"],
                    "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        mx = [num(p[2]) for p in inside if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for p in inside:
            for i, nm in enumerate(names):
                if p[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def run_child(argv, steps=20, warmup=3, timeout_s=300):
    """bench.py in its own process with argv (device-timed only: no e2e, no
    CPU baseline, no secondary runs); its JSON line, or {"error": ...}."""
    cmd = [sys.executable, os.path.abspath(__file__), *argv, "--steps", str(steps),
           "--warmup", str(warmup), "--no-cpu-baseline", "--no-e2e", "--no-extra"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
        last = [x for x in r.stdout.splitlines() if x.startswith("{")]
        if r.returncode != 0 or not last:
            return {"error": ("exit %d: %s" % (r.returncode,
                                               (r.stderr.strip().splitlines() or [""])[-1]))[:300]}
        return json.loads(last[-1])
    except subprocess.TimeoutExpired:
        return {"error": "timed out after %d s" % timeout_s}
    except Exception as exc:  # never lose the headline line to a secondary run
        return {"error": ("%s: %s" % (type(exc).__name__, exc))[:300]}


def summarise_child(d):
    rec = {k: d.get(k) for k in ("value", "unit", "ms_per_step", "steps", "queries_per_s",
                                 "mean_queries", "abandon_rate", "bler", "gpu_launches")}
    rec["workload"] = d["config"]["workload"]
    rec["form"] = d["config"].get("form")
    rec["tuning_source"] = d["config"].get("tuning_source")
    rec["timed"] = d["config"].get("timed")
    rec["roofline"] = {k: d["roofline"].get(k)
                       for k in ("bound", "achieved", "peak", "unit", "frac", "issued_frac",
                                 "traffic")}
    rec["clocks"] = d.get("clocks")
    if "per_point" in d:
        rec["per_point"] = d["per_point"]
    if "parity" in d:
        rec["parity"] = {k: d["parity"].get(k) for k in ("checked", "blocks", "mismatches",
                                                          "abandoned_checked")}
    return rec


def run_forms():
    """The plain single launch against the batched form on the same inputs:
    the BCH(127,113) workload (4 x 100,000 blocks at 4-7 dB, cap 1e6),
    each form in its own process, each with its own parity check (the whole
    workload against the oracle).  Identical outputs give identical BLER."""
    out = {}
    every = ["--parity-per-code", "400000"]
    for name, argv in (("batched", ["--workload", "bch"] + every),
                       ("plain", ["--workload", "bch", "--form", "plain"] + every)):
        d = run_child(argv)
        out[name] = d if "error" in d else summarise_child(d)
    b, p = out["batched"], out["plain"]
    if "error" not in b and "error" not in p:
        out["same_bler"] = b["bler"] == p["bler"]
        out["batched_over_plain"] = b["value"] / p["value"]
    return out


def run_serving(seconds, timeout_s=420):
    """The serving measurement (paper_2202_13951_gb300.serve --measure) in
    its own process: capacity, half capacity and 2e6 blocks/s offered."""
    cmd = [sys.executable, "-m", "paper_2202_13951_gb300.serve", "--measure", "--seconds",
           str(seconds)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
        last = [x for x in r.stdout.splitlines() if x.startswith("{")]
        if r.returncode != 0 or not last:
            return {"error": ("exit %d: %s" % (r.returncode,
                                               (r.stderr.strip().splitlines() or [""])[-1]))[:300]}
        return json.loads(last[-1])
    except subprocess.TimeoutExpired:
        return {"error": "timed out after %d s" % timeout_s}
    except Exception as exc:
        return {"error": ("%s: %s" % (type(exc).__name__, exc))[:300]}


def extra_runs():
    """(label, argv) of the secondary measurements."""
    return [("bch, one-line full ORBGRAND J0=%d beta=%d" % EXTRA_LINE,
             ["--workload", "bch", "--line", "%d,%d" % EXTRA_LINE]),
            ("bch, 3-segment full ORBGRAND %s" % describe_model(EXTRA_MODEL),
             ["--workload", "bch", "--model",
              ";".join(",".join(str(x) for x in f) for f in EXTRA_MODEL)]),
            ("bch, one-line full ORBGRAND with a line fitted per block",
             ["--workload", "bch", "--fitted"]),
            ("bch, full ORBGRAND with a 3-line model fitted per block",
             ["--workload", "bch", "--fitted-lines", "3"]),
            ("paper256, basic ORBGRAND", ["--workload", "paper256"]),
            ("ca-polar[256,234] at 5-5.3 dB (BLER about 1e-3), full ORBGRAND with a 3-line "
             "model fitted per block (the paper's operating point, Sec. IV-B)",
             ["--workload", "capolar256", "--fitted-lines", "3"])]


def run_extra(steps=20, warmup=3, timeout_s=300, budget_s=420):
    """Secondary measurements, each in its own process after the headline
    one (same box): full ORBGRAND orders on the BCH workload and the
    paper-shaped [256,234] workload.  Device-timed values only (no e2e, no
    CPU baseline), each with its own parity check; a failure records its
    message instead of a number; runs that would start after budget_s
    seconds are skipped, so the whole bench stays within minutes."""
    out = []
    t0 = time.time()
    for label, argv in extra_runs():
        rec = {"label": label, "args": " ".join(argv)}
        if time.time() - t0 > budget_s:
            rec["error"] = "skipped: the secondary runs' %d s budget was spent" % budget_s
            out.append(rec)
            continue
        d = run_child(argv, steps, warmup, timeout_s)
        rec.update(d if "error" in d else summarise_child(d))
        out.append(rec)
    return out


# ------------------------------------------------------------- CPU side

def _oracle_decode(H, llr, cap, line, model, fitted):
    """The oracle's decoding of llr [B][n] in the bench's order: basic, a
    line, a model, or a model fitted per block (fitted = lines, or (lines,
    divisible))."""
    import oracle
    if fitted:
        lines, div = fitted if isinstance(fitted, tuple) else (int(fitted), False)
        return oracle.decode_batch_fit(H, llr, cap, lines, div)
    if model:
        return oracle.decode_batch_mline(H, llr, cap, model)
    if line:
        return oracle.decode_batch_1line(H, llr, cap, *line)
    return oracle.decode_batch(H, llr, cap)


def _oracle_worker(args):
    H, llr, cap, line, model, fitted = args[:6]
    t = time.perf_counter()
    cw, q, ab, _ = _oracle_decode(H, llr, cap, line, model, fitted)
    return time.perf_counter() - t, int(q.sum()), llr.shape[0]


def _oracle_outputs(args):
    """(block indices, oracle outputs) of one chunk, for the parity check."""
    idx, H, llr, cap, line, model, fitted = args
    cw, q, ab, sw = _oracle_decode(H, llr, cap, line, model, fitted)
    return idx, cw, q, ab, sw


def cpu_sample(llr, per_point, step):
    """Bounded sample: `per_point` blocks of each Eb/N0 point, the step-th
    slice of each point's blocks (so steps see different blocks)."""
    idx = []
    for p in range(len(POINTS)):
        base = p * B_PER_POINT
        lo = (step * per_point) % max(1, B_PER_POINT - per_point + 1)
        idx.append(np.arange(base + lo, base + lo + per_point))
    return llr[np.concatenate(idx)]


def run_oracle(H, llr, cap, procs):
    """Decode llr on `procs` spawned single-threaded oracle processes."""
    if procs <= 1:
        return _oracle_worker((H, llr, cap, LINE, MODEL, FITTED))
    import multiprocessing as mp
    chunks = np.array_split(llr, procs)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(H, c, cap, LINE, MODEL, FITTED) for c in chunks])
    return max(r[0] for r in res), sum(r[1] for r in res), sum(r[2] for r in res)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return "unknown"


def bench_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on the host cores, on
    bounded samples of the same workload."""
    if rank != 0:
        return None
    import oracle
    oracle.build_oracle()
    cores = os.cpu_count() or 1
    if WORKLOAD_NAME in MIXED:
        from paper_2202_13951_gb300 import workloads
        gen, mult = MIXED[WORKLOAD_NAME]
        B = mult * B_PER_POINT
        codes, cid, llr_flat, off, _, _ = getattr(workloads, gen)(B=B, seed=SEEDS[0])
        per_point = args.ref_sample

        def step_work(step):
            """ref_sample blocks in a stride walk, grouped by code, split over
            the cores."""
            idx = (np.arange(step * per_point, (step + 1) * per_point) * 9973) % B
            work = []
            for j, code in enumerate(codes):
                sel = idx[cid[idx] == j]
                if sel.size:
                    blk = np.stack([llr_flat[off[b]:off[b] + code.n] for b in sel])
                    work += [(code.H, c, CAP, LINE, MODEL, FITTED)
                             for c in np.array_split(blk, max(1, cores // len(codes)))
                             if c.shape[0]]
            return work, idx.size
    else:
        code, llr = make_inputs(0)
        per_point = max(1, args.ref_sample // len(POINTS))

        def step_work(step):
            sample = cpu_sample(llr, per_point, step)
            return ([(code.H, c, CAP, LINE, MODEL, FITTED)
                     for c in np.array_split(sample, cores)], sample.shape[0])
    # the pool is started once, before any timing
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores)
    times, blocks, queries = [], 0, 0
    try:
        for s in range(args.warmup + args.steps):
            work, nblk = step_work(s)
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, work)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
                blocks += nblk
                queries += sum(r[1] for r in res)
    finally:
        pool.close()
        pool.join()
    total = sum(times)
    value = blocks / total
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-llr/u32-syndrome",
        "data": "synthetic BPSK/AWGN, seeded",
        "config": {"workload": WORKLOAD, "sample_blocks_per_step": nblk,
                   "l2": "n/a (CPU)"},
        "queries_per_s": queries / total,
        "cpu_baseline": {"value": value, "unit": "blocks/s", "cores": cores,
                         "kind": "oracle",
                         "sample": "%d blocks per step (%s), %d timed steps, "
                                   "%d single-threaded oracle processes (%s)"
                                   % (nblk, ("a stride walk over the mixed batch"
                                             if WORKLOAD_NAME in MIXED else
                                             "%d per Eb/N0 point" % per_point),
                                      args.steps, cores, cpu_model())},
        "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    return line


# ------------------------------------------------------------- GPU side

class Job:
    """One workload on the device: codes, inputs, outputs and the step."""

    def __init__(self, orbg, dev, rank, args):
        import torch
        from paper_2202_13951_gb300 import workloads
        self.orbg = orbg
        self.form = args.form
        if WORKLOAD_NAME in MIXED:
            gen, mult = MIXED[WORKLOAD_NAME]
            B = mult * B_PER_POINT
            codes, cid, llr, off, cwt, _ = getattr(workloads, gen)(B=B,
                                                                   seed=SEEDS[0] + 1000 * rank)
            self.codes = codes
            self.cid_np, self.off_np, self.llr_np = cid, off, llr
            self.sent = cwt
        else:
            code, llr, cwt = make_inputs(rank, with_codewords=True)
            self.codes = [code]
            B = llr.shape[0]
            self.cid_np = np.zeros(B, np.int32)
            self.off_np = None
            self.llr_np = llr
            self.sent = cwt.reshape(-1)
        if self.form == "plain" and len(self.codes) != 1:
            raise SystemExit("--form plain needs a single-code workload")
        self.B = B
        self.n_of_block = np.array([c.n for c in self.codes], np.int64)[self.cid_np]
        if MODEL is not None and any(MODEL[0] and MODEL[0][-1] >= c.n for c in self.codes):
            raise SystemExit("--model: every anchor must lie below each code's n")
        self.objs = [orbg.Code(c.H, max_query_cap=CAP, line=LINE, model=MODEL)
                     for c in self.codes]
        self.cs = orbg.CodeSet(self.objs)
        self.fitted = None
        self.search = isinstance(FITTED, tuple)
        if FITTED:
            if len(self.codes) != 1 or self.form != "batched":
                raise SystemExit("--fitted needs a single-code workload and the batched form")
            if not self.search:
                self.fitted = orbg.Fitted(self.objs[0])
            self.rec = torch.empty((B, orbg.ORBG_FIT_STRIDE), dtype=torch.int32, device=dev)
        self.llr = torch.from_numpy(self.llr_np).to(dev)
        n_total = int(self.n_of_block.sum())
        self.cw = torch.empty((n_total,), dtype=torch.uint8, device=dev)
        self.q = torch.empty((B,), dtype=torch.int32, device=dev)
        self.ab = torch.empty((B,), dtype=torch.uint8, device=dev)
        if self.off_np is not None:
            self.cid = torch.from_numpy(self.cid_np).to(dev)
            self.off = torch.from_numpy(self.off_np).to(dev)
        else:
            self.cid = self.off = None
        self.stream = torch.cuda.current_stream(dev)

    def capture(self):
        """Capture one step (its scratch allocation, counter reset and both
        launches) into a CUDA graph; later steps replay it."""
        import torch
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.call(torch.cuda.current_stream())
        self.graph = g

    def step(self):
        if getattr(self, "graph", None) is not None:
            self.graph.replay()
            return
        self.call(self.stream)

    def call(self, stream):
        if self.search:
            # no model records are asked for: a block whose hard decision is a
            # code word decodes at query 1 in any order, unfitted
            self.orbg.orbg_decode_fitted(self.objs[0].handle, self.llr, self.B, CAP, FITTED[0],
                                         FITTED[1], self.cw, self.q, self.ab, None, stream)
            return
        if self.fitted is not None:
            lib = self.orbg.load_library()
            rc = lib.orbg_fitted_decode(self.fitted.handle, self.llr.data_ptr(), self.B, CAP,
                                        self.cw.data_ptr(), self.q.data_ptr(),
                                        self.ab.data_ptr(), self.rec.data_ptr(),
                                        self.orbg._stream(stream))
            if rc != 0:
                raise self.orbg.OrbgError(rc, "orbg_fitted_decode")
            return
        if self.form == "plain":
            self.orbg.orbg_decode(self.objs[0].handle, self.llr, self.B, CAP, self.cw, self.q,
                                  self.ab, stream)
            return
        self.orbg.orbg_decode_batched(self.cs.handle, self.cid, self.off, self.llr, self.B, CAP,
                                      self.cw, self.off, self.q, self.ab, stream)

    def block_starts(self):
        """First codeword byte of each block in the output buffer."""
        return (np.concatenate([[0], np.cumsum(self.n_of_block)[:-1]])
                if self.off_np is None else self.off_np)

    def bler(self, cw=None):
        """Fraction of blocks whose decoding differs from the sent codeword."""
        got = self.cw.cpu().numpy() if cw is None else cw
        diff = got != self.sent
        return float(np.logical_or.reduceat(diff, self.block_starts()).mean())

    def per_point(self, got):
        """BLER, mean queries and abandon rate of each Eb/N0 point (single-code
        workloads: the points' blocks are consecutive)."""
        cw, q, ab = got
        n = self.codes[0].n
        wrong = (cw.reshape(-1, n) != self.sent.reshape(-1, n)).any(axis=1)
        out = []
        for i, e in enumerate(POINTS):
            sl = slice(i * B_PER_POINT, (i + 1) * B_PER_POINT)
            out.append({"ebn0_db": e, "blocks": B_PER_POINT, "bler": float(wrong[sl].mean()),
                        "block_errors": int(wrong[sl].sum()),
                        "mean_queries": float(q[sl].mean()),
                        "abandon_rate": float((ab[sl] == 1).mean())})
        return out

    def variants(self):
        """Decoder variants among the job's codes, as the library counts
        them: keys per lane from n (<= 32, 64, 128, 256) and syndrome words
        (1, 2, 3-4)."""
        kw = set()
        for c in self.codes:
            n, r = c.n, c.r
            w = (r + 31) // 32
            kw.add((1 if n <= 32 else 2 if n <= 64 else 4 if n <= 128 else 8,
                    1 if w <= 1 else 2 if w == 2 else 4))
        return len(kw)

    def launches_per_step(self):
        """Kernels of this library launched by one step: per-block codes
        (code ids) run phase 1 as one launch per decoder variant, after a
        two-kernel grouping by variant when there are several; phase 2 is
        one launch (whatever the budget: it also decodes the blocks whose
        phase-1 walk ran past the warp's own triple table)."""
        if self.form == "plain":
            return 1
        if self.search:
            return 3  # fit, one-warp search of the open blocks, CTA search of the long ones
        phase2 = 1
        if self.fitted is not None:
            return 3 + 1 + phase2  # fit, mark, map; one variant (handles of one code); phase 2
        if self.off_np is not None:
            v = self.variants()
            return (2 if v > 1 else 0) + v + phase2
        return 1 + phase2

    def kernel_names(self):
        if self.form == "plain":
            return "orbg_plain_kernel"
        if self.search:
            return "orbg_fitprep_kernel + orbg_fitsearch_kernel + orbg_fitsearch_cta_kernel"
        names = "orbg_batched_kernel + orbg_heavy_kernel"
        if self.fitted is not None:
            return "orbg_fit_kernel + line marking + " + names
        if self.off_np is not None and self.variants() > 1:
            names = ("orbg_batched_kernel (one launch per decoder variant) + orbg_heavy_kernel "
                     "+ the two code-sort kernels")
        return names

    def autotune(self):
        return self.orbg.orbg_codeset_autotune(self.cs.handle, self.cid, self.off, self.llr,
                                               self.B, CAP, self.cw, self.off, self.q, self.ab,
                                               3, self.stream)

    def alg_ops(self, qh, sample=None):
        """Algorithmic integer ops of one step: per query sum_t W32 (w_t + 1),
        per block n ceil(log2 n) sort compares.  For a model fitted per
        block (each block its own order) the per-block mean of q + sum_t w_t
        comes from the oracle on the parity check's sample (`sample`: code
        -> [blocks, sum]); None without one."""
        total = 0
        for j, code in enumerate(self.codes):
            sel = self.cid_np == j
            if not sel.any():
                continue
            w32 = (code.r + 31) // 32
            if self.search:
                if not sample or j not in sample or not sample[j][0]:
                    return None
                nb, acc = sample[j]
                total += int(round(w32 * acc / nb * int(sel.sum())))
            elif self.fitted is not None:
                # each block in its own line's order (beta = 1, J_0 per block)
                rec = self.rec.cpu().numpy()
                J0 = np.where(rec[:, 0] == 0, 0, rec[:, 8])
                for j0 in np.unique(J0):
                    ends, ws = class_weight_prefix(code.n, CAP, (int(j0), 1))
                    qj = qh[J0 == j0]
                    total += w32 * (sum_weights(qj, ends, ws) + int(qj.sum()))
            else:
                ends, ws = class_weight_prefix(code.n, CAP, LINE, MODEL)
                qj = qh[sel]
                total += w32 * (sum_weights(qj, ends, ws) + int(qj.sum()))
            total += int(sel.sum()) * code.n * math.ceil(math.log2(code.n))
        return total


def bench_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2202_13951_gb300 import build, orbg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    orbg.load_library()

    job = Job(orbg, dev, rank, args)
    B = job.B
    tuned = "default"
    if args.shape:
        f = [int(x) for x in args.shape.split(",")]
        orbg.orbg_codeset_set_tuning(job.cs.handle, orbg.OrbgTuning(*f))
        tuned = "given (--shape)"
    elif isinstance(FITTED, tuple):
        tuned = "none (one warp per block, blocks from a work queue)"
    elif FITTED:
        tuned = "default (the fitted decoder's own code set)"
    elif not args.no_autotune and args.form == "batched":
        job.autotune()  # untimed: scheduling knobs only, results do not change
        tuned = "autotuned on this workload before warm-up"

    for _ in range(max(3, args.warmup)):
        job.step()
    torch.cuda.synchronize(dev)
    graph = "direct calls (--no-graph)"
    if FITTED is True:
        graph = "direct calls (the fitted decoder reads each block's line back mid-step)"
    elif not args.no_graph:
        try:
            job.capture()
            for _ in range(3):  # warm-up replays
                job.step()
            torch.cuda.synchronize(dev)
            graph = "replays of a captured CUDA graph of one call"
        except Exception as exc:  # capture refused: time the direct calls
            job.graph = None
            torch.cuda.synchronize(dev)
            graph = "direct calls (capture failed: %s)" % str(exc).splitlines()[0][:120]

    sampler = ClockSampler(local)
    sampler.start()
    stream = job.stream
    events = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    events[0].record(stream)
    for i in range(args.steps):
        job.step()
        events[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    t_wall1 = time.time()
    if world > 1:
        dist.barrier()
    sampler.stop()
    per_step = [events[i].elapsed_time(events[i + 1]) for i in range(args.steps)]
    local_ms = events[0].elapsed_time(events[-1])
    total_ms = max_over_ranks(local_ms, world, dev)
    blocks_total = sum_over_ranks(float(B * args.steps), world, dev)
    value = blocks_total / (total_ms / 1000.0)

    # work done per step, from one more (untimed) step whose output buffers
    # were first filled with values no decode writes: a block the step left
    # unwritten cannot pass parity on an earlier step's results
    poison_outputs(job)
    job.step()
    torch.cuda.synchronize(dev)
    got = gpu_outputs(job)
    qh, abh = got[1], got[2]
    q_step = int(qh.sum())
    queries_total = sum_over_ranks(float(q_step * args.steps), world, dev)
    alg_ops = None if job.search else job.alg_ops(qh)  # per-block models: after parity
    kernel_ms = statistics.mean(per_step)
    achieved = alg_ops / (kernel_ms / 1000.0) / 1e12 if alg_ops is not None else None  # Tops/s

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    clocks = sampler.summary(t_wall0, t_wall1)
    max_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    run_mhz = (clocks.get("sm_mhz") if clocks.get("window") == "timed" and clocks.get("sm_mhz")
               else max_mhz)
    lanes = measured_int_lanes(orbg)
    peak = lanes * sms * run_mhz * 1e6 / 1e12 if lanes else None
    smem_bpc = measured_smem_bytes(orbg)
    prof = stored_profile(build, job_profile_key(args))

    # end to end: host (pinned) buffers through the same C call
    e2e = None
    if not args.no_e2e and not FITTED:
        e2e = bench_e2e(orbg, job, args, world, dev)

    line = {
        "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-llr/u32-syndrome",
        "data": "synthetic BPSK/AWGN, seeded (numpy PCG64); each rank its own seeds",
        "config": {"workload": WORKLOAD, "blocks_per_step": B, "query_cap": CAP,
                   "input_mb": round(job.llr_np.nbytes / 1e6, 1),
                   "form": ("plain single launch (orbg_decode)" if args.form == "plain" else
                            "batched persistent launch (orbg_decode_batched)"),
                   "l2": ("inputs %.0f MB %s 129 MB L2, no flush"
                          % (job.llr_np.nbytes / 1e6,
                             ">" if job.llr_np.nbytes > 129e6 else "<=")),
                   "tuning": orbg.orbg_codeset_get_tuning(job.cs.handle).as_dict(),
                   "tuning_source": tuned, "timed": graph,
                   "order": ("full ORBGRAND, a %d-line model fitted per block (Sec. III-E)"
                             % (FITTED[0] if isinstance(FITTED, tuple) else 1)
                             if FITTED else
                             ("%d-segment full ORBGRAND, %s"
                              % (len(MODEL[1]), describe_model(MODEL))) if MODEL
                             else ("one-line full ORBGRAND, J0=%d beta=%d" % LINE) if LINE
                             else "basic ORBGRAND"),
                   "parallelism": "replicas x%d (blocks sharded by rank, no collective)" % world},
        "queries_per_s": queries_total / (total_ms / 1000.0),
        "latency_ms": {"step_p50": statistics.median(per_step),
                       "step_p99": float(np.percentile(per_step, 99)),
                       "what": "one %d-block batch, launch to completion (request latency "
                               "under load: see serving)" % B},
        "abandon_rate": float(abh.mean()),
        "mean_queries": float(qh.mean()),
        "bler": job.bler(got[0]),
        "gpu_launches": job.launches_per_step() * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s",
                     "frac": (achieved / peak) if peak and achieved is not None else None,
                     "traffic": prof.get("traffic_bytes_per_step") if prof else None,
                     "issued_frac": prof.get("issued_frac") if prof else None,
                     "what": ("the step's decode kernels together (%s), timed by CUDA events "
                              "around each step on the launching stream; algorithmic 32-bit "
                              "integer ops per step = sum_t W32 (w_t + 1) + B n ceil(log2 n) "
                              "= %s, which charges each column XOR as one op although one "
                              "3-input lop3 can retire two, and charges every query in full "
                              "although the triple-range walk tests sixteen queries with "
                              "about thirty instructions (so frac can exceed 1 on "
                              "search-heavy work); peak = measured lop3 lanes/clk/SM (%s) x "
                              "%d SMs x %.0f MHz (the median SM clock sampled during the "
                              "timed steps); issued_frac = the ALU pipe's issue utilisation "
                              "(ncu, time-weighted over the step's kernels, same source "
                              "digest); traffic = their DRAM bytes per step (ncu, same "
                              "digest; null when the kernels changed since the capture)"
                              % (job.kernel_names(), alg_ops, lanes, sms, run_mhz)),
                     "profile": prof.get("source") if prof else None},
        "clocks": clocks,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
        "smem_peak": {"bytes_per_clk_per_sm": smem_bpc,
                      "tb_s": (smem_bpc * sms * run_mhz * 1e6 / 1e12) if smem_bpc else None,
                      "what": "measured 64-bit conflict-free shared loads (the search's "
                              "column and triple-table reads are shared loads)"},
    }
    if e2e:
        line["e2e"] = e2e
    if job.off_np is None and len(POINTS) > 1:
        line["per_point"] = job.per_point(got)
    have = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], have = cpu_baseline(job)
    if not args.no_parity:
        line["parity"] = parity_check(job, got, have, budget_s=args.parity_budget,
                                      per_code=args.parity_per_code)
        sample = line["parity"].pop("_alg")
        if job.search:
            # each block in its own order: the work per block is the oracle's
            # own count on the checked sample, scaled to the step
            alg_ops = job.alg_ops(qh, sample)
            if alg_ops is not None:
                rf = line["roofline"]
                rf["achieved"] = alg_ops / (kernel_ms / 1000.0) / 1e12
                rf["frac"] = rf["achieved"] / peak if peak else None
                rf["what"] = rf["what"].replace(
                    "= None,", "= %d (estimated: the oracle's q + sum_t w_t per block on the "
                               "%d checked blocks, times the blocks of the step)," %
                    (alg_ops, line["parity"]["checked"]))
    default = (rank == 0 and world == 1 and not args.no_extra and WORKLOAD_NAME == "mixed" and
               LINE is None and MODEL is None and not FITTED and args.form == "batched")
    if default:
        line["forms"] = run_forms()
        if not args.no_serving:
            line["serving"] = run_serving(args.serving_seconds)
        try:
            line["extra_workloads"] = run_extra()
        except Exception as exc:
            line["extra_workloads"] = [{"error": ("%s: %s" % (type(exc).__name__, exc))[:300]}]
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


# DRAM traffic and ALU issue utilisation of a step's kernels, from one ncu
# capture each (`profiles/` holds the summaries and commands); keyed by
# workload/form/order and valid only while the device code of the kernels
# they cover is the code they were taken on (its digest: PROFILE_SOURCES).
# Traffic is per step, scaled from the captured size by the blocks decoded
# when the capture was smaller.
PROFILES = {
    "mixed/batched/basic": {
        "kernels": "batched",
        "digest": "2c12445a5d48257a47c952b322d3bff627fe866c08f362acfe76301aa124f4ac",
        # the step's kernels' DRAM bytes on 250,000 blocks (222.4 MB), x 4
        # ALU pipe issue share per kernel, weighted by the full-size step's
        # time shares (phase 2 62.6 % x 0.542, phase 1 n = 256 42.7 % x 0.367,
        # n = 128 36.5 % x 0.056, n = 64 32.9 % x 0.033)
        "traffic_bytes_per_step": 889.6e6,
        "issued_frac": 0.527,
        "source": "profiles/orbg_batched_mixed_250k_full.md, "
                  "profiles/orbg_batched_mixed_1m_launches.md",
    },
    "bch/batched/fitted3": {
        "kernels": "fitsearch",
        "digest": "de5fe7c9402f8746661f22207cfd249604b74f2bced388ba6bcd2e522d9358f9",
        # 346.4 MB on 280,000 blocks, x 400,000 / 280,000
        "traffic_bytes_per_step": 494.9e6,
        "issued_frac": 0.317,
        "source": "profiles/orbg_fitsearch_bch127_3line_280k_full.md",
    },
    "bch/batched/basic": {
        "kernels": "batched",
        "digest": "2c12445a5d48257a47c952b322d3bff627fe866c08f362acfe76301aa124f4ac",
        # 166.8 MB on the captured case, x 1.4286
        "traffic_bytes_per_step": 238.3e6,
        "issued_frac": 0.554,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
    "bch/plain/basic": {
        "kernels": "plain",
        "digest": "c529c1ef75f6f3ff68d8e84ae7a9ed48dd5b78b9e935a6f10120dd8354ec41b8",
        # 165.0 MB on the captured case, x 1.4286
        "traffic_bytes_per_step": 235.7e6,
        "issued_frac": 0.344,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
    "bch/batched/line": {
        "kernels": "batched",
        "digest": "2c12445a5d48257a47c952b322d3bff627fe866c08f362acfe76301aa124f4ac",
        # 169.1 MB on the captured case, x 1.4286
        "traffic_bytes_per_step": 241.6e6,
        "issued_frac": 0.557,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
    "bch/batched/model": {
        "kernels": "batched",
        "digest": "2c12445a5d48257a47c952b322d3bff627fe866c08f362acfe76301aa124f4ac",
        # 166.4 MB on the captured case, x 1.4286
        "traffic_bytes_per_step": 237.7e6,
        "issued_frac": 0.614,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
    "bch/batched/fitted1": {
        "kernels": "fitline",
        "digest": "97ba7642ce2a3a88e76f54600d1b4350c6c75f61b0d9d555182f9b108aa4bd8b",
        # 399.9 MB on the captured case, x 1.4286
        "traffic_bytes_per_step": 571.3e6,
        "issued_frac": 0.414,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
    "paper256/batched/basic": {
        "kernels": "batched",
        "digest": "2c12445a5d48257a47c952b322d3bff627fe866c08f362acfe76301aa124f4ac",
        # 207.0 MB on the captured case, x 2.8571
        "traffic_bytes_per_step": 591.4e6,
        "issued_frac": 0.598,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
    "capolar256/batched/fitted3": {
        "kernels": "fitsearch",
        "digest": "de5fe7c9402f8746661f22207cfd249604b74f2bced388ba6bcd2e522d9358f9",
        # 363.9 MB on the captured case, x 2.8571
        "traffic_bytes_per_step": 1039.7e6,
        "issued_frac": 0.305,
        "source": "profiles/bench_workloads_traffic_alu.md",
    },
}


def job_profile_key(args):
    order = ("fitted%d" % (FITTED[0] if isinstance(FITTED, tuple) else 1) if FITTED else
             "model" if MODEL else "line" if LINE else "basic")
    return "%s/%s/%s" % (WORKLOAD_NAME, args.form, order)


# the device-code files each kernel family is built from (a stored profile
# is valid while their digest is unchanged)
PROFILE_SOURCES = {
    "batched": ["orbg_batched.cuh", "orbg_heavy.cuh", "orbg_decode_block.cuh", "orbg_batched.cu",
                "orbg_batched_inst.cu", "orbg_internal.h"],
    "plain": ["orbg_plain.cu", "orbg_decode_block.cuh", "orbg_internal.h"],
    "fitline": ["orbg_batched.cuh", "orbg_heavy.cuh", "orbg_decode_block.cuh", "orbg_batched.cu",
                "orbg_batched_inst.cu", "orbg_internal.h", "orbg_fit.cu", "orbg_fit.cuh"],
    "fitsearch": ["orbg_fitted_search.cuh", "orbg_fitted_search_inst.cu", "orbg_fit.cuh",
                  "orbg_decode_block.cuh", "orbg_internal.h"],
}


def stored_profile(build, key):
    """The stored ncu figures for key, if they were taken on these sources."""
    rec = PROFILES.get(key)
    if not rec:
        return None
    try:
        if rec.get("digest") != build.kernel_digest(PROFILE_SOURCES[rec["kernels"]]):
            return None
    except Exception:
        return None
    return rec


def measured_int_lanes(orbg):
    """LOP3 lanes per clock per SM, from the library's probe kernel."""
    try:
        return orbg.orbg_probe_int_lanes()
    except Exception:
        return None


def measured_smem_bytes(orbg):
    """Shared-memory bytes per clock per SM, from the library's probe kernel."""
    try:
        return orbg.orbg_probe_smem_bytes()
    except Exception:
        return None


def bench_e2e(orbg, job, args, world, dev):
    """The same call with the inputs and outputs in pinned host memory: the
    library stages them (H2D, both kernels, D2H, stream sync), all timed."""
    import torch
    B = job.B
    pin_llr = torch.empty(job.llr_np.shape, dtype=torch.float32, pin_memory=True)
    pin_llr.numpy()[...] = job.llr_np
    n_total = int(job.n_of_block.sum())
    h_cw = torch.empty((n_total,), dtype=torch.uint8, pin_memory=True)
    h_q = torch.empty((B,), dtype=torch.int32, pin_memory=True)
    h_ab = torch.empty((B,), dtype=torch.uint8, pin_memory=True)
    cid = off = None
    in_meta = 0
    if job.off_np is not None:
        cid = torch.from_numpy(job.cid_np).pin_memory()
        off = torch.from_numpy(job.off_np).pin_memory()
        in_meta = B * (4 + 8 + 8)

    def step():
        if job.form == "plain":
            orbg.orbg_decode(job.objs[0].handle, pin_llr, B, CAP, h_cw, h_q, h_ab, job.stream)
        else:
            orbg.orbg_decode_batched(job.cs.handle, cid, off, pin_llr, B, CAP, h_cw, off, h_q,
                                     h_ab, job.stream)

    for _ in range(3):
        step()
    steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize(dev)
    per = []
    import gc
    gc.disable()  # no collector pause inside a timed call
    try:
        t0 = time.perf_counter()
        for _ in range(steps):
            ts = time.perf_counter()
            step()  # host-buffer calls synchronise before returning
            per.append((time.perf_counter() - ts) * 1e3)
        dt = time.perf_counter() - t0
    finally:
        gc.enable()
    dt = max_over_ranks(dt, world, dev)
    blocks = sum_over_ranks(float(B * steps), world, dev)
    return {"value": blocks / dt, "unit": "blocks/s",
            "h2d_bytes_per_step": int(job.llr_np.nbytes + in_meta),
            "d2h_bytes_per_step": int(n_total + B * 4 + B),
            "steps": steps,
            "step_ms": {"p50": statistics.median(per), "min": min(per), "max": max(per)},
            "what": ("the same call on pinned host buffers: H2D, kernels, D2H, sync; value = "
                     "all steps' blocks / their total wall time (a step whose host-device "
                     "copies ran slow counts in full: see step_ms)")}


def block_rows(job, idx, code_j):
    """LLR rows [len(idx)][n] of blocks idx (all of code code_j)."""
    n = job.codes[code_j].n
    if job.off_np is None:
        return job.llr_np[idx]
    return np.stack([job.llr_np[job.off_np[b]:job.off_np[b] + n] for b in idx])


def stratified_order(idx, stride=97):
    """idx in a stratified order: every stride-th entry, then the next
    residue, and so on (any prefix samples the whole range evenly)."""
    return np.concatenate([idx[r::stride] for r in range(min(stride, max(1, idx.size)))])


def cpu_baseline(job, budget_s=15.0):
    """The oracle as it stands, one process, on a bounded sample of the same
    workload: blocks taken in a stratified order (every stride-th block,
    then the next residue, ...) in chunks, until about budget_s seconds of
    CPU work; the whole workload if it finishes sooner.  Also returns the
    oracle's outputs of those blocks ({block: (codeword, q, abandon, sum of
    the queries' Hamming weights)}), which the parity check reuses."""
    import oracle
    oracle.build_oracle()
    B = job.B
    order = stratified_order(np.arange(B))
    t_total = 0.0
    nb = 0
    qsum = 0
    chunk = 1000
    outputs = {}
    for c0 in range(0, B, chunk):
        idx = order[c0:c0 + chunk]
        for j in np.unique(job.cid_np[idx]):
            sel = idx[job.cid_np[idx] == j]
            llr = block_rows(job, sel, j)
            t = time.perf_counter()
            cw, q, ab, sw = _oracle_decode(job.codes[j].H, llr, CAP, LINE, MODEL, FITTED)
            t_total += time.perf_counter() - t
            qsum += int(q.sum())
            nb += sel.size
            for k, b in enumerate(sel):
                outputs[int(b)] = (cw[k], int(q[k]), int(ab[k]), int(sw[k]))
        if t_total > budget_s:
            break
    what = ("the whole %d-block workload" % nb if nb == B else
            "%d of the %d blocks (stratified: every 97-th block, residues in turn; ~%.0f s)"
            % (nb, B, budget_s))
    return ({"value": nb / t_total, "unit": "blocks/s", "cores": 1, "kind": "oracle",
             "queries_per_s": qsum / t_total,
             "sample": "%s, one single-threaded process on %s" % (what, cpu_model())},
            outputs)


def poison_outputs(job):
    """Fill the step's output buffers with values no decode writes
    (codeword bytes 255, q 2^32 - 1, abandon flag 255)."""
    job.cw.fill_(0xFF)
    job.q.fill_(-1)
    job.ab.fill_(0xFF)


def gpu_outputs(job):
    """The timed step's outputs on the host: codeword bytes, q, abandon."""
    return (job.cw.cpu().numpy(), job.q.cpu().numpy().astype(np.int64),
            job.ab.cpu().numpy())


def parity_check(job, got, have=None, budget_s=60.0, per_code=20000):
    """The GPU outputs of the timed step against the oracle, block by block
    (codeword, query count, abandon flag; tolerance 0), outside the timed
    region.  Blocks the CPU baseline already decoded (`have`) are compared
    directly; then, per code, blocks in a stratified order are decoded by the
    oracle on all host cores (spawned single-threaded processes) until every
    code has `per_code` blocks checked (or all of its blocks), or until
    budget_s seconds have passed.  Blocks the GPU abandoned are put first in
    each code's order, up to 500 per code checked in all (even when the CPU
    baseline's sample already reaches per_code), so the longest searches are
    among those checked.  Also returns, under "_alg", per code the blocks
    checked and the sum over them of q + sum_t w_t (the oracle's own count
    of the queries' Hamming weights), from which the algorithmic work of
    orders with a model per block is estimated."""
    import multiprocessing as mp
    import oracle
    oracle.build_oracle()
    cw_g, q_g, ab_g = got
    starts = job.block_starts()
    have = have or {}
    checked = {}
    mism = []
    ncodes = len(job.codes)
    done = np.zeros(job.B, bool)

    alg = {}

    def compare(b, cw, q, ab, sw):
        n = int(job.n_of_block[b])
        ok = (q == q_g[b] and ab == ab_g[b] and
              np.array_equal(np.asarray(cw, np.uint8), cw_g[starts[b]:starts[b] + n]))
        j = int(job.cid_np[b])
        checked[j] = checked.get(j, 0) + 1
        a = alg.setdefault(j, [0, 0])
        a[0] += 1
        a[1] += int(sw) + int(q)
        done[b] = True
        if not ok:
            mism.append(int(b))

    for b, (cw, q, ab, sw) in have.items():
        compare(b, cw, q, ab, sw)
    t0 = time.time()
    todo = []
    for j in range(ncodes):
        idx = np.nonzero((job.cid_np == j) & ~done)[0]
        # the GPU-abandoned blocks first (up to 500 per code checked in all,
        # whatever the CPU baseline's sample already covered), then the
        # stratified rest up to per_code
        seen = int((done & (ab_g == 1) & (job.cid_np == j)).sum())
        aband = idx[ab_g[idx] == 1][:max(0, 500 - seen)]
        rest = stratified_order(idx[ab_g[idx] != 1])
        want = max(0, min(per_code - checked.get(j, 0) - aband.size, rest.size))
        todo.append((j, np.concatenate([aband, rest[:want]])))
    chunk = 256
    tasks = []
    for j, idx in todo:
        for c in range(0, idx.size, chunk):
            sel = idx[c:c + chunk]
            tasks.append((c, j, sel))
    tasks.sort(key=lambda t: t[0])   # codes interleaved, abandoned blocks first
    cores = os.cpu_count() or 1
    timed_out = False
    if tasks:
        ctx = mp.get_context("spawn")
        pool = ctx.Pool(cores)
        try:
            gen = ((sel, job.codes[j].H, block_rows(job, sel, j), CAP, LINE, MODEL, FITTED)
                   for _, j, sel in tasks)
            for sel, cw, q, ab, sw in pool.imap_unordered(_oracle_outputs, gen):
                for k, b in enumerate(sel):
                    compare(int(b), cw[k], int(q[k]), int(ab[k]), int(sw[k]))
                if time.time() - t0 > budget_s:
                    timed_out = True
                    break
        finally:
            pool.terminate()
            pool.join()
    n_checked = int(done.sum())
    return {"checked": n_checked, "blocks": job.B, "mismatches": len(mism),
            "mismatch_blocks": mism[:10],
            "abandoned_checked": int((done & (ab_g == 1)).sum()),
            "per_code": {str(j): checked.get(j, 0) for j in range(ncodes)},
            "what": ("the timed step's codeword, query count and abandon flag of every "
                     "checked block equal the oracle's (tolerance 0); blocks: %s"
                     % ("all" if n_checked == job.B else
                        "the CPU baseline's sample plus, per code, the GPU-abandoned blocks "
                        "(up to 500) and a stratified sample, up to %d per code%s"
                        % (per_code, ", cut by the %.0f s budget" % budget_s
                           if timed_out else ""))),
            "cores": cores, "wall_s": round(time.time() - t0, 1), "_alg": alg}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if args.impl == "reference":
        line = bench_reference(args, rank, world)
    else:
        line = bench_ours(args, rank, world, local)
    if line is not None and rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
