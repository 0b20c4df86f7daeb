"""bench.py's multi-GPU host logic on CPU with gloo, world size 2: every rank
decodes its own seeded workload (replicas, no data-path collective) and the
timing / work totals are reduced over ranks (max / sum)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.select_workload("bch", 50)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    code, llr = bench.make_inputs(rank)
    t = bench.max_over_ranks(1.0 + rank, world)
    s = bench.sum_over_ranks(float(llr.shape[0]), world)
    out[rank] = (t, s, float(llr[0, 0]), bench.rank_seeds(rank)[0])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reductions_and_sharding():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (t0, s0, x0, seed0), (t1, s1, x1, seed1) = out[0], out[1]
    assert t0 == t1 == 2.0            # max over ranks
    assert s0 == s1 == 2 * 4 * 50     # total blocks of both replicas
    assert seed0 != seed1 and x0 != x1  # each rank its own seeded data


def test_class_weight_prefix_matches_oracle():
    import bench
    import oracle
    from paper_2202_13951_gb300 import workloads
    code = workloads.rlc(64, 48, 5)
    llr, _ = workloads.awgn_llr(code, 200, 3.0, 6)
    _, q, _, sw = oracle.decode_batch(code.H, llr, 10 ** 5)
    ends, ws = bench.class_weight_prefix(code.n, 10 ** 5)
    assert bench.sum_weights(q, ends, ws) == int(sw.sum())



@pytest.mark.parametrize("line", [(3, 1), (5, 2), (20, 1)])
def test_class_weight_prefix_one_line_matches_oracle(line):
    """The bench's per-query Hamming-weight sums in the one-line order
    (Sec. III-D) equal the one-line oracle's own count."""
    import bench
    import oracle
    from paper_2202_13951_gb300 import workloads
    code = workloads.rlc(64, 48, 5)
    llr, _ = workloads.awgn_llr(code, 150, 3.0, 7)
    _, q, _, sw = oracle.decode_batch_1line(code.H, llr, 10 ** 5, *line)
    ends, ws = bench.class_weight_prefix(code.n, 10 ** 5, line)
    assert bench.sum_weights(q, ends, ws) == int(sw.sum())


def test_class_weight_prefix_m_segment_matches_oracle():
    """The same for m-segment orders (Sec. III-D, Eq. relest_seg): a model
    with a zero-weight position and models fitted (Sec. III-E) to blocks."""
    import bench
    import oracle
    from paper_2202_13951_gb300 import workloads
    code = workloads.rlc(64, 48, 5)
    llr, _ = workloads.awgn_llr(code, 150, 3.0, 8)
    for model in (((8,), (-2, 11), (2, 1)), oracle.fit(llr[0], 3), oracle.fit(llr[1], 2, True)):
        _, q, _, sw = oracle.decode_batch_mline(code.H, llr, 10 ** 5, model)
        ends, ws = bench.class_weight_prefix(code.n, 10 ** 5, model=model)
        assert bench.sum_weights(q, ends, ws) == int(sw.sum()), model


def test_extra_models_are_the_fits_of_the_mean_curve():
    """The bench's secondary full-ORBGRAND orders are the one- and
    three-line fits (Sec. III-E) of the mean ordered |LLR| curve of 10,000
    BCH(127,113) blocks at 5.5 dB (seed 7), as its comment states."""
    import bench
    import oracle
    from paper_2202_13951_gb300 import workloads
    llr, _ = workloads.awgn_llr(workloads.config2_code(), 10000, 5.5, 7)
    curve = np.sort(np.abs(llr), axis=1).mean(axis=0).astype(np.float32)
    anchors, J, beta = oracle.fit(curve, 1)
    assert anchors == () and (J[0], beta[0]) == bench.EXTRA_LINE
    assert oracle.fit(curve, 3) == bench.EXTRA_MODEL


def test_extra_runs_parse_their_arguments():
    """The secondary runs' command lines parse: the model and the line are
    taken, the paper-shaped workload is selected."""
    import bench
    try:
        a = bench.parse_args(["--model", ";".join(",".join(str(x) for x in f)
                                                  for f in bench.EXTRA_MODEL)])
        assert bench.MODEL == bench.EXTRA_MODEL and bench.LINE is None
        bench.MODEL = None
        bench.parse_args(["--line", "%d,%d" % bench.EXTRA_LINE])
        assert bench.LINE == bench.EXTRA_LINE
        bench.LINE = None
        bench.parse_args(["--workload", "paper256"])
        assert bench.CAP == 5_000_000 and "paper-shaped" in bench.WORKLOAD
        assert not a.no_extra
        bench.parse_args(["--workload", "bch", "--cap", "33"])
        assert bench.CAP == 33 and bench.WORKLOAD.endswith("query cap 33")
        bench.parse_args(["--workload", "mixed", "--cap", "1"])
        assert bench.CAP == 1 and "query cap 1, one launch, autotuned" in bench.WORKLOAD
    finally:
        bench.MODEL = None
        bench.LINE = None
        bench.parse_args([])


def test_class_weight_prefix_fitted_lines_match_oracle():
    """The bench's op count for one line fitted per block (each block's own
    J_0, beta = 1; J_0 = -1 included) equals the oracle's weight sums of its
    fit-then-decode."""
    import bench
    import oracle
    from paper_2202_13951_gb300 import workloads
    code = workloads.rlc(64, 48, 5)
    llr = np.concatenate([workloads.awgn_llr(code, 60, eb, 9 + int(eb))[0]
                          for eb in (1.0, 3.0, 6.0)])
    _, q, _, sw = oracle.decode_batch_fit(code.H, llr, 10 ** 5, 1)
    J0 = np.array([oracle.fit(x, 1)[1][0] for x in llr])
    assert (J0 == -1).any() and len(set(J0.tolist())) > 3
    total = 0
    for j0 in np.unique(J0):
        ends, ws = bench.class_weight_prefix(code.n, 10 ** 5, (int(j0), 1))
        total += bench.sum_weights(q[J0 == j0].astype(np.int64), ends, ws)
    assert total == int(sw.sum())


def test_run_extra_parses_child_lines(monkeypatch):
    """The secondary runs' results are read from each child's JSON line
    (here a stand-in line; no GPU), and a failing child records its error
    instead of raising."""
    import json
    import subprocess
    import types
    import bench
    line = {"value": 1.0e6, "unit": "blocks/s", "ms_per_step": 0.4, "steps": 20,
            "queries_per_s": 2.0e9, "mean_queries": 12.5, "abandon_rate": 0.0, "bler": 0.01,
            "gpu_launches": 40,
            "config": {"workload": "w", "tuning_source": "given (--shape)"},
            "roofline": {"bound": "alu", "achieved": 3.0, "peak": 20.1, "unit": "Tops/s",
                         "frac": 0.15, "traffic": None, "what": "x"},
            "clocks": {"sm_mhz": 2070}}
    calls = []

    def fake_run(cmd, **kw):
        calls.append(cmd)
        if "paper256" in cmd:
            return types.SimpleNamespace(returncode=1, stdout="", stderr="boom\nRuntimeError: x")
        return types.SimpleNamespace(returncode=0, stdout="log\n" + json.dumps(line) + "\n",
                                     stderr="")
    monkeypatch.setattr(subprocess, "run", fake_run)
    out = bench.run_extra()
    assert len(out) == len(calls) == len(bench.extra_runs())
    ok = [r for r in out if "error" not in r]
    assert len(ok) == len(calls) - 1 and all(r["value"] == 1.0e6 and
                                             r["roofline"]["frac"] == 0.15 and
                                             r["workload"] == "w" for r in ok)
    bad = [r for r in out if "error" in r]
    assert len(bad) == 1 and "RuntimeError" in bad[0]["error"]
    assert all("--no-extra" in c and "--no-cpu-baseline" in c for c in calls)


class _FakeJob:
    """What bench.parity_check reads of a job, for a mixed batch on the CPU."""

    def __init__(self, codes, cid, llr, off):
        self.codes, self.cid_np, self.llr_np, self.off_np = codes, cid, llr, off
        self.B = cid.shape[0]
        self.n_of_block = np.array([c.n for c in codes], np.int64)[cid]

    def block_starts(self):
        return self.off_np


def test_parity_check_counts_mismatches_on_mixed_blocks():
    """bench.parity_check compares every checked block's codeword, query
    count and abandon flag with the oracle's: outputs that are the oracle's
    own give no mismatch; a planted wrong query count, codeword bit or
    abandon flag in three blocks gives three, each named."""
    import bench
    import oracle
    from paper_2202_13951_gb300 import workloads
    codes = [workloads.rlc(32, 24, 3), workloads.rlc(48, 36, 4)]
    codes, cid, llr, off, _, _ = workloads.mixed_inputs(codes, 300, 11, 2.0, 5.0)
    job = _FakeJob(codes, cid, llr, off)
    cw = np.zeros(llr.shape[0], np.uint8)
    q = np.zeros(job.B, np.int64)
    ab = np.zeros(job.B, np.uint8)
    bench.select_workload("mixed", 100)
    for j, c in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        rows = np.stack([llr[off[b]:off[b] + c.n] for b in idx])
        wc, wq, wab, _ = oracle.decode_batch(c.H, rows, bench.CAP)
        for k, b in enumerate(idx):
            cw[off[b]:off[b] + c.n] = wc[k]
        q[idx], ab[idx] = wq, wab
    res = bench.parity_check(job, (cw, q, ab), budget_s=120, per_code=1000)
    assert res["checked"] == job.B and res["mismatches"] == 0
    q2, cw2, ab2 = q.copy(), cw.copy(), ab.copy()
    q2[5] += 1
    cw2[off[17]] ^= 1
    ab2[40] ^= 1
    res = bench.parity_check(job, (cw2, q2, ab2), budget_s=120, per_code=1000)
    assert res["mismatches"] == 3 and sorted(res["mismatch_blocks"]) == [5, 17, 40]
    res = bench.parity_check(job, (cw, q, ab), budget_s=120, per_code=50)
    assert res["checked"] == 100 and res["mismatches"] == 0
