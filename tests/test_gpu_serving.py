"""Serving loop (orbg_server): requests of mixed codes arriving while others
run are batched together on the GPU, and each request's result is the same,
block for block, as decoding it alone -- and as the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2202_13951_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orbg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_13951_gb300 import build, orbg as ob
    build.build()
    ob.load_library()
    return ob


def _alone(ob, cs, cd, llr, cap, code_index, ncodes):
    """One request by itself through orbg_decode_batched."""
    B = llr.shape[0]
    x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    cid = torch.full((B,), code_index, dtype=torch.int32, device="cuda")
    off = torch.arange(B, dtype=torch.int64, device="cuda") * cd.n
    cw, q, ab = ob.decode_batched(cs, x.reshape(-1), cap, code_id=cid, llr_offset=off,
                                  cw_offset=off, n_total=B * cd.n)
    torch.cuda.synchronize()
    return cw.cpu().numpy().reshape(B, cd.n), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()


@pytest.mark.parametrize("budget_mb,streams", [(256, 4), (3, 2)])
def test_each_request_same_alone_and_in_the_mix(orbg, budget_mb, streams):
    cap = 200000
    tr = workloads.serving_trace(rate_blocks_s=3e5, seconds=0.25, max_size=400, seed=77)
    codes = [orbg.Code(c.H, max_query_cap=cap) for c in tr["codes"]]
    cs = orbg.CodeSet(codes)
    srv = orbg.orbg_server_create(cs.handle, budget_mb << 20, cap, streams, 0)
    m = tr["arrival_s"].shape[0]
    nb = int(tr["B"].sum())
    cw = np.zeros(tr["llr_all"].shape[0], np.uint8)
    q = np.zeros(nb, np.uint32)
    ab = np.zeros(nb, np.uint8)
    lat = np.zeros(m)
    try:
        orbg.orbg_server_replay(srv, tr["arrival_s"], tr["code"], tr["B"], tr["llr_off"],
                                tr["blk_off"], tr["llr_all"], cw, q, ab, lat)
        st = orbg.orbg_server_stats_get(srv)
    finally:
        orbg.orbg_server_destroy(srv)
    assert st["completed"] == m and st["blocks_done"] == nb
    assert st["batches"] < m  # requests were batched together
    assert (lat > 0).all()
    rng = np.random.default_rng(3)
    for i in range(m):
        cd = tr["codes"][tr["code"][i]]
        B = int(tr["B"][i])
        lo, bo = int(tr["llr_off"][i]), int(tr["blk_off"][i])
        llr = tr["llr_all"][lo:lo + B * cd.n].reshape(B, cd.n)
        mixed = (cw[lo:lo + B * cd.n].reshape(B, cd.n), q[bo:bo + B].astype(np.int64),
                 ab[bo:bo + B])
        alone = _alone(orbg, cs, cd, llr, cap, int(tr["code"][i]), len(codes))
        for g, w in zip(mixed, alone):
            assert np.array_equal(g, w), "request %d differs alone vs in the mix" % i
        if i % 7 == 0:  # and against the oracle on a few blocks
            pick = rng.choice(B, size=min(4, B), replace=False)
            wc, wq, wab, _ = oracle.decode_batch(cd.H, llr[pick], cap)
            assert np.array_equal(mixed[0][pick], wc)
            assert np.array_equal(mixed[1][pick], wq.astype(np.int64))
            assert np.array_equal(mixed[2][pick], wab)


def test_overlapping_batches_and_admission(orbg):
    """Requests submitted back to back, each heavy enough (CA-Polar at 2.5 dB,
    about half its blocks run to the 1e6 cap) to keep a batch on the GPU
    for a while: several batches are in flight at once; and a request that
    can never fit the pools is refused up front."""
    cap = 10 ** 6
    codes_w = workloads.config5_codes()
    codes = [orbg.Code(c.H, max_query_cap=cap) for c in codes_w]
    cs = orbg.CodeSet(codes)
    srv = orbg.orbg_server_create(cs.handle, 64 << 20, cap, 4, 2048)
    try:
        reqs = [workloads.awgn_llr(codes_w[1], 1500, 2.5, 1000 + i)[0] for i in range(12)]
        for i, llr in enumerate(reqs):  # code 1: CA-Polar
            orbg.orbg_server_submit(srv, i, 1, llr, llr.shape[0])
        got = set()
        while len(got) < len(reqs):
            got.update(orbg.orbg_server_poll(srv, 64, 100000))
        for i in range(len(reqs)):
            orbg.orbg_server_fetch(srv, i)
        st = orbg.orbg_server_stats_get(srv)
        assert st["batches"] == len(reqs)  # max_batch_blocks 2048: one request each
        assert st["max_inflight_batches"] >= 2
        big = np.zeros((1 << 17, 128), np.float32)
        with pytest.raises(orbg.OrbgError) as ei:
            orbg.orbg_server_submit(srv, 999, 0, big, 1 << 17)
        assert ei.value.status == orbg.ORBG_ELIMIT
    finally:
        orbg.orbg_server_destroy(srv)


def test_cancel_waiting_running_and_finished_requests(orbg):
    """orbg_server_cancel withdraws a request wherever it is: still waiting
    (removed), in a batch (it runs, its results are dropped), or finished
    and not yet fetched (discarded).  A cancelled id is never reported by
    poll and cannot be fetched; every other request completes as usual and
    decodes as it does alone.  Which of the three cases a cancel meets
    depends on timing; each outcome is checked the same way."""
    import time
    cap = 10 ** 6
    codes_w = workloads.config5_codes()
    codes = [orbg.Code(c.H, max_query_cap=cap) for c in codes_w]
    cs = orbg.CodeSet(codes)
    srv = orbg.orbg_server_create(cs.handle, 64 << 20, cap, 2, 2048)
    try:
        reqs = [workloads.awgn_llr(codes_w[1], 1500, 2.5, 2000 + i)[0] for i in range(8)]
        for i, llr in enumerate(reqs):  # one request a batch, two batches at a time
            orbg.orbg_server_submit(srv, i, 1, llr, llr.shape[0])
        cancel = [0, 6, 7]
        for i in cancel:
            orbg.orbg_server_cancel(srv, i)
        for bad in (6, 12345):  # already withdrawn; never submitted
            with pytest.raises(orbg.OrbgError) as ei:
                orbg.orbg_server_cancel(srv, bad)
            assert ei.value.status == orbg.ORBG_EINVAL
        want = set(range(len(reqs))) - set(cancel)
        got = set()
        t0 = time.time()
        while got != want:
            ids = orbg.orbg_server_poll(srv, 64, 100000)
            assert not set(ids) & set(cancel)
            got.update(ids)
            assert time.time() - t0 < 120
        # a request that finishes and is neither polled nor fetched
        small = workloads.awgn_llr(codes_w[0], 8, 6.0, 2100)[0]
        orbg.orbg_server_submit(srv, 50, 0, small, small.shape[0])
        while True:
            st = orbg.orbg_server_stats_get(srv)
            if st["pending"] == 0 and st["inflight_batches"] == 0:
                break
            assert time.time() - t0 < 120
            time.sleep(0.001)
        orbg.orbg_server_cancel(srv, 50)
        assert 50 not in orbg.orbg_server_poll(srv, 64, 1000)
        for i in cancel + [50]:
            with pytest.raises(orbg.OrbgError):
                orbg.orbg_server_fetch(srv, i)
        cd = codes_w[1]
        for i in sorted(want):
            B = reqs[i].shape[0]
            cw = np.zeros(B * cd.n, np.uint8)
            q = np.zeros(B, np.uint32)
            ab = np.zeros(B, np.uint8)
            orbg.orbg_server_fetch(srv, i, cw, q, ab)
            if i in (1, 5):
                alone = _alone(orbg, cs, cd, reqs[i], cap, 1, len(codes))
                assert np.array_equal(cw.reshape(B, cd.n), alone[0])
                assert np.array_equal(q.astype(np.int64), alone[1])
                assert np.array_equal(ab, alone[2])
        st = orbg.orbg_server_stats_get(srv)
        assert st["cancelled"] == len(cancel) + 1
        assert st["submitted"] == len(reqs) + 1
    finally:
        orbg.orbg_server_destroy(srv)
