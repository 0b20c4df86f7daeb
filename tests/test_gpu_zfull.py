"""GPU parity of full ORBGRAND and the paper-shaped workload, through the
C ABI, bit for bit against the oracle: decoding in m-segment orders (Sec.
III-D, Eq. relest_seg) through model tables, the per-block fit on the
device (Sec. III-E, Eq. Q, Eq. quant), and the [256,234] family of Sec. IV
at full size."""
import numpy as np
import pytest

import oracle
from paper_2202_13951_gb300 import workloads
from test_gpu_parity import assert_same, gpu_batched, gpu_plain, tiny_inputs

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


# ------------------------------------------- m-segment full ORBGRAND

def _models(n, llr):
    """Hand-set models — a zero-weight least reliable position; light
    positions far down the order, which leave the flat table empty — and
    models fitted (Sec. III-E) to three of the blocks."""
    return [((n // 8,), (-2, n // 8 + 3), (2, 1)), ((n * 5 // 8,), (-4, 0), (9, 4)),
            oracle.fit(llr[0], 3), oracle.fit(llr[1], 2, True), oracle.fit(llr[2], 4)]


def test_m_segment_orbgrand(orbg):
    """m-segment full ORBGRAND (Sec. III-D, Eq. relest_seg): codes loaded
    with a model decode, plain, batched and all in the second phase,
    exactly as the m-segment oracle."""
    cap = 20000
    for n, k, seed, ebn0 in ((64, 51, 93, 3.5), (127, 113, 94, 4.0)):
        code = workloads.rlc(n, k, seed)
        rng = np.random.default_rng(seed + 1)
        awgn = workloads.awgn_llr(code, 180, ebn0, seed + 2)[0]
        llr = np.concatenate([tiny_inputs(n, rng, 20), awgn])
        for model in _models(n, awgn):
            want = oracle.decode_batch_mline(code.H, llr, cap, model)[:3]
            c = orbg.Code(code.H, max_query_cap=cap, model=model)
            assert_same(gpu_plain(orbg, c, llr, cap), want)
            cs = orbg.CodeSet([c])
            assert_same(gpu_batched(orbg, cs, llr, cap), want)
            orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 1, 64, 8))
            assert_same(gpu_batched(orbg, cs, llr, cap), want)


def test_m_segment_and_basic_codes_in_one_launch(orbg):
    """Blocks of a basic code and of the same code under an m-segment model
    in one batched launch decode as each order's oracle."""
    cap = 20000
    code = workloads.rlc(64, 51, 95)
    llr = workloads.awgn_llr(code, 300, 3.5, 96)[0]
    model = oracle.fit(llr[0], 3)
    cs = orbg.CodeSet([orbg.Code(code.H, max_query_cap=cap),
                       orbg.Code(code.H, max_query_cap=cap, model=model)])
    cid = (np.arange(llr.shape[0]) % 2).astype(np.int32)
    llr_t = torch.from_numpy(llr).cuda()
    cid_t = torch.from_numpy(cid).cuda()
    cw, q, ab = orbg.decode_batched(cs, llr_t, cap, code_id=cid_t)
    torch.cuda.synchronize()
    got = (cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy())
    basic = oracle.decode_batch(code.H, llr[cid == 0], cap)[:3]
    seg = oracle.decode_batch_mline(code.H, llr[cid == 1], cap, model)[:3]
    assert_same(tuple(x[cid == 0] for x in got), basic)
    assert_same(tuple(x[cid == 1] for x in got), seg)


# ------------------------------------------- paper-shaped workload

def test_paper256_full_size_sampled(orbg):
    """The paper-shaped [256, 234] family of Sec. IV (CA-Polar, CRC, RLC and
    BCH[255, 231]), 400,000 blocks at Eb/N0 U[4, 7] dB, cap 5e6, one batched
    launch: 40 seeded random blocks of each code against the oracle, and
    every decoded block a codeword."""
    cap = 5 * 10 ** 6
    codes, cid, llr, off, _, _ = workloads.paper256_inputs()
    cs = orbg.CodeSet([orbg.Code(cd.H, max_query_cap=cap) for cd in codes])
    llr_t = torch.from_numpy(llr).cuda()
    off_t = torch.from_numpy(off).cuda()
    cid_t = torch.from_numpy(cid).cuda()
    cw, q, ab = orbg.decode_batched(cs, llr_t, cap, code_id=cid_t, llr_offset=off_t,
                                    cw_offset=off_t, n_total=llr.shape[0])
    torch.cuda.synchronize()
    cw, q, ab = cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()
    rng = np.random.default_rng(8)
    for j, cd in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        rows = np.stack([cw[off[b]:off[b] + cd.n] for b in idx])
        ok = ab[idx] == 0
        assert not ((rows[ok].astype(np.int64) @ cd.H.T.astype(np.int64)) % 2).any()
        pick = np.sort(rng.choice(idx.shape[0], size=40, replace=False))
        blocks = np.stack([llr[off[b]:off[b] + cd.n] for b in idx[pick]])
        want = oracle.decode_batch(cd.H, blocks, cap)[:3]
        assert_same((rows[pick], q[idx[pick]], ab[idx[pick]]), want)


# ------------------------------------------- per-block fit on the device

def _blocks(n, k, rng):
    code = workloads.rlc(n, k, seed=n + 7)
    parts = [workloads.awgn_llr(code, 40, snr, seed=int(10 * snr) + n)[0]
             for snr in (1.0, 3.0, 5.0, 7.0)]
    extra = np.stack([rng.normal(0.0, 2.0, n), np.round(rng.normal(0.0, 2.0, n)),
                      np.full(n, 1.5), np.full(n, np.inf)]).astype(np.float32)
    extra[0, :3] = np.inf
    return np.concatenate(parts + [extra])


@pytest.mark.parametrize("n,k", [(4, 2), (31, 20), (64, 48), (127, 113), (255, 231),
                                 (256, 234)])
def test_fit_models_match_oracle(orbg, n, k):
    rng = np.random.default_rng(n)
    llr = _blocks(n, k, rng)
    d = torch.from_numpy(llr).cuda()
    for lines in (1, 2, 3, 4, 8):
        for div in (False, True):
            rec = orbg.fit_models(d, n, lines, div).cpu().numpy()
            torch.cuda.synchronize()
            for b in range(llr.shape[0]):
                assert orbg.model_of_record(rec[b]) == oracle.fit(llr[b], lines, div), (
                    n, lines, div, b)


def test_fit_models_small_n_nan_and_empty(orbg):
    """n < 4 gives the basic model; a NaN block gives m = 0 and leaves the
    others alone; B = 0 is a no-op; host buffers are refused."""
    rng = np.random.default_rng(5)
    for n in (1, 2, 3):
        x = rng.normal(0.0, 2.0, (3, n)).astype(np.float32)
        rec = orbg.fit_models(torch.from_numpy(x).cuda(), n, 3).cpu().numpy()
        assert all(orbg.model_of_record(r) == ((), (0,), (1,)) for r in rec)
    x = rng.normal(0.0, 2.0, (3, 64)).astype(np.float32)
    x[1, 10] = np.nan
    rec = orbg.fit_models(torch.from_numpy(x).cuda(), 64, 3).cpu().numpy()
    assert orbg.model_of_record(rec[1]) is None and not rec[1].any()
    for b in (0, 2):
        assert orbg.model_of_record(rec[b]) == oracle.fit(x[b], 3)
    lib = orbg.load_library()
    empty = torch.empty((0,), dtype=torch.float32, device="cuda")
    out = torch.empty((0,), dtype=torch.int32, device="cuda")
    assert lib.orbg_fit_models(empty.data_ptr(), 0, 64, 3, 0, out.data_ptr(), None) == 0
    host = np.zeros((2, 64), np.float32)
    hout = np.zeros((2, 24), np.int32)
    assert lib.orbg_fit_models(host.ctypes.data, 2, 64, 3, 0, hout.ctypes.data,
                               None) == orbg.ORBG_EINVAL
    assert lib.orbg_fit_models(None, 2, 300, 3, 0, None, None) == orbg.ORBG_EINVAL


def test_fitted_model_decodes_as_oracle(orbg):
    """A model fitted on the device, loaded with orbg_load_code_model,
    decodes the blocks as the oracle's fit-then-decode (Sec. III-E then the
    m-segment order) does for the block it was fitted to."""
    code = workloads.rlc(64, 51, 97)
    llr, _ = workloads.awgn_llr(code, 60, 4.0, 98)
    rec = orbg.fit_models(torch.from_numpy(llr).cuda(), 64, 3).cpu().numpy()
    model = orbg.model_of_record(rec[0])
    c = orbg.Code(code.H, max_query_cap=20000, model=model)
    llr_t = torch.from_numpy(llr[:1]).cuda()
    cw, q, ab = orbg.decode(c, llr_t, 20000)
    torch.cuda.synchronize()
    wc, wq, wab, _ = oracle.decode_batch_fit(code.H, llr[:1], 20000, 3)
    assert (cw.cpu().numpy() == wc).all() and int(q[0]) == int(wq[0]) and int(ab[0]) == int(wab[0])


def test_fitted_line_decode_as_oracle(orbg):
    """One-line full ORBGRAND with each block's own line (Sec. III-E, one
    line, then Sec. III-D's order), in one call: equal to the oracle's
    fit-then-decode block by block, over SNRs that give many distinct
    lines (including J_0 = -1), with a NaN block, both quantisations, and
    a second call that reuses the cached handles."""
    cap = 20000
    for code, seed in ((workloads.rlc(64, 51, 99), 100), (workloads.config2_code(), 101)):
        llr = np.concatenate([workloads.awgn_llr(code, 120, eb, seed + int(eb))[0]
                              for eb in (2.0, 4.0, 6.0, 8.0)])
        llr[7, 3] = np.nan
        c = orbg.Code(code.H, max_query_cap=cap)
        for div in (False, True):
            f = orbg.Fitted(c, divisible=div)
            d = torch.from_numpy(llr).cuda()
            for _ in range(2):
                cw, q, ab, rec = f.decode(d, cap)
                torch.cuda.synchronize()
                ok = np.ones(llr.shape[0], bool)
                ok[7] = False
                want = oracle.decode_batch_fit(code.H, llr[ok], cap, 1, div)[:3]
                assert_same((cw.cpu().numpy()[ok], q.cpu().numpy().astype(np.int64)[ok],
                             ab.cpu().numpy()[ok]), want)
                assert int(ab[7]) == 2 and int(q[7]) == 0
                rec = rec.cpu().numpy()
                for b in np.nonzero(ok)[0][::17]:
                    assert orbg.model_of_record(rec[b]) == oracle.fit(llr[b], 1, div)
            f.close()


def test_fitted_decode_after_a_failed_line(orbg):
    """A call that adds one line's handle and then fails on a later line
    (here a block whose fitted J_0 orders n = 256 positions Hamming weight
    first, which the tables refuse) must not leave the object decoding with
    a code set that lacks the added handle: the next call over blocks of
    that line equals the oracle's fit-then-decode."""
    cap = 5000
    code = workloads.rlc(256, 240, 71)
    c = orbg.Code(code.H, max_query_cap=cap)
    f = orbg.Fitted(c)
    first = workloads.awgn_llr(code, 1, 7.0, 72)[0]  # one block: one line
    cw, q, ab, rec = f.decode(torch.from_numpy(first).cuda(), cap)
    torch.cuda.synchronize()
    seen = {orbg.model_of_record(r)[1][0] for r in rec.cpu().numpy()}
    # blocks at a lower SNR: lines not met in the first call
    low = workloads.awgn_llr(code, 256, 2.0, 73)[0]
    j0 = np.array([oracle.fit(x, 1)[1][0] for x in low])
    new = low[~np.isin(j0, list(seen))][:8]
    assert new.shape[0] > 0
    rng = np.random.default_rng(74)
    flat = (10.0 + 1e-4 * np.arange(1, 257)) * rng.choice([-1.0, 1.0], 256)
    flat = flat[rng.permutation(256)].astype(np.float32)[None, :]
    assert oracle.fit(flat[0], 1)[1][0] > 256 * 257 // 2
    with pytest.raises(orbg.OrbgError):
        f.decode(torch.from_numpy(np.concatenate([new, flat])).cuda(), cap)
    torch.cuda.synchronize()
    cw, q, ab, _ = f.decode(torch.from_numpy(new).cuda(), cap)
    torch.cuda.synchronize()
    want = oracle.decode_batch_fit(code.H, new, cap, 1)[:3]
    assert_same((cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()), want)
    f.close()
