"""GPU parity of full ORBGRAND with a piece-wise linear model fitted to every
block (Sec. III-E, Eq. Q, Eq. quant) and each block searched in its own
order (Sec. III-D, Eq. relest_seg): orbg_decode_fitted through the C ABI,
bit for bit (codeword, query count, abandon flag and model record) against
the oracle's fit-then-decode, for 1 to 4 lines, both quantisations, codes
of every keys-per-lane class and syndrome width, edge inputs, caps at the
hit, host buffers, and the BCH(127,113) workload at full size.  A block
whose one-warp search passes a quarter of the cap goes to the search where
all warps of a CTA share it, so these caps exercise both."""
import numpy as np
import pytest

import oracle
from paper_2202_13951_gb300 import workloads
from test_gpu_parity import assert_same, tiny_inputs

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


def run_fitted(orbg, c, llr, cap, lines, div):
    cw, q, ab, rec = orbg.decode_fitted(c, torch.from_numpy(llr).cuda(), cap, lines, div)
    torch.cuda.synchronize()
    return (cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy(),
            rec.cpu().numpy())


def check(orbg, code, llr, cap, lines, div):
    c = orbg.Code(code.H, max_query_cap=1 << 10)  # the fitted search needs no tables
    got = run_fitted(orbg, c, llr, cap, lines, div)
    want = oracle.decode_batch_fit(code.H, llr, cap, lines, div)[:3]
    assert_same(got[:3], want)
    for b in range(llr.shape[0]):
        assert orbg.model_of_record(got[3][b]) == oracle.fit(llr[b], lines, div), b
    return got


# (code, Eb/N0 points, cap): n in each keys-per-lane class (<= 32, 64, 128,
# 256) and syndromes of 1, 2 and 4 words
CASES = [
    ("rlc(24,16)", lambda: workloads.rlc(24, 16, 31), (1.0, 3.0, 5.0), 3000),
    ("rlc(64,51)", workloads.config1_code, (2.0, 4.0, 6.0), 20000),
    ("bch(127,113)", workloads.config2_code, (3.0, 4.0, 5.0, 6.0), 20000),
    ("ca-polar(128,94)", workloads.config3_code, (4.0, 5.0, 6.0), 20000),
    ("rlc(160,60)", lambda: workloads.rlc(160, 60, 32), (8.0,), 2000),
    ("ca-polar[256,234]", lambda: workloads.paper256_codes()[0], (4.0, 5.0, 6.0), 50000),
]


@pytest.mark.parametrize("name,make,points,cap", CASES, ids=[c[0] for c in CASES])
def test_fitted_search_matches_oracle(orbg, name, make, points, cap):
    code = make()
    rng = np.random.default_rng(code.n)
    llr = np.concatenate([workloads.awgn_llr(code, 40, eb, code.n + int(10 * eb))[0]
                          for eb in points] + [tiny_inputs(code.n, rng, 10)])
    for lines in (1, 2, 3, 4):
        for div in (False, True):
            got = check(orbg, code, llr, cap, lines, div)
            assert (got[2] != orbg.ORBG_BLOCK_RANGE).all()


def test_fitted_search_edges(orbg):
    """NaN blocks (flag 2, query 0, hard decision, record m = 0), a
    noiseless block (query 1), cap 1, and caps exactly at and one below each
    block's hit."""
    code = workloads.config2_code()
    llr, sent = workloads.awgn_llr(code, 60, 4.0, 41)
    llr[3, 7] = np.nan
    llr[4] = np.where(sent[4] == 1, 5.0, -5.0)
    c = orbg.Code(code.H, max_query_cap=1 << 10)
    for lines in (2, 3):
        cw, q, ab, rec = run_fitted(orbg, c, llr, 20000, lines, False)
        assert ab[3] == orbg.ORBG_BLOCK_NAN and q[3] == 0 and not rec[3].any()
        assert (cw[3] == (llr[3] > 0)).all()
        assert q[4] == 1 and ab[4] == 0 and (cw[4] == sent[4]).all()
        ok = np.ones(llr.shape[0], bool)
        ok[3] = False
        want = oracle.decode_batch_fit(code.H, llr[ok], 20000, lines)
        assert_same((cw[ok], q[ok], ab[ok]), want[:3])
        got1 = run_fitted(orbg, c, llr[ok], 1, lines, False)
        assert_same(got1[:3], oracle.decode_batch_fit(code.H, llr[ok], 1, lines)[:3])
        dec = np.nonzero(want[2] == 0)[0][:12]
        for b in dec:
            row = llr[ok][b:b + 1]
            for cap in (int(want[1][b]), int(want[1][b]) - 1):
                if cap < 1:
                    continue
                got = run_fitted(orbg, c, row, cap, lines, False)
                assert_same(got[:3], oracle.decode_batch_fit(code.H, row, cap, lines)[:3])


def test_fitted_search_host_buffers(orbg):
    """Host buffers are staged; a NaN block makes the call return ENAN after
    writing every block."""
    code = workloads.config1_code()
    llr = workloads.awgn_llr(code, 30, 3.0, 43)[0]
    c = orbg.Code(code.H, max_query_cap=1 << 10)
    B, n = llr.shape
    cw = np.zeros((B, n), np.uint8)
    q = np.zeros(B, np.uint32)
    ab = np.zeros(B, np.uint8)
    rec = np.zeros((B, orbg.ORBG_FIT_STRIDE), np.int32)
    orbg.orbg_decode_fitted(c.handle, llr, B, 5000, 3, False, cw, q, ab, rec)
    want = oracle.decode_batch_fit(code.H, llr, 5000, 3)
    assert_same((cw, q.astype(np.int64), ab), want[:3])
    llr[5, 0] = np.nan
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_decode_fitted(c.handle, llr, B, 5000, 3, False, cw, q, ab, None)
    assert ei.value.status == orbg.ORBG_ENAN and ab[5] == orbg.ORBG_BLOCK_NAN
    with pytest.raises(orbg.OrbgError):
        orbg.orbg_decode_fitted(c.handle, llr, B, 5000, 9, False, cw, q, ab, None)


def test_fitted_search_bch_workload_full_size(orbg):
    """The BCH(127,113) workload (4 x 100,000 blocks at 4-7 dB, cap 1e6)
    with three lines fitted per block in one launch: 1,500 seeded random
    blocks against the oracle, the longest searches among them, and every
    decoded block a codeword."""
    code = workloads.config2_code()
    llr = np.concatenate([workloads.awgn_llr(code, 100000, eb, s)[0]
                          for eb, s in zip((4.0, 5.0, 6.0, 7.0), (201, 202, 203, 204))])
    c = orbg.Code(code.H, max_query_cap=1 << 10)
    cw, q, ab, _ = run_fitted(orbg, c, llr, 10 ** 6, 3, False)
    assert (ab != orbg.ORBG_BLOCK_RANGE).all()
    dec = ab == 0
    assert not ((cw[dec].astype(np.int64) @ code.H.T.astype(np.int64)) % 2).any()
    rng = np.random.default_rng(9)
    pick = np.concatenate([rng.choice(llr.shape[0], 1400, replace=False),
                           np.argsort(q)[-100:]])
    pick = np.unique(pick)
    want = oracle.decode_batch_fit(code.H, llr[pick], 10 ** 6, 3)[:3]
    assert_same((cw[pick], q[pick], ab[pick]), want)
