"""GPU parity of the per-block fit (Sec. III-E, Eq. Q, Eq. quant) through
the C ABI: orbg_fit_models against the oracle's fit, block by block, bit
for bit (the model records are integers)."""
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
