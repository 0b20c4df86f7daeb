"""The allocation-free batched entry point (orbg_decode_batched_noalloc).

It exists for callers that must not allocate device memory while they
decode -- for example a receiver that reserves all of its GPU memory at
start-up and treats any later allocation as a failure.  It runs the same
kernels as orbg_decode_batched with their scratch in a fixed array inside
the library, so its results must equal orbg_decode_batched's bit for bit
(the tolerance of every decoder test here is zero).

This file is collected last so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

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


def _run(ob, fn, cs, llr_t, n, cap):
    B = llr_t.shape[0]
    cw = torch.full((B, n), 0xAB, dtype=torch.uint8, device="cuda")
    q = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    ab = torch.full((B,), 0xCD, dtype=torch.uint8, device="cuda")
    fn(cs.handle, None, None, llr_t, B, cap, cw, None, q, ab, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return cw.cpu().numpy(), q.cpu().numpy(), ab.cpu().numpy()


def test_noalloc_equals_batched_on_two_calls_in_a_row(orbg):
    code = workloads.config2_code()
    c = orbg.Code(code.H, max_query_cap=10 ** 6)
    cs = orbg.CodeSet([c])
    # a small phase-1 budget so that the open-block list in the fixed array
    # is used by many blocks
    orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 8, 256, 16))
    for seed in (901, 902):   # two calls in a row, different inputs
        llr, _ = workloads.awgn_llr(code, 20000, 4.0, seed)
        llr_t = torch.from_numpy(llr).cuda()
        want = _run(orbg, orbg.orbg_decode_batched, cs, llr_t, code.n, 10 ** 6)
        got = _run(orbg, orbg.orbg_decode_batched_noalloc, cs, llr_t, code.n, 10 ** 6)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
        assert (want[1] > 256).any()  # phase 2 had work


def test_noalloc_rejects_what_it_cannot_do(orbg):
    code = workloads.config1_code()
    c = orbg.Code(code.H, max_query_cap=1000)
    cs = orbg.CodeSet([c])
    B = orbg.ORBG_NOALLOC_MAX_BLOCKS + 1
    x = torch.zeros((8, code.n), dtype=torch.float32, device="cuda")
    out = torch.zeros((8, code.n), dtype=torch.uint8, device="cuda")
    q = torch.zeros((8,), dtype=torch.int32, device="cuda")
    ab = torch.zeros((8,), dtype=torch.uint8, device="cuda")
    with pytest.raises(orbg.OrbgError) as ei:  # more blocks than the array holds
        orbg.orbg_decode_batched_noalloc(cs.handle, None, None, x, B, 1000, out, None, q, ab)
    assert ei.value.status == orbg.ORBG_ELIMIT
    with pytest.raises(orbg.OrbgError) as ei:  # host buffers would need staging
        orbg.orbg_decode_batched_noalloc(cs.handle, None, None, x.cpu().numpy(), 8, 1000,
                                         out, None, q, ab)
    assert ei.value.status == orbg.ORBG_EINVAL


def test_noalloc_mixed_codes_with_offsets(orbg):
    """Mixed codes of different n and syndrome widths in one call, with
    device code-id and offset arrays and a small phase-1 budget (so the
    open-block list, the per-code counts and the block order in the fixed
    array are all used): bit for bit the same as orbg_decode_batched."""
    codes = workloads.config4_codes() + [workloads.config3_code()]  # r = 13..34: 1 and 2 words
    cs = orbg.CodeSet([orbg.Code(c.H, max_query_cap=10 ** 5) for c in codes])
    orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 4, 128, 8))
    for seed in (903, 904):
        _, cid, llr, off, _, _ = workloads.mixed_inputs(codes, 6000, seed)
        llr_t = torch.from_numpy(llr).cuda()
        cid_t = torch.from_numpy(cid).cuda()
        off_t = torch.from_numpy(off).cuda()
        B = cid.shape[0]
        outs = []
        for fn in (orbg.orbg_decode_batched, orbg.orbg_decode_batched_noalloc):
            cw = torch.full((llr.shape[0],), 0xAB, dtype=torch.uint8, device="cuda")
            q = torch.full((B,), -1, dtype=torch.int32, device="cuda")
            ab = torch.full((B,), 0xCD, dtype=torch.uint8, device="cuda")
            fn(cs.handle, cid_t, off_t, llr_t, B, 10 ** 5, cw, off_t, q, ab,
               torch.cuda.current_stream())
            torch.cuda.synchronize()
            outs.append((cw.cpu().numpy(), q.cpu().numpy(), ab.cpu().numpy()))
        for g, w in zip(outs[1], outs[0]):
            assert np.array_equal(g, w)
        assert (outs[0][1] > 128).any() and (outs[0][2] == 0).any()
