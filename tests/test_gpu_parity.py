"""GPU parity: the CUDA decoder, called through the C ABI, against the CPU
oracle, element by element.  Bit-exact (tolerance 0) on the codeword, the
query count and the abandon flag: all three are integer results.

Sizes: small cases the oracle finishes in seconds (several warp groups of
runs, ragged n), and the full benchmark configurations decoded in the same
launch configuration the benchmark times, checked on a seeded random
sample of blocks the oracle decodes one by one.
"""
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


def gpu_plain(ob, code_obj, llr, cap):
    llr_t = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).cuda()
    cw, q, ab = ob.decode(code_obj, llr_t, cap)
    torch.cuda.synchronize()
    return (cw.cpu().numpy(), q.cpu().numpy().astype(np.int64),
            ab.cpu().numpy())


def gpu_batched(ob, codeset, llr, cap):
    llr_t = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).cuda()
    cw, q, ab = ob.decode_batched(codeset, llr_t, cap)
    torch.cuda.synchronize()
    return (cw.cpu().numpy(), q.cpu().numpy().astype(np.int64),
            ab.cpu().numpy())


def assert_same(got, want, idx=None):
    cw, q, ab = got
    wc, wq, wab = want[0], want[1].astype(np.int64), want[2]
    if idx is not None:
        cw, q, ab = cw[idx], q[idx], ab[idx]
    bad = np.nonzero((cw != wc).any(axis=1) | (q != wq) | (ab != wab))[0]
    assert bad.size == 0, "first mismatches %s: gpu q=%s ab=%s, oracle q=%s ab=%s" % (
        bad[:5], q[bad[:5]], ab[bad[:5]], wq[bad[:5]], wab[bad[:5]])


def tiny_inputs(n, rng, blocks):
    out = []
    for b in range(blocks):
        llr = rng.normal(0.0, 2.0, n).astype(np.float32)
        kind = b % 5
        if kind == 1:
            llr = np.round(llr).astype(np.float32)
        elif kind == 2:
            llr[rng.integers(0, n, 2)] = 0.0
            llr[rng.integers(0, n, 1)] = -0.0
            llr[rng.integers(0, n, 1)] = np.inf
            llr[rng.integers(0, n, 1)] = -np.inf
        elif kind == 3:
            llr = np.where(rng.random(n) < 0.5, -1.0, 1.0).astype(np.float32)
        out.append(llr)
    return np.stack(out)


# ------------------------------------------------------------ small codes

@pytest.mark.parametrize("cap", [1, 2, 3, 5, 17, 64, 128])
def test_hamming74_every_cap(orbg, cap):
    code = workloads.hamming74()
    c = orbg.Code(code.H)
    llr = tiny_inputs(7, np.random.default_rng(1), 200)
    want = oracle.decode_batch(code.H, llr, cap)[:3]
    assert_same(gpu_plain(orbg, c, llr, cap), want)


@pytest.mark.parametrize("n,k,seed", [(16, 11, 16), (32, 20, 3), (33, 20, 4),
                                      (64, 32, 5), (64, 31, 6), (65, 40, 7),
                                      (96, 70, 8), (127, 113, 9), (128, 96, 10),
                                      (160, 140, 11), (256, 240, 12), (256, 128, 13)])
def test_random_codes_plain_and_batched(orbg, n, k, seed):
    """n across key-padding cases (7..256), n-k on both sides of the 32/64
    word boundaries, up to n-k = 128."""
    code = workloads.rlc(n, k, seed)
    rng = np.random.default_rng(seed + 100)
    llr = np.concatenate([
        tiny_inputs(n, rng, 40),
        workloads.awgn_llr(code, 160, 3.0 + (seed % 4), seed + 200)[0]])
    cap = 20000
    want = oracle.decode_batch(code.H, llr, cap)[:3]
    c = orbg.Code(code.H, max_query_cap=cap)
    assert_same(gpu_plain(orbg, c, llr, cap), want)
    cs = orbg.CodeSet([c])
    assert_same(gpu_batched(orbg, cs, llr, cap), want)


def near_tie_inputs(code, blocks, ebn0, seed):
    """AWGN blocks in which pairs of reliabilities differ only in the lowest
    mantissa bits, the more reliable of each pair at the lower index: the
    decoder's sort keys keep only the high bits of |L| and must fall back to
    the exact order (Section II: ties in |L| are broken by index, not by
    value).  Pairs sit among the least reliable positions (read by the first
    queries) and deeper (read only by long searches)."""
    llr, _ = workloads.awgn_llr(code, blocks, ebn0, seed)
    rng = np.random.default_rng(seed + 1)
    bits = llr.view(np.uint32)
    for b in range(blocks):
        order = np.argsort(np.abs(llr[b]), kind="stable")
        ranks = [(0, 1), (2, 3 + int(rng.integers(0, 3))),
                 tuple(sorted(rng.choice(np.arange(6, min(40, code.n)), 2, replace=False)))]
        for r0, r1 in ranks[: 1 + b % 3]:
            i, j = sorted((int(order[r0]), int(order[r1])))
            base = bits[b, i] & np.uint32(0xFFFFFF00)
            sign_i = bits[b, i] & np.uint32(0x80000000)
            sign_j = bits[b, j] & np.uint32(0x80000000)
            mag = base & np.uint32(0x7FFFFFFF)
            bits[b, i] = sign_i | mag | np.uint32(0x05)   # lower index, larger |L|
            bits[b, j] = sign_j | mag | np.uint32(0x02)   # same high bits
    return llr


@pytest.mark.parametrize("n,k,seed", [(31, 20, 71), (64, 45, 72), (127, 113, 73),
                                      (200, 180, 74), (255, 239, 75)])
def test_near_ties_exact_order(orbg, n, k, seed):
    code = workloads.rlc(n, k, seed)
    llr = near_tie_inputs(code, 300, 3.5, seed + 10)
    cap = 20000
    want = oracle.decode_batch(code.H, llr, cap)[:3]
    c = orbg.Code(code.H, max_query_cap=cap)
    assert_same(gpu_plain(orbg, c, llr, cap), want)
    cs = orbg.CodeSet([c])
    assert_same(gpu_batched(orbg, cs, llr, cap), want)
    orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 1, 1, 8))
    assert_same(gpu_batched(orbg, cs, llr, cap), want)


def test_generator_matrix_input_same_result(orbg):
    """Loading G (the library derives its own H) decodes identically."""
    code = workloads.config1_code()
    llr, _ = workloads.awgn_llr(code, 500, 4.0, 77)
    want = oracle.decode_batch(code.H, llr, 100000)[:3]
    cg = orbg.Code(code.G, kind=orbg.ORBG_MAT_G, n=code.n, k=code.k, max_query_cap=100000)
    assert_same(gpu_plain(orbg, cg, llr, 100000), want)


def test_cap_exactly_at_hit(orbg):
    code = workloads.rlc(64, 50, 31)
    llr, _ = workloads.awgn_llr(code, 300, 3.0, 32)
    _, q, ab, _ = oracle.decode_batch(code.H, llr, 200000)
    c = orbg.Code(code.H, max_query_cap=200000)
    for b in np.nonzero((ab == 0) & (q > 40))[0][:20]:
        qb = int(q[b])
        for cap in (qb - 1, qb):
            want = oracle.decode_batch(code.H, llr[b:b + 1], cap)[:3]
            assert_same(gpu_plain(orbg, c, llr[b:b + 1], cap), want)


def test_nan_block_flagged(orbg):
    code = workloads.config1_code()
    llr, _ = workloads.awgn_llr(code, 64, 5.0, 5)
    llr[3, 7] = np.nan
    c = orbg.Code(code.H, max_query_cap=1000)
    cw, q, ab = gpu_plain(orbg, c, llr, 1000)
    assert ab[3] == orbg.ORBG_BLOCK_NAN and q[3] == 0
    others = np.arange(64) != 3
    want = oracle.decode_batch(code.H, llr[others], 1000)[:3]
    assert_same((cw[others], q[others], ab[others]), want)
    # host-buffer call reports ENAN
    cwh = np.zeros((64, code.n), np.uint8)
    qh = np.zeros(64, np.uint32)
    abh = np.zeros(64, np.uint8)
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_decode(c.handle, llr, 64, 1000, cwh, qh, abh)
    assert ei.value.status == orbg.ORBG_ENAN


def test_empty_batch(orbg):
    code = workloads.config1_code()
    c = orbg.Code(code.H)
    e = torch.empty((0, code.n), dtype=torch.float32, device="cuda")
    cw, q, ab = orbg.decode(c, e, 100)
    assert cw.shape == (0, code.n)


def test_host_buffers_match_device_buffers(orbg):
    code = workloads.config2_code()
    llr, _ = workloads.awgn_llr(code, 3000, 4.5, 9)
    c = orbg.Code(code.H, max_query_cap=10 ** 6)
    dev = gpu_plain(orbg, c, llr, 10 ** 6)
    cw = np.zeros((3000, code.n), np.uint8)
    q = np.zeros(3000, np.uint32)
    ab = np.zeros(3000, np.uint8)
    orbg.orbg_decode(c.handle, llr, 3000, 10 ** 6, cw, q, ab)
    assert_same((cw, q.astype(np.int64), ab), dev)
    cs = orbg.CodeSet([c])
    orbg.orbg_decode_batched(cs.handle, None, None, llr, 3000, 10 ** 6, cw, None, q, ab)
    assert_same((cw, q.astype(np.int64), ab), dev)


def test_single_code_with_offsets(orbg):
    """One code, no code ids, but a custom layout: blocks stored out of order
    with gaps (per-block LLR and codeword offsets).  Same results as the
    oracle, block by block, in both phases."""
    code = workloads.rlc(127, 106, 81)
    llr, _ = workloads.awgn_llr(code, 700, 3.5, 82)
    B, n = llr.shape
    rng = np.random.default_rng(83)
    order = rng.permutation(B)
    stride = n + 9
    flat = np.full(B * stride + 5, np.nan, np.float32)   # gaps hold NaN: never read
    off = np.empty(B, np.int64)
    for pos, b in enumerate(order):
        off[b] = 5 + pos * stride
        flat[off[b]:off[b] + n] = llr[b]
    cap = 30000
    want = oracle.decode_batch(code.H, llr, cap)[:3]
    c = orbg.Code(code.H, max_query_cap=cap)
    cs = orbg.CodeSet([c])
    for tuning in (None, (8, 0, 1, 64, 8)):
        if tuning:
            orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(*tuning))
        off_t = torch.from_numpy(off).cuda()
        cw, q, ab = orbg.decode_batched(cs, torch.from_numpy(flat).cuda(), cap,
                                        llr_offset=off_t, cw_offset=off_t,
                                        n_total=flat.shape[0])
        torch.cuda.synchronize()
        cw = cw.cpu().numpy()
        got = (np.stack([cw[o:o + n] for o in off]), q.cpu().numpy().astype(np.int64),
               ab.cpu().numpy())
        assert_same(got, want)


def test_pipelined_host_buffers(orbg):
    """A large single-code call on host buffers is cut into chunks whose
    copies and decodes overlap on three streams: every block equals the
    device-buffer call, and a NaN block in a late chunk is still reported."""
    code, llr, _ = workloads.config2_inputs(B_per_point=50_000)
    B, n = llr.shape
    c = orbg.Code(code.H, max_query_cap=10 ** 6)
    cs = orbg.CodeSet([c])
    dev = gpu_batched(orbg, cs, llr, 10 ** 6)
    cw = np.zeros((B, n), np.uint8)
    q = np.zeros(B, np.uint32)
    ab = np.zeros(B, np.uint8)
    orbg.orbg_decode_batched(cs.handle, None, None, llr, B, 10 ** 6, cw, None, q, ab)
    assert_same((cw, q.astype(np.int64), ab), dev)
    llr2 = llr.copy()
    llr2[B - 5, 3] = np.nan
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_decode_batched(cs.handle, None, None, llr2, B, 10 ** 6, cw, None, q, ab)
    assert ei.value.status == orbg.ORBG_ENAN
    assert ab[B - 5] == orbg.ORBG_BLOCK_NAN and q[B - 5] == 0
    keep = np.arange(B) != B - 5
    assert_same((cw[keep], q[keep].astype(np.int64), ab[keep]),
                (dev[0][keep], dev[1][keep], dev[2][keep]))


def test_pipelined_host_buffers_mixed_codes(orbg):
    """The chunked host-buffer path with code ids and per-block offsets
    (blocks in order, no overlap): equal to the same call on device
    buffers, block by block."""
    codes, cid, llr, off, cwt, ebn0 = workloads.config4_inputs(B=160_000, seed=4403)
    objs = [orbg.Code(cd.H, max_query_cap=10 ** 5) for cd in codes]
    cs = orbg.CodeSet(objs)
    B = cid.shape[0]
    n_total = llr.shape[0]
    cw_d, q_d, ab_d = orbg.decode_batched(cs, torch.from_numpy(llr).cuda(), 10 ** 5,
                                          code_id=torch.from_numpy(cid).cuda(),
                                          llr_offset=torch.from_numpy(off).cuda(),
                                          cw_offset=torch.from_numpy(off).cuda(),
                                          n_total=n_total)
    torch.cuda.synchronize()
    cw = np.zeros(n_total, np.uint8)
    q = np.zeros(B, np.uint32)
    ab = np.zeros(B, np.uint8)
    orbg.orbg_decode_batched(cs.handle, cid, off, llr, B, 10 ** 5, cw, off, q, ab)
    assert np.array_equal(cw, cw_d.cpu().numpy())
    assert np.array_equal(q, q_d.cpu().numpy().astype(np.uint32))
    assert np.array_equal(ab, ab_d.cpu().numpy())


def test_pipelined_host_buffers_many_phase2_blocks(orbg):
    """With a phase-1 budget of one query nearly every block goes to phase 2:
    more than the 65,536 whose outputs the chunked path gathers, so it copies
    every output again after phase 2; with a budget of 64 fewer go, and the
    gathered outputs land over the chunk copies.  Both equal the unchunked
    device-buffer call."""
    code = workloads.config2_code()
    llr = workloads.awgn_llr(code, 160_000, 3.5, 4406)[0]
    B, n = llr.shape
    cs = orbg.CodeSet([orbg.Code(code.H, max_query_cap=10 ** 4)])
    for budget in (1, 64):
        orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 4, budget, 8))
        dev = gpu_batched(orbg, cs, llr, 10 ** 4)
        if budget == 1:
            assert (dev[1] > 1).sum() > 65536
        cw = np.zeros((B, n), np.uint8)
        q = np.zeros(B, np.uint32)
        ab = np.zeros(B, np.uint8)
        orbg.orbg_decode_batched(cs.handle, None, None, llr, B, 10 ** 4, cw, None, q, ab)
        assert_same((cw, q.astype(np.int64), ab), dev)


def test_pipelined_host_buffers_unordered_and_invalid(orbg):
    """Host offsets that do not place the blocks in order (here the second
    half before the first) take the unchunked path with the same results;
    a code id outside the set in a late chunk is rejected (ORBG_EINVAL)
    with the outputs untouched."""
    codes, cid, llr, off, _, _ = workloads.config4_inputs(B=140_000, seed=4405)
    cs = orbg.CodeSet([orbg.Code(cd.H, max_query_cap=10 ** 4) for cd in codes])
    B = cid.shape[0]
    n_total = llr.shape[0]
    half = B // 2
    perm = np.concatenate([np.arange(half, B), np.arange(half)])
    cid2, off2 = cid[perm].copy(), off[perm].copy()
    cw_d, q_d, ab_d = orbg.decode_batched(cs, torch.from_numpy(llr).cuda(), 10 ** 4,
                                          code_id=torch.from_numpy(cid2).cuda(),
                                          llr_offset=torch.from_numpy(off2).cuda(),
                                          cw_offset=torch.from_numpy(off2).cuda(),
                                          n_total=n_total)
    torch.cuda.synchronize()
    cw = np.zeros(n_total, np.uint8)
    q = np.zeros(B, np.uint32)
    ab = np.zeros(B, np.uint8)
    orbg.orbg_decode_batched(cs.handle, cid2, off2, llr, B, 10 ** 4, cw, off2, q, ab)
    assert np.array_equal(cw, cw_d.cpu().numpy())
    assert np.array_equal(q, q_d.cpu().numpy().astype(np.uint32))
    assert np.array_equal(ab, ab_d.cpu().numpy())
    bad = cid.copy()
    bad[B - 3] = len(codes)
    cw[:] = 0
    q[:] = 0
    ab[:] = 0
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_decode_batched(cs.handle, bad, off, llr, B, 10 ** 4, cw, off, q, ab)
    assert ei.value.status == orbg.ORBG_EINVAL
    assert not cw.any() and not q.any() and not ab.any()
    orbg.orbg_pool_trim()


def test_batched_call_in_cuda_graph(orbg):
    """A batched call on device buffers (stream-ordered scratch allocation,
    counter reset, both launches) captures into a CUDA graph; every replay
    equals the direct call."""
    code, llr, _ = workloads.config2_inputs(B_per_point=5000)
    B, n = llr.shape
    c = orbg.Code(code.H, max_query_cap=10 ** 6)
    cs = orbg.CodeSet([c])
    x = torch.from_numpy(llr).cuda()
    want = gpu_batched(orbg, cs, llr, 10 ** 6)
    cw = torch.empty((B, n), dtype=torch.uint8, device="cuda")
    q = torch.empty(B, dtype=torch.int32, device="cuda")
    ab = torch.empty(B, dtype=torch.uint8, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        orbg.orbg_decode_batched(cs.handle, None, None, x, B, 10 ** 6, cw, None, q, ab,
                                 torch.cuda.current_stream())
    for _ in range(2):
        cw.fill_(0xFF)
        q.fill_(-1)
        ab.fill_(0xFF)
        g.replay()
        torch.cuda.synchronize()
        assert_same((cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()),
                    want)


@pytest.mark.parametrize("line", [(3, 1), (5, 2), (20, 1)], ids=lambda l: "J%d_b%d" % l)
def test_one_line_orbgrand(orbg, line):
    """One-line full ORBGRAND (Sec. III-D): codes loaded with a line decode,
    in both forms, exactly as the one-line oracle."""
    cap = 20000
    for n, k, seed, ebn0 in ((64, 51, 91, 3.5), (127, 113, 92, 4.0)):
        code = workloads.rlc(n, k, seed)
        rng = np.random.default_rng(seed + 1)
        llr = np.concatenate([tiny_inputs(n, rng, 20),
                              workloads.awgn_llr(code, 180, ebn0, seed + 2)[0]])
        want = oracle.decode_batch_1line(code.H, llr, cap, *line)[:3]
        c = orbg.Code(code.H, max_query_cap=cap, line=line)
        assert_same(gpu_plain(orbg, c, llr, cap), want)
        cs = orbg.CodeSet([c])
        assert_same(gpu_batched(orbg, cs, llr, cap), want)
        orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 1, 64, 8))
        assert_same(gpu_batched(orbg, cs, llr, cap), want)


def test_mixed_codes_one_launch_equals_alone(orbg):
    """Blocks of four codes with different n and n-k in one batched launch
    give what each code's blocks give alone, and what the oracle gives."""
    codes, cid, llr, off, cwt, ebn0 = workloads.config4_inputs(B=4000, seed=4401)
    objs = [orbg.Code(cd.H, max_query_cap=10 ** 6) for cd in codes]
    cs = orbg.CodeSet(objs)
    llr_t = torch.from_numpy(llr).cuda()
    off_t = torch.from_numpy(off).cuda()
    cid_t = torch.from_numpy(cid).cuda()
    cw, q, ab = orbg.decode_batched(cs, llr_t, 10 ** 6, code_id=cid_t, llr_offset=off_t,
                                    cw_offset=off_t, n_total=llr.shape[0])
    torch.cuda.synchronize()
    cw, q, ab = cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()
    rng = np.random.default_rng(5)
    for j, cd in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        blocks = np.stack([llr[off[b]:off[b] + cd.n] for b in idx])
        alone = gpu_plain(orbg, objs[j], blocks, 10 ** 6)
        mixed = (np.stack([cw[off[b]:off[b] + cd.n] for b in idx]), q[idx], ab[idx])
        assert_same(mixed, alone)
        pick = rng.choice(idx.shape[0], size=min(40, idx.shape[0]), replace=False)
        want = oracle.decode_batch(cd.H, blocks[pick], 10 ** 6)[:3]
        assert_same(alone, want, pick)


def test_code_ids_outside_the_set_and_one_variant_sets(orbg):
    """Device code ids outside the set give queries 0 and flag 2, in a set
    of several decoder variants (blocks grouped by variant, ids outside the
    set with the last) and in a set of two codes of one variant (one launch,
    no grouping); every other block equals its code's plain decode."""
    small = workloads.rlc(64, 51, 71)
    other = workloads.rlc(60, 45, 72)      # same variant as `small` (n <= 64, one word)
    big = workloads.rlc(200, 180, 73)
    rng = np.random.default_rng(74)
    for codes in ([small, other], [big, small, other]):
        B = 3000
        cid = rng.integers(0, len(codes), B).astype(np.int32)
        bad = rng.choice(B, 25, replace=False)
        cid[bad[:12]] = len(codes)
        cid[bad[12:]] = -1
        n_of = np.array([c.n for c in codes] + [codes[0].n], np.int64)
        n_blk = n_of[np.where(cid >= 0, np.minimum(cid, len(codes)), len(codes))]
        off = np.concatenate([[0], np.cumsum(n_blk)[:-1]]).astype(np.int64)
        llr = (rng.standard_normal(int(n_blk.sum())) * 2.0 + 3.0).astype(np.float32)
        objs = [orbg.Code(c.H, max_query_cap=10 ** 5) for c in codes]
        cs = orbg.CodeSet(objs)
        cw = torch.full((llr.shape[0],), 7, dtype=torch.uint8, device="cuda")
        q = torch.full((B,), -1, dtype=torch.int32, device="cuda")
        ab = torch.full((B,), 0xFF, dtype=torch.uint8, device="cuda")
        off_t = torch.from_numpy(off).cuda()
        orbg.orbg_decode_batched(cs.handle, torch.from_numpy(cid).cuda(), off_t,
                                 torch.from_numpy(llr).cuda(), B, 10 ** 5, cw, off_t, q, ab,
                                 torch.cuda.current_stream())
        torch.cuda.synchronize()
        cw, q, ab = cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()
        assert (q[bad] == 0).all() and (ab[bad] == orbg.ORBG_BLOCK_NAN).all()
        for b in bad:
            assert (cw[off[b]:off[b] + n_blk[b]] == 7).all()
        for j, cd in enumerate(codes):
            idx = np.nonzero(cid == j)[0]
            blocks = np.stack([llr[off[b]:off[b] + cd.n] for b in idx])
            alone = gpu_plain(orbg, objs[j], blocks, 10 ** 5)
            assert_same((np.stack([cw[off[b]:off[b] + cd.n] for b in idx]), q[idx], ab[idx]),
                        alone)


# ------------------------------------------------ benchmark configurations

def test_config1_full_parity(orbg):
    """RLC(64,51), 5 dB, all-zero and random information, 2 x 10,000 blocks,
    cap 1e5, plain single launch: every block against the oracle."""
    code, llr, _ = workloads.config1_inputs()
    want = oracle.decode_batch(code.H, llr, 10 ** 5)[:3]
    c = orbg.Code(code.H, max_query_cap=10 ** 5)
    assert_same(gpu_plain(orbg, c, llr, 10 ** 5), want)


def _sampled(orbg, code, llr, cap, nsample, seed):
    c = orbg.Code(code.H, max_query_cap=cap)
    cs = orbg.CodeSet([c])
    got = gpu_batched(orbg, cs, llr, cap)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(llr.shape[0], size=nsample, replace=False))
    want = oracle.decode_batch(code.H, llr[pick], cap)[:3]
    assert_same(got, want, pick)
    return got


def test_config2_full_size_sampled(orbg):
    """BCH(127,113), 4 x 100,000 blocks at 4..7 dB, cap 1e6, one batched
    launch (the benchmark's call); 3000 seeded random blocks checked, and
    every block when oracle.cache holds this configuration."""
    from oracle import cache
    code, llr, _ = workloads.config2_inputs()
    got = _sampled(orbg, code, llr, 10 ** 6, 3000, 2)
    full = cache.load(2)
    if full is not None:
        assert_same(got, (full["cw"].reshape(llr.shape), full["q"], full["ab"]))
    # property at any size: every decoded block is a codeword
    cw, q, ab = got
    ok = ab == 0
    H = torch.from_numpy(code.H.astype(np.float32)).cuda()
    syn = (torch.from_numpy(cw[ok].astype(np.float32)).cuda() @ H.T) % 2
    assert int(syn.abs().sum().item()) == 0


def _stratified_pick(q, ab, rng, n_abandoned, n_longest, n_random, within=None):
    """Blocks to check: some the GPU abandoned, the longest decoded
    searches, and seeded random ones (indices into q, sorted, unique)."""
    idx = np.arange(q.shape[0]) if within is None else within
    aband = idx[ab[idx] == 1]
    dec = idx[ab[idx] == 0]
    first = np.unique(np.concatenate([rng.choice(aband, min(n_abandoned, aband.size),
                                                 replace=False),
                                      dec[np.argsort(q[dec])[-n_longest:]]]))
    rest = np.setdiff1d(idx, first)
    return np.unique(np.concatenate([first,
                                     rng.choice(rest, min(n_random, rest.size), replace=False)]))


def test_config3_full_size_sampled(orbg):
    """CA-Polar(128,94), 4 x 100,000 blocks at 3..6 dB, cap 1e6 (64-bit
    syndromes, heavy abandonment), one batched launch: 2,000 blocks or more
    against the oracle -- 400 the GPU abandoned, the 300 longest decoded
    searches (deep in the CTA phase) and 1,300 seeded random ones -- or
    every block when oracle.cache holds this configuration."""
    import oracle_pool
    from oracle import cache
    code, llr, _ = workloads.config3_inputs()
    c = orbg.Code(code.H, max_query_cap=10 ** 6)
    got = gpu_batched(orbg, orbg.CodeSet([c]), llr, 10 ** 6)
    full = cache.load(3)
    if full is not None:
        assert_same(got, (full["cw"].reshape(llr.shape), full["q"], full["ab"]))
    pick = _stratified_pick(got[1], got[2], np.random.default_rng(3), 400, 300, 1300)
    assert pick.size >= 1900 and (got[2][pick] == 1).sum() >= 300
    want = oracle_pool.decode_batch(code.H, llr[pick], 10 ** 6)[:3]
    assert_same(got, want, pick)


def test_config4_full_size(orbg):
    """The benchmark's headline workload in its launch configuration: 1,000,000
    blocks of the four random codes in one batched call (device buffers,
    per-block code ids and offsets), checked per code on 500 or more blocks
    (GPU-abandoned ones, the longest searches, random ones), every decoded
    block a codeword, and every block against oracle.cache when present."""
    import oracle_pool
    from oracle import cache
    codes, cid, llr, off, _, _ = workloads.config4_inputs()
    cs = orbg.CodeSet([orbg.Code(cd.H, max_query_cap=10 ** 6) for cd in codes])
    cw, q, ab = orbg.decode_batched(cs, torch.from_numpy(llr).cuda(), 10 ** 6,
                                    code_id=torch.from_numpy(cid).cuda(),
                                    llr_offset=torch.from_numpy(off).cuda(),
                                    cw_offset=torch.from_numpy(off).cuda(),
                                    n_total=llr.shape[0])
    torch.cuda.synchronize()
    cw, q, ab = cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()
    full = cache.load(4)
    if full is not None:
        assert np.array_equal(cw, full["cw"]) and np.array_equal(q, full["q"].astype(np.int64))
        assert np.array_equal(ab, full["ab"])
    rng = np.random.default_rng(4)
    for j, cd in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        rows = np.stack([cw[off[b]:off[b] + cd.n] for b in idx])
        ok = ab[idx] == 0
        assert not ((rows[ok].astype(np.int64) @ cd.H.T.astype(np.int64)) % 2).any()
        pick = _stratified_pick(q, ab, rng, 100, 100, 400, within=idx)
        assert pick.size >= 500
        blocks = np.stack([llr[off[b]:off[b] + cd.n] for b in pick])
        want = oracle_pool.decode_batch(cd.H, blocks, 10 ** 6)[:3]
        assert_same((np.stack([cw[off[b]:off[b] + cd.n] for b in pick]), q[pick], ab[pick]),
                    want)


@pytest.mark.parametrize("tuning", [(8, 0, 8, 1, 16), (4, 0, 1, 64, 4), (16, 0, 32, 4096, 1),
                                    (2, 1, 3, 100, 7), (8, 0, 8, 10 ** 6, 16)],
                         ids=lambda t: "wpc%d_cps%d_grab%d_budget%d_hw%d" % t)
def test_batched_tuning_does_not_change_results(orbg, tuning):
    """Phase-1 budget down to one group (nearly every block goes to the CTA
    phase), one to sixteen warps per open block, any grab size: the batched
    form still returns the oracle's first hit, abandons included."""
    code = workloads.rlc(64, 44, 61)
    llr, _ = workloads.awgn_llr(code, 600, 2.5, 62)
    cap = 100000
    want = oracle.decode_batch(code.H, llr, cap)[:3]
    assert want[2].any() and not want[2].all()  # some blocks abandon
    c = orbg.Code(code.H, max_query_cap=cap)
    cs = orbg.CodeSet([c])
    orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(*tuning))
    assert_same(gpu_batched(orbg, cs, llr, cap), want)



# In basic ORBGRAND's CTA table, phase 1's walk reaches its first group
# needing triple sums past the warp's own table at this query index, whatever
# the code's length (the run layout depends on the order alone).
WARP_TRIPLES_END = 14798


def test_budget_at_or_above_cap_still_runs_phase_2(orbg):
    """A phase-1 walk on the CTA table stops, open, where it needs triple sums
    past the warp's own table, whatever the budget.  With the default budget
    (16384) and a cap between that point and the budget, and with a budget
    far above the cap, the open blocks still reach phase 2: outputs start
    poisoned and equal the oracle's, on device buffers."""
    code = workloads.rlc(64, 44, 61)
    llr, _ = workloads.awgn_llr(code, 4000, 2.5, 63)
    cap = 16000
    want = oracle.decode_batch(code.H, llr, cap)[:3]
    assert (want[1].astype(np.int64) > WARP_TRIPLES_END).sum() >= 10
    c = orbg.Code(code.H, max_query_cap=10 ** 5)
    for tuning in (None, (8, 0, 4, 16384, 8), (8, 0, 4, 10 ** 6, 4)):
        cs = orbg.CodeSet([c])
        if tuning is not None:
            orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(*tuning))
        assert_same(gpu_batched(orbg, cs, llr, cap), want)


def test_budget_above_cap_host_buffers(orbg):
    """The chunked host-buffer path with a budget above the cap: its phase 2
    over every chunk's open blocks still runs.  Host outputs start poisoned;
    they equal the device-buffer call, and the oracle on every block past the
    warp's own triple table."""
    code = workloads.rlc(64, 44, 61)
    llr, _ = workloads.awgn_llr(code, 140000, 3.5, 64)
    B, n = llr.shape
    cap = 16000
    c = orbg.Code(code.H, max_query_cap=10 ** 5)
    cs = orbg.CodeSet([c])
    orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 4, 10 ** 6, 4))
    dev = gpu_batched(orbg, cs, llr, cap)
    cw = np.full((B, n), 0xFF, np.uint8)
    q = np.full(B, 0xFFFFFFFF, np.uint32)
    ab = np.full(B, 0xFF, np.uint8)
    orbg.orbg_decode_batched(cs.handle, None, None, llr, B, cap, cw, None, q, ab)
    assert_same((cw, q.astype(np.int64), ab), dev)
    far = np.nonzero(dev[1] > WARP_TRIPLES_END)[0]
    assert far.size >= 10
    want = oracle.decode_batch(code.H, llr[far], cap)[:3]
    assert_same((cw[far], q[far].astype(np.int64), ab[far]), want)


def test_mixed_codes_phase2(orbg):
    """Mixed n and n-k in one batched call with a small phase-1 budget, so
    the CTA phase sees blocks of every code."""
    codes, cid, llr, off, cwt, ebn0 = workloads.config4_inputs(B=3000, seed=4402)
    objs = [orbg.Code(cd.H, max_query_cap=2 * 10 ** 5) for cd in codes]
    cs = orbg.CodeSet(objs)
    orbg.orbg_codeset_set_tuning(cs.handle, orbg.OrbgTuning(8, 0, 4, 32, 8))
    llr_t = torch.from_numpy(llr).cuda()
    off_t = torch.from_numpy(off).cuda()
    cid_t = torch.from_numpy(cid).cuda()
    cw, q, ab = orbg.decode_batched(cs, llr_t, 2 * 10 ** 5, code_id=cid_t, llr_offset=off_t,
                                    cw_offset=off_t, n_total=llr.shape[0])
    torch.cuda.synchronize()
    cw, q, ab = cw.cpu().numpy(), q.cpu().numpy().astype(np.int64), ab.cpu().numpy()
    rng = np.random.default_rng(6)
    for j, cd in enumerate(codes):
        idx = np.nonzero(cid == j)[0]
        pick = np.sort(rng.choice(idx, size=min(60, idx.shape[0]), replace=False))
        blocks = np.stack([llr[off[b]:off[b] + cd.n] for b in pick])
        want = oracle.decode_batch(cd.H, blocks, 2 * 10 ** 5)[:3]
        got = (np.stack([cw[off[b]:off[b] + cd.n] for b in pick]), q[pick], ab[pick])
        assert_same(got, want)
