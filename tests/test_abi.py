"""The C-ABI library builds, loads and exports every symbol include/orbg.h
declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2202_13951_gb300 import build, orbg, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "orbg.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return orbg.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(orbg_\w+)\s*\(", src)))


def test_header_compiles_as_c_and_cxx():
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        subprocess.check_call(["gcc", "-x", lang, std, "-fsyntax-only", "-Wall",
                               "-Werror", HEADER])


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    for s in range(-7, 1):
        assert orbg.orbg_status_string(s) not in ("", "unknown status")
    assert orbg.orbg_status_string(-99) == "unknown status"
    assert orbg.orbg_version() == 200


def test_tuning_argument_checks(lib):
    t = orbg.OrbgTuning(8, 0, 8, 4096, 16)
    assert lib.orbg_codeset_set_tuning(None, ctypes.byref(t)) == orbg.ORBG_EINVAL
    assert lib.orbg_codeset_get_tuning(None, ctypes.byref(t)) == orbg.ORBG_EINVAL


def test_load_code_rejects_bad_input_before_any_cuda_call(lib):
    H = workloads.hamming74().H
    cases = [
        (H, 7, 7, 4, orbg.ORBG_EINVAL),          # kind
        (H, orbg.ORBG_MAT_H, 0, 0, orbg.ORBG_EINVAL),
        (H, orbg.ORBG_MAT_H, 7, 7, orbg.ORBG_EINVAL),  # k >= n
        (np.full_like(H, 2), orbg.ORBG_MAT_H, 7, 4, orbg.ORBG_EINVAL),
        (np.zeros((3, 300), np.uint8), orbg.ORBG_MAT_H, 300, 297, orbg.ORBG_ELIMIT),
        (np.zeros((129, 200), np.uint8), orbg.ORBG_MAT_H, 200, 71, orbg.ORBG_ELIMIT),
        (np.vstack([H[:2], H[:1]]), orbg.ORBG_MAT_H, 7, 4, orbg.ORBG_ERANK),
    ]
    for mat, kind, n, k, want in cases:
        with pytest.raises(orbg.OrbgError) as ei:
            orbg.orbg_load_code(mat, kind, n, k)
        assert ei.value.status == want, (kind, n, k)
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_load_code(H, orbg.ORBG_MAT_H, 7, 4, orbg.ORBG_MAX_QUERY_CAP + 1)
    assert ei.value.status == orbg.ORBG_ELIMIT
    # null output pointer
    rc = lib.orbg_load_code(H.ctypes.data, 0, 7, 4, 0, None)
    assert rc == orbg.ORBG_EINVAL


def test_decode_argument_checks_without_gpu(lib):
    # NULL code handle and negative sizes fail before any CUDA call
    assert lib.orbg_decode(None, None, 1, 10, None, None, None, None) == orbg.ORBG_EINVAL
    assert lib.orbg_decode_batched(None, None, None, None, 1, 10, None, None, None, None,
                                   None) == orbg.ORBG_EINVAL
    assert lib.orbg_code_info(None, None, None, None, None) == orbg.ORBG_EINVAL
    assert lib.orbg_free_code(None) == orbg.ORBG_OK
    assert lib.orbg_codeset_free(None) == orbg.ORBG_OK
    assert lib.orbg_probe_int_lanes(None) == orbg.ORBG_EINVAL
    assert lib.orbg_probe_smem_bytes(None) == orbg.ORBG_EINVAL
    out = np.zeros((4, 8), np.int32)
    for J0, beta in ((-1, 1), (0, 0), (2000, 1), (0, 2000)):
        assert lib.orbg_query_order_line(7, 4, 0, J0, beta, out.ctypes.data) == orbg.ORBG_EINVAL
        assert lib.orbg_load_code_line(None, 0, 7, 4, 0, J0, beta, None) == orbg.ORBG_EINVAL
    H = np.zeros((3, 7), np.uint8)
    h = ctypes.c_void_p()
    # m-segment models out of range: a position weighing below 0, beta 0,
    # anchors out of order or outside 1..n-1, too many segments
    for m, anchors, J, beta in ((1, [], [-2], [1]), (1, [], [0], [0]), (2, [4], [0, -3], [1, 2]),
                                (2, [0], [0, 0], [1, 1]), (2, [7], [0, 0], [1, 1]),
                                (3, [4, 3], [0, 0, 0], [1, 1, 1]), (9, [1] * 8, [0] * 9, [1] * 9),
                                (0, [], [0], [1]), (1, [], [1 << 21], [1])):
        a = np.array(anchors or [0], np.int32)
        j = np.array(J, np.int32)
        b = np.array(beta, np.int32)
        assert lib.orbg_query_order_model(7, 4, 0, m, a.ctypes.data, j.ctypes.data,
                                          b.ctypes.data, out.ctypes.data) == orbg.ORBG_EINVAL
        assert lib.orbg_load_code_model(H.ctypes.data, 0, 7, 4, 0, m, a.ctypes.data,
                                        j.ctypes.data, b.ctypes.data,
                                        ctypes.byref(h)) == orbg.ORBG_EINVAL
    assert lib.orbg_query_order_model(7, 4, 0, 1, None, None, None,
                                      out.ctypes.data) == orbg.ORBG_EINVAL


@pytest.mark.parametrize("n,count", [(1, 2), (3, 8), (7, 128), (12, 4096),
                                     (16, 65536), (64, 150000), (127, 150000),
                                     (128, 150000), (256, 40000)])
def test_query_order_tables_match_oracle(lib, n, count):
    """Both tables the kernels walk expand to exactly the oracle's order."""
    want = oracle.enumerate_patterns(n, count)
    assert orbg.orbg_query_order(n, count, 0) == want
    assert orbg.orbg_query_order(n, count, 1) == want
    flat = orbg.orbg_query_order(n, count, 2)
    assert len(flat) == min(count, 256) or n <= 10
    assert flat == want[:len(flat)]


def test_query_order_depth_for_cap(lib):
    """Counting the table's patterns per logistic weight at the 1e6 cap depth
    agrees with the oracle's count (W <= 82, n = 128 and 64)."""
    for n in (64, 128):
        cnt = oracle.count_by_weight(n, 82)
        total = int(cnt.sum())
        got = lib.orbg_query_order(n, 0, 0, None)
        assert got == 0
        # the library must cover at least `total` patterns for that cap
        out = np.zeros((1, n + 1), np.int32)
        # last pattern of depth 82 is the (total)-th; its weight must be 82
        rows = orbg.orbg_query_order(n, total)
        assert len(rows) == total
        assert sum(rows[-1]) == 82 and sum(rows[0]) == 0


@pytest.mark.parametrize("n,count", [(3, 8), (7, 128), (12, 4096), (40, 60000), (127, 60000),
                                     (256, 20000)])
@pytest.mark.parametrize("line", [(0, 1), (1, 1), (3, 1), (20, 1), (5, 2), (2, 3)],
                         ids=lambda l: "J%d_b%d" % l)
def test_query_order_line_tables_match_oracle(lib, n, count, line):
    """The one-line tables (Sec. III-D) expand to exactly the one-line
    oracle's order, in all three tables the kernels read."""
    want = oracle.enumerate_patterns_1line(n, count, *line)
    assert orbg.orbg_query_order_line(n, count, 0, *line) == want
    assert orbg.orbg_query_order_line(n, count, 1, *line) == want
    flat = orbg.orbg_query_order_line(n, count, 2, *line)
    assert 0 < len(flat) <= 256
    assert flat == want[:len(flat)]


def _check_model_tables(n, count, model):
    want = oracle.enumerate_patterns_mline(n, count, model)
    assert orbg.orbg_query_order_model(n, count, 0, model) == want
    assert orbg.orbg_query_order_model(n, count, 1, model) == want
    flat = orbg.orbg_query_order_model(n, count, 2, model)
    assert len(flat) <= 256  # empty when the first patterns reach past rank 31
    assert flat == want[:len(flat)]


def test_query_order_model_tables_match_oracle(lib):
    """The m-segment tables (Sec. III-D, Eq. relest_seg) expand to exactly
    the m-segment oracle's order in all three tables the kernels read: the
    whole order for n = 10 under models of one to four segments, zero-weight
    positions included."""
    import oracle_pins
    for model in oracle_pins.MODELS10:
        _check_model_tables(10, 1 << 10, model)


@pytest.mark.parametrize("n,k", [(64, 48), (127, 113), (128, 105), (255, 231)])
def test_query_order_fitted_model_tables_match_oracle(lib, n, k):
    """Models fitted (Sec. III-E) to AWGN blocks at three SNRs, one to four
    lines, both quantisations: the tables expand to the oracle's order."""
    code = workloads.rlc(n, k, seed=n)
    seen = set()
    for snr in (2.0, 4.0, 6.0):
        llr, _ = workloads.awgn_llr(code, 2, snr, seed=int(snr) + n)
        for b in range(llr.shape[0]):
            for lines in (1, 2, 3, 4):
                for div in (False, True):
                    model = oracle.fit(llr[b], lines, div)
                    if model not in seen:
                        seen.add(model)
                        _check_model_tables(n, 20000, model)
    assert len(seen) >= 6


def test_query_order_one_segment_model_is_the_line(lib):
    """One segment with J_0 >= 0 is the one-line order; J_0 = 0, beta = 1
    the basic order (built without triple runs here)."""
    for n in (12, 64, 128):
        for J0, beta in ((0, 1), (3, 1), (5, 2)):
            assert (orbg.orbg_query_order_model(n, 30000, 0, ((), (J0,), (beta,))) ==
                    orbg.orbg_query_order_line(n, 30000, 0, J0, beta))


def test_query_order_model_limit(lib):
    """A model whose order reaches position 256 among a pattern's leading
    positions, which a run stores in a byte, is refused with ELIMIT."""
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_query_order_model(256, 8, 0, ((255,), (1000, 0), (1, 1)))
    assert ei.value.status == orbg.ORBG_ELIMIT


def test_fitted_argument_checks(lib):
    """The per-block one-line fitted decoder refuses NULL objects and codes
    without a GPU call."""
    h = ctypes.c_void_p()
    assert lib.orbg_fitted_create(None, 0, ctypes.byref(h)) == orbg.ORBG_EINVAL
    assert lib.orbg_fitted_create(None, 0, None) == orbg.ORBG_EINVAL
    assert lib.orbg_fitted_free(None) == orbg.ORBG_OK
    assert lib.orbg_fitted_decode(None, None, 1, 10, None, None, None, None,
                                  None) == orbg.ORBG_EINVAL
    assert lib.orbg_fit_models(None, -1, 64, 3, 0, None, None) == orbg.ORBG_EINVAL
    assert lib.orbg_fit_models(None, 4, 64, 0, 0, None, None) == orbg.ORBG_EINVAL
    assert lib.orbg_fit_models(None, 4, 64, 9, 0, None, None) == orbg.ORBG_EINVAL


def test_query_order_model_deep_n256(lib):
    """Deeper m-segment tables at n = 256: 100,000 patterns of models fitted
    (Sec. III-E) to blocks of a [256, 234] code expand to the oracle's order
    in both run tables."""
    code = workloads.rlc(256, 234, seed=61)
    llr, _ = workloads.awgn_llr(code, 2, 5.0, seed=3)
    for b, lines in ((0, 3), (1, 4)):
        model = oracle.fit(llr[b], lines)
        want = oracle.enumerate_patterns_mline(256, 100000, model)
        assert orbg.orbg_query_order_model(256, 100000, 0, model) == want
        assert orbg.orbg_query_order_model(256, 100000, 1, model) == want


def test_large_line_intercept_needs_model_tables(lib):
    """A large J_0 makes the line tables stop at logistic weight 255 before
    the cap (ELIMIT); the one-segment model tables, which the fitted decoder
    falls back to, hold the same order to the cap."""
    with pytest.raises(orbg.OrbgError) as ei:
        orbg.orbg_query_order_line(255, 20000, 0, 202, 1)
    assert ei.value.status == orbg.ORBG_ELIMIT
    model = ((), (202,), (1,))
    want = oracle.enumerate_patterns_mline(255, 20000, model)
    assert orbg.orbg_query_order_model(255, 20000, 0, model) == want


def test_query_order_random_models_match_oracle(lib):
    """Random m-segment models — one to five segments, slopes 1..9, intercepts
    from -beta (a zero-weight first position) up, weights not monotone
    across segments — expand to the oracle's order in all three tables."""
    rng = np.random.default_rng(53)
    for trial in range(30):
        n = int(rng.choice([12, 40, 100]))
        m = int(rng.integers(1, 6))
        anchors = tuple(sorted(rng.choice(np.arange(1, n), size=m - 1, replace=False).tolist()))
        beta = tuple(int(b) for b in rng.integers(1, 10, size=m))
        J = tuple(int(rng.integers(-b, 3 * b + 20)) for b in beta)
        model = (anchors, J, beta)
        count = 4096 if n == 12 else 15000
        _check_model_tables(n, count, model)


def test_model_with_empty_flat_table(lib):
    """A model whose first patterns reach past rank 31 (a second segment of
    light positions far down the order) leaves the flat table empty; its
    run tables still hold the oracle's order (the GPU test decodes with the
    same model shape, covering the kernels' path with no flat table)."""
    for n in (64, 127):
        model = ((n * 5 // 8,), (-4, 0), (9, 4))
        assert orbg.orbg_query_order_model(n, 5000, 2, model) == []
        _check_model_tables(n, 5000, model)


def test_output_poisoning_of_the_decode_helpers(monkeypatch):
    """The binding's decode helpers allocate their outputs through _out:
    with ORBG_POISON_OUTPUTS=1 (which this suite sets) every byte of a fresh
    output holds all-ones bits, a value no decode writes (codeword bytes are
    0 or 1, q >= 1 or 0 for NaN blocks, flags 0-2); without it the tensor is
    only allocated."""
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("ORBG_POISON_OUTPUTS", "1")
    cw = orbg._out((3, 5), torch.uint8, "cpu")
    q = orbg._out((3,), torch.int32, "cpu")
    assert (cw == 255).all() and (q.view(torch.uint8) == 255).all()
    monkeypatch.setenv("ORBG_POISON_OUTPUTS", "0")
    assert orbg._out((2,), torch.uint8, "cpu").shape == (2,)
