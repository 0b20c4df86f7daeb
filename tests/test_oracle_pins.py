"""The CPU oracle against the paper's examples, closed forms, brute force
and invariants (no GPU)."""
import numpy as np
import pytest

import oracle
import oracle_pins
from paper_2202_13951_gb300 import workloads


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("pin", oracle_pins.FAST_PINS, ids=lambda p: p.__name__)
def test_pin(orc, pin):
    pin(orc)


def test_cumulative_counts(orc):
    oracle_pins.pin_cumulative_counts(orc)


def test_pure_noise_mean_queries(orc):
    """Sec. I: on pure noise every GRAND variant stops at an erroneous
    code-book member after about 2^(n-k) queries on average (a statistical
    check, not parity)."""
    code = workloads.rlc(24, 16, seed=21)
    rng = np.random.default_rng(22)
    llr = rng.normal(0.0, 1.0, (3000, code.n)).astype(np.float32)
    _, q, ab, _ = orc.decode_batch(code.H, llr, 1 << 20)
    assert not ab.any()
    mean = float(q.mean())
    assert abs(mean - 2 ** code.r) / 2 ** code.r < 0.1, mean


def test_nan_rejected(orc):
    code = workloads.hamming74()
    llr = np.ones(7, np.float32)
    llr[3] = np.nan
    with pytest.raises(oracle.OracleError):
        orc.decode(code.H, llr, 10)


def test_sort_ties_and_zero(orc):
    """Sec. III-A sort, with this library's tie reading: equal |LLR| keep the
    received order, -0 and +0 are equal, +inf is most reliable."""
    llr = np.array([2.0, -0.0, 1.0, -2.0, 0.0, np.inf, -1.0, -np.inf],
                   np.float32)
    pi = orc.sort_reliability(llr)
    assert list(pi) == [1, 4, 2, 6, 0, 3, 5, 7]
