"""The device fit's steps (orbg_fit.cuh: anchor search and quantisation of
Sec. III-E), built for the host, against the oracle's fit on the same
curves: the integers must be identical (no GPU needed; the GPU test then
covers the device sort and the launch)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2202_13951_gb300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_13951_gb300", "csrc")


@pytest.fixture(scope="module")
def fit_host(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("fit") / "libfit_host.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
                           "-I", CSRC, os.path.join(HERE, "fit_host.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.fit_host.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.c_void_p]
    lib.fit_host.restype = ctypes.c_int

    def run(llr, lines, divisible=False):
        llr = np.ascontiguousarray(llr, np.float32)
        res = np.zeros(24, np.int32)
        assert lib.fit_host(llr.ctypes.data, llr.shape[0], lines, int(divisible),
                            res.ctypes.data) == 0
        m = int(res[0])
        return (tuple(int(x) for x in res[1:m]), tuple(int(x) for x in res[8:8 + m]),
                tuple(int(x) for x in res[16:16 + m]))
    return run


def _curves():
    rng = np.random.default_rng(43)
    out = []
    for n, k in ((64, 48), (127, 113), (256, 234)):
        code = workloads.rlc(n, k, seed=n)
        for snr in (1.0, 3.0, 5.0, 8.0):
            llr, _ = workloads.awgn_llr(code, 6, snr, seed=int(snr) + n)
            out += list(llr)
    for n in (1, 2, 3, 4, 5, 7, 31, 32, 33, 100, 255, 256):
        out.append(rng.normal(0.0, 2.0, n).astype(np.float32))
        out.append(np.round(rng.normal(0.0, 2.0, n)).astype(np.float32))  # ties, flat runs
    x = rng.normal(0.0, 2.0, 64).astype(np.float32)
    x[:5] = np.inf
    out.append(x)
    out.append(np.full(40, np.inf, np.float32))
    out.append(np.full(40, 1.5, np.float32))
    out.append(np.array([1e-30, 1e-30, 3e-30] + [1e30] * 37, np.float32))
    out.append(np.array([1e-20 * j if j <= 5 else 5e-20 + 1e20 * (j - 5)
                         for j in range(1, 41)], np.float32))  # a ratio beyond 2^24
    return out


def test_fit_steps_match_oracle(fit_host):
    n_fitted = 0
    for llr in _curves():
        for lines in range(1, 9):
            for div in (False, True):
                want = oracle.fit(llr, lines, div)
                assert fit_host(llr, lines, div) == want, (llr.shape[0], lines, div)
                n_fitted += len(want[1]) > 1
    assert n_fitted > 100  # most curves give several segments


def test_fit_steps_parabola_closed_forms(fit_host):
    """The hand-worked closed forms of the oracle's pins hold for the host
    build of the device steps too."""
    import oracle_pins
    rng = np.random.default_rng(3)
    for (n, lines), (plain, div) in oracle_pins.PARABOLA_FITS.items():
        llr = oracle_pins._disguise([j * j for j in range(1, n + 1)], rng)
        assert fit_host(llr, lines) == plain
        assert fit_host(llr, lines, True) == div


def test_bitonic_network_sorts_every_length(fit_host):
    """The kernel's 256-slot bitonic network (orbg_fit.cuh's step, stages in
    the kernel's order) sorts |LLR| ascending for every n = 1..256, with
    ties, zeros and infinities; the host build returns an error otherwise."""
    rng = np.random.default_rng(47)
    for n in range(1, 257):
        x = rng.normal(0.0, 2.0, n).astype(np.float32)
        if n % 3 == 0:
            x = np.round(x)
        if n % 5 == 0:
            x[rng.integers(0, n, 2)] = np.inf
            x[rng.integers(0, n, 1)] = -0.0
        fit_host(x, 1)  # asserts the sort held
