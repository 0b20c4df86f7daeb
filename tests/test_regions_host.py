"""The serving loop's pool allocator (orbg_regions.h), built for the host:
seeded random placements and returns against a granule-by-granule model
of the pool -- first fit at the lowest offset, never over a live range,
freed neighbours merged, the whole pool one range again at the end."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_13951_gb300", "csrc")


@pytest.fixture(scope="module")
def regions(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("regions") / "libregions_host.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                           os.path.join(HERE, "regions_host.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.regions_run.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_uint64)]
    lib.regions_run.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("seed,granules,steps", [(1, 64, 4000), (2, 1000, 4000),
                                                 (3, 7, 2000), (4, 4096, 3000),
                                                 (5, 1, 500)])
def test_regions_against_a_granule_model(regions, seed, granules, steps):
    placed = ctypes.c_uint64()
    rc = regions.regions_run(seed, granules, steps, ctypes.byref(placed))
    assert rc == 0, "check %d failed" % rc
    assert placed.value > steps // 4
