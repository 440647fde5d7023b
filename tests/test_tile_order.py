"""The single-pass build's ticket-to-tile mapping along anti-diagonals
(tile_order.cuh), built for the host: a bijection from tickets onto tiles in
which every tile's neighbours above and to the left come first, the
property the decoupled look-back needs (a warp only waits for tiles whose
tickets were taken before its own), on grids from 1 x 1 to the 70,000 x
85,000 image's 1,094 x 333 tiles (CPU only)."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(), "tile_order_host.so")
    subprocess.check_call([
        "g++", "-O2", "-std=c++17", "-fPIC", "-shared",
        "-I", os.path.join(ROOT, "paper_2410_16291_gb300", "csrc"),
        os.path.join(ROOT, "tests", "tile_order_host.cpp"), "-o", out])
    L = ctypes.CDLL(out)
    L.tile_of.argtypes = [ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64]
    L.tile_of.restype = ctypes.c_uint32
    L.check_grid.argtypes = [ctypes.c_int64, ctypes.c_int64]
    L.check_grid.restype = ctypes.c_int64
    return L


def test_small_grids_exhaustive(lib):
    for R in range(1, 40):
        for C in range(1, 40):
            assert lib.check_grid(R, C) == 0, (R, C)


@pytest.mark.parametrize("R,C", [(1094, 333), (333, 1094), (625, 157), (1250, 157),
                                 (192, 128), (1, 5000), (5000, 1), (2187, 41)])
def test_large_grids(lib, R, C):
    assert lib.check_grid(R, C) == 0


def test_first_tickets_walk_the_first_diagonals(lib):
    # 4 x 3 grid: diagonals {0}, {1, 3}, {2, 4, 6}, {5, 7, 9}, {8, 10}, {11}
    # (row-major indices), b ascending along each.
    got = [lib.tile_of(k, 4, 3) for k in range(12)]
    assert got == [0, 1, 3, 2, 4, 6, 5, 7, 9, 8, 10, 11]
