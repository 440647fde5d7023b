"""Threshold count tables (swa_build_count_sat) against the oracle: the
table equals the summed-area table of the 0/1 indicator "pixel > thr", and
window statistics on it equal, bit for bit, the oracle's count map by the
definition (count, fraction, indicator std) -- for both dtypes, thresholds
at and beyond the pixel range, rectangular windows and strides, and
unaligned, pitched images."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2410_16291_gb300 as swa
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(4242)
WINDOWS = [(1, 1, 1, 1), (5, 7, 1, 1), (16, 16, 3, 2), (40, 9, 2, 5)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    from paper_2410_16291_gb300 import build
    build.build()


def _check(img, thr, dev, windows, brute):
    sat = swa.build_count_sat(dev, thr)
    S, Q = sat.tables()
    ind = (img > thr).astype(np.uint8)
    S_ref, _ = oracle.sat(ind, with_sq=False)
    np.testing.assert_array_equal(u64(S), S_ref)
    res = sat.window_stats(windows)
    want = ([oracle.count_brute(img, thr, *w) for w in windows] if brute
            else oracle.count_sat(img, thr, windows))
    for w, got, ref in zip(windows, res, want):
        np.testing.assert_array_equal(u64(got["sum"]), ref["sum"], err_msg=str(w))
        np.testing.assert_array_equal(f64(got["mean"]), ref["mean"], err_msg=str(w))
        np.testing.assert_array_equal(f64(got["std"]), ref["std"], err_msg=str(w))
    sat.free()


@pytest.mark.parametrize("dtype,hi", [(np.uint8, 256), (np.uint16, 65536)])
def test_count_maps_by_definition(dtype, hi):
    img = RNG.integers(0, hi, size=(61, 83)).astype(dtype)
    for thr in (0, hi // 4, hi // 2, hi - 1, hi + 5):
        _check(img, thr, to_device(img), WINDOWS, brute=True)


@pytest.mark.parametrize("dtype,hi", [(np.uint8, 256), (np.uint16, 65536)])
@pytest.mark.parametrize("pad,offset", [(0, 0), (3, 1), (5, 3)])
def test_count_maps_larger_and_unaligned(dtype, hi, pad, offset):
    img = RNG.integers(0, hi, size=(300, 517)).astype(dtype)
    _check(img, hi // 3, to_device(img, pad_cols=pad, offset_px=offset),
           WINDOWS + [(64, 64, 8, 8), (300, 517, 1, 1)], brute=False)


def test_count_handle_aliases_q_and_reports_count():
    img = RNG.integers(0, 256, size=(40, 50)).astype(np.uint8)
    sat = swa.build_count_sat(to_device(img), 100)
    S, Q = ctypes.c_void_p(), ctypes.c_void_p()
    ld = ctypes.c_int64()
    swa.check(swa.lib().swa_sat_data(sat.handle, ctypes.byref(S), ctypes.byref(Q),
                                     ctypes.byref(ld)), "swa_sat_data")
    assert S.value == Q.value
    fl = ctypes.c_uint32()
    swa.check(swa.lib().swa_sat_info(sat.handle, None, None, None, ctypes.byref(fl)),
              "swa_sat_info")
    assert fl.value == swa.SWA_WITH_SQ | swa.SWA_COUNT
    sat.free()
