"""Pins of the threshold count-map oracle (pixels strictly above a threshold
per window, the cluster-calling analysis of the paper's stated future work,
Section V), checked against things other than itself: numpy's sliding
window views over the boolean image, closed forms at extreme thresholds,
monotonicity in the threshold, the exact rational fraction, and the
closed-form std of a Bernoulli window sqrt(p (1 - p))."""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(77)


def np_counts(img, thr, wh, ww, sy, sx):
    v = np.lib.stride_tricks.sliding_window_view(img > thr, (wh, ww))[::sy, ::sx]
    return v.sum(axis=(2, 3)).astype(np.uint64)


@pytest.mark.parametrize("dtype,hi", [(np.uint8, 256), (np.uint16, 65536)])
@pytest.mark.parametrize("wh,ww,sy,sx", [(1, 1, 1, 1), (3, 5, 1, 2), (8, 8, 3, 3), (17, 4, 2, 5)])
def test_counts_equal_numpy_window_views(dtype, hi, wh, ww, sy, sx):
    img = RNG.integers(0, hi, size=(41, 53)).astype(dtype)
    for thr in (0, hi // 3, hi // 2, hi - 2):
        got = oracle.count_brute(img, thr, wh, ww, sy, sx)["sum"]
        np.testing.assert_array_equal(got, np_counts(img, thr, wh, ww, sy, sx))


def test_table_path_equals_definition():
    img = RNG.integers(0, 256, size=(37, 29)).astype(np.uint8)
    wins = [(4, 4, 1, 1), (9, 2, 2, 3), (37, 29, 1, 1)]
    for thr in (10, 127, 254):
        viat = oracle.count_sat(img, thr, wins)
        for (wh, ww, sy, sx), t in zip(wins, viat):
            d = oracle.count_brute(img, thr, wh, ww, sy, sx)
            for k in ("sum", "mean", "std"):
                np.testing.assert_array_equal(t[k], d[k])


def test_extreme_thresholds():
    img = RNG.integers(1, 200, size=(20, 30)).astype(np.uint8)
    none = oracle.count_brute(img, 255, 6, 7)
    assert (none["sum"] == 0).all() and (none["mean"] == 0).all() and (none["std"] == 0).all()
    allp = oracle.count_brute(img, 0, 6, 7)
    assert (allp["sum"] == 42).all() and (allp["mean"] == 1.0).all() and (allp["std"] == 0).all()


def test_monotone_in_threshold():
    img = RNG.integers(0, 65536, size=(25, 25)).astype(np.uint16)
    prev = None
    for thr in range(0, 65536, 4096):
        c = oracle.count_brute(img, thr, 5, 5)["sum"].astype(np.int64)
        if prev is not None:
            assert (c <= prev).all()
        prev = c


def test_fraction_and_std_closed_forms():
    img = RNG.integers(0, 256, size=(24, 31)).astype(np.uint8)
    wh, ww = 6, 5
    n = wh * ww
    r = oracle.count_brute(img, 100, wh, ww)
    for c, m, s in zip(r["sum"].ravel(), r["mean"].ravel(), r["std"].ravel()):
        c = int(c)
        assert m == float(Fraction(c, n))                  # correctly rounded c / n
        p = c / n
        want = math.sqrt(p * (1 - p))
        assert abs(s - want) <= 4 * math.ulp(max(want, 1e-300)), (c, s, want)
