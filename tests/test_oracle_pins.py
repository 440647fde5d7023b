"""Pins of the CPU oracle to things other than itself (CPU only).

Each check ties an oracle function to what the paper and the mathematics fix:
numpy's cumulative sums and window views (library routines for the special
case the definition reduces to), closed forms, invariants, exact rational
values and brute force on tiny inputs.  A dropped term, a wrong sign or index
or a transposed operand anywhere in the oracle fails one of them.
"""
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import golden_util
import oracle
import synth

RNG = np.random.default_rng(12345)


def rand_img(r, c, dtype, hi=None, pitch_pad=0):
    hi = hi if hi is not None else (256 if dtype == np.uint8 else 65536)
    base = RNG.integers(0, hi, size=(r, c + pitch_pad), dtype=np.int64).astype(dtype)
    return base[:, :c]          # a view whose row pitch exceeds its width


# ---------------------------------------------------------------- tables --

@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (13, 1), (7, 9), (33, 64), (64, 31)])
def test_sat_equals_numpy_double_cumsum(dtype, shape):
    """Section II-B: S[y][x] = sum_{i<=y, j<=x} I[i][j]; numpy's cumsum along
    both axes is that definition's library routine."""
    img = rand_img(*shape, dtype, pitch_pad=3)
    S, Q = oracle.sat(img)
    a = img.astype(np.uint64)
    np.testing.assert_array_equal(S, a.cumsum(0).cumsum(1))
    np.testing.assert_array_equal(Q, (a * a).cumsum(0).cumsum(1))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_sat_recurrence_and_total(dtype):
    """The inclusion-exclusion recurrence holds everywhere and the last entry
    equals the flat-loop total (and numpy's sum)."""
    img = rand_img(41, 57, dtype)
    S, Q = oracle.sat(img)
    a = img.astype(np.uint64)
    P = np.zeros((42, 58), np.uint64)
    P[1:, 1:] = S
    rec = P[1:, 1:] - P[:-1, 1:] - P[1:, :-1] + P[:-1, :-1]
    np.testing.assert_array_equal(rec, a)
    s, q = oracle.total(img)
    assert S[-1, -1] == s == int(a.sum())
    assert Q[-1, -1] == q == int((a * a).sum())


def test_sat_hand_worked():
    """The hand-worked tables of tests/golden/hand_worked.txt (Section II-B's
    inclusive table), for both pixel types."""
    for case in golden_util.load_cases():
        if "S" not in case:
            continue
        for dt in (np.uint8, np.uint16):
            S, Q = oracle.sat(case["image"].astype(dt))
            np.testing.assert_array_equal(S, case["S"])
            np.testing.assert_array_equal(Q, case["Q"])


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_sat_rows_streamed_equals_full(dtype):
    img = rand_img(50, 70, dtype)
    S, Q = oracle.sat(img)
    want = [0, 1, 17, 48, 49]
    Sr, Qr = oracle.sat_rows(img, want)
    np.testing.assert_array_equal(Sr, S[want])
    np.testing.assert_array_equal(Qr, Q[want])


def test_sat_all_max_u16_bound_invariants():
    """All-65535 image: S_last = r c 65535 and Q_last = r c 65535^2 exactly."""
    img = np.full((300, 200), 65535, np.uint16)
    S, Q = oracle.sat(img)
    assert int(S[-1, -1]) == 300 * 200 * 65535
    assert int(Q[-1, -1]) == 300 * 200 * 65535 ** 2
    assert int(S[9, 19]) == 10 * 20 * 65535


def test_fits_u64_edges():
    """Worst-case bound: S needs r c max < 2^64, Q needs r c max^2 < 2^64.
    4295098371 = 7809 * 550019 px is the largest u16 image whose Q fits;
    4295098372 = 184252 * 23311 px is the smallest that does not."""
    assert 7809 * 550019 * 65535 ** 2 < 2 ** 64 <= 184252 * 23311 * 65535 ** 2
    assert oracle.fits_u64(7809, 550019, "u16", True)
    assert not oracle.fits_u64(184252, 23311, "u16", True)
    assert oracle.fits_u64(184252, 23311, "u16", False)
    # u8 S-only bound: 72340172838076673 = (2^64 - 1) // 255 = 164737 * 439125228929
    assert oracle.fits_u64(257 * 641, 65537 * 6700417, "u8", False)
    assert not oracle.fits_u64(1 << 28, 1 << 28, "u8", True)
    assert oracle.fits_u64(70000, 85000, "u8", True)
    assert not oracle.fits_u64(70000, 85000, "u16", True)


# --------------------------------------------------------------- windows --

def numpy_window_sums(img, wh, ww, sy, sx):
    v = np.lib.stride_tricks.sliding_window_view(img.astype(np.uint64), (wh, ww))
    return v.sum(axis=(2, 3))[::sy, ::sx]


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_brute_sum_equals_numpy_window_view(dtype):
    """Naive SWA (Section II-A) against numpy's window view, every window
    shape and stride on a small image."""
    img = rand_img(11, 13, dtype)
    for wh in range(1, 12):
        for ww in range(1, 14, 3):
            for sy, sx in [(1, 1), (2, 3), (4, 1), (5, 7)]:
                got = oracle.window_brute(img, wh, ww, sy, sx, outputs=("sum",))["sum"]
                np.testing.assert_array_equal(got, numpy_window_sums(img, wh, ww, sy, sx))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape", [(9, 9), (16, 23), (31, 20)])
def test_three_window_algorithms_agree_bitwise(dtype, shape):
    """Naive, integral-image and DP sliding SWA give the same sums, and the
    same mean and std bit for bit, for every window and stride."""
    img = rand_img(*shape, dtype)
    S, Q = oracle.sat(img)
    r, c = shape
    for wh in (1, 2, 3, 5, r):
        for ww in (1, 4, 7, c):
            for sy, sx in [(1, 1), (3, 2), (2, 5)]:
                a = oracle.window_brute(img, wh, ww, sy, sx)
                b = oracle.window_sat(S, Q, wh, ww, sy, sx)
                d = oracle.window_sliding(img, wh, ww, sy, sx)
                for k in ("sum", "mean", "std"):
                    np.testing.assert_array_equal(a[k], b[k])
                    np.testing.assert_array_equal(a[k], d[k])


def test_window_shape_rule():
    """Section III-A counts (r - w + 1)(c - w + 1) valid windows at stride 1."""
    assert oracle.window_shape(1024, 1024, 32, 32, 1, 1) == (993, 993)
    assert oracle.window_shape(20000, 20000, 200, 200, 1, 1) == (19801, 19801)
    assert oracle.window_shape(70000, 85000, 256, 256, 16, 16) == (4360, 5297)
    assert oracle.window_shape(70000, 85000, 1024, 1024, 16, 16) == (4312, 5249)
    assert oracle.window_shape(5, 5, 5, 5, 3, 3) == (1, 1)
    with pytest.raises(ValueError):
        oracle.window_shape(5, 5, 6, 1, 1, 1)
    with pytest.raises(ValueError):
        oracle.window_shape(5, 5, 2, 2, 0, 1)


def test_windows_hand_worked():
    """Every window of tests/golden/hand_worked.txt through the three window
    algorithms: sums exact, means the correctly rounded quotient, stds within
    2 ulp of the exact root (Section II-A's average and standard deviation)."""
    for case in golden_util.load_cases():
        img = case["image"].astype(np.uint8)
        S, Q = oracle.sat(img)
        for w in case["windows"]:
            wh, ww, sy, sx = w["shape"]
            R, C = oracle.window_shape(*img.shape, wh, ww, sy, sx)
            s, m, d = golden_util.expected(w, R, C)
            for out in (oracle.window_brute(img, wh, ww, sy, sx),
                        oracle.window_sat(S, Q, wh, ww, sy, sx),
                        oracle.window_sliding(img, wh, ww, sy, sx)):
                np.testing.assert_array_equal(out["sum"], s)
                np.testing.assert_array_equal(out["mean"], m)
                assert (np.abs(out["std"] - d) <= 2 * np.spacing(d)).all(), (case["name"], w)


def test_closed_forms():
    ones = np.ones((40, 50), np.uint8)
    out = oracle.window_brute(ones, 7, 9, 1, 1)
    assert (out["sum"] == 63).all() and (out["mean"] == 1.0).all() and (out["std"] == 0).all()
    const = np.full((30, 30), 37, np.uint16)
    out = oracle.window_sliding(const, 5, 6, 2, 1)
    assert (out["sum"] == 37 * 30).all() and (out["mean"] == 37.0).all()
    assert (out["std"] == 0.0).all()
    # full-image window = total
    img = rand_img(23, 29, np.uint16)
    s, q = oracle.total(img)
    full = oracle.window_brute(img, 23, 29)
    assert full["sum"].shape == (1, 1) and int(full["sum"][0, 0]) == s
    # checkerboard {0, a}, even window: sum a w^2/2, mean a/2, std a/2
    a = 200
    cb = ((np.indices((24, 24)).sum(0) % 2) * a).astype(np.uint8)
    for w in (2, 4, 6, 8):
        out = oracle.window_sat(*oracle.sat(cb), w, w, 1, 1)
        assert (out["sum"] == a * w * w // 2).all()
        assert (out["mean"] == a / 2).all() and (out["std"] == a / 2).all()
    # impulse at (p, q): 1 in the windows covering it, 0 elsewhere
    imp = np.zeros((20, 25), np.uint8)
    imp[7, 11] = 1
    sums = oracle.window_brute(imp, 4, 5, 1, 1, outputs=("sum",))["sum"]
    ii, jj = np.indices(sums.shape)
    cover = (ii <= 7) & (7 <= ii + 3) & (jj <= 11) & (11 <= jj + 4)
    np.testing.assert_array_equal(sums, cover.astype(np.uint64))


def exact_std(vals):
    """Exact population std of integers, as a Decimal at 60 digits."""
    getcontext().prec = 60
    n = len(vals)
    s = sum(vals)
    q = sum(v * v for v in vals)
    D = n * q - s * s
    return Decimal(D).sqrt() / Decimal(n)


def ulp(x):
    return math.ulp(x) if x else 5e-324


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_std_within_two_ulp_of_exact(dtype):
    """std = sqrt((double)D)/n, D exact: at most two rounding errors from the
    exact population standard deviation (and mean correctly rounded)."""
    img = rand_img(12, 12, dtype)
    for wh, ww in [(1, 2), (3, 3), (5, 4), (12, 12)]:
        out = oracle.window_brute(img, wh, ww, 1, 1)
        for i in range(out["std"].shape[0]):
            for j in range(out["std"].shape[1]):
                vals = [int(v) for v in img[i:i + wh, j:j + ww].ravel()]
                ex = exact_std(vals)
                got = out["std"][i, j]
                assert abs(Decimal(got) - ex) <= 2 * Decimal(ulp(float(ex)))
                assert out["mean"][i, j] == float(Fraction(sum(vals), len(vals)))
                assert int(out["sum"][i, j]) == sum(vals)


def test_std_two_valued_closed_form():
    """A window with k pixels of value a and n-k of value b has population
    std |a - b| sqrt(p (1 - p)), p = k/n."""
    a, b = 3000, 60000
    for n, k in [(4, 1), (16, 5), (64, 32), (100, 7)]:
        img = np.full((1, n), b, np.uint16)
        img[0, :k] = a
        _, _, m, s = oracle.window_one(img, 0, 0, 1, n)
        p = k / n
        assert math.isclose(s, abs(a - b) * math.sqrt(p * (1 - p)), rel_tol=1e-15)
        assert m == float(Fraction(k * a + (n - k) * b, n))


def test_u128_to_double_round_to_nearest_even():
    """Python's int -> float conversion is correctly rounded (ties to even)."""
    vals = [0, 1, 2**53 - 1, 2**53, 2**53 + 1, 2**53 + 2, 2**53 + 3, 2**64 - 1, 2**64,
            2**64 + 1, 2**64 + 2**11, 2**64 + 2**12, 2**64 + 3 * 2**11, 2**100 + 2**47,
            2**100 + 2**47 + 1, 2**127, 2**128 - 1]
    rng = np.random.default_rng(7)
    for _ in range(2000):
        bits = int(rng.integers(1, 128))
        vals.append(int(rng.integers(0, 2**63)) << max(0, bits - 63) | int(rng.integers(0, 2**20)))
    for v in vals:
        v &= 2**128 - 1
        assert oracle.u128_to_double(v) == float(v), v


def test_sliding_matches_brute_on_cfg0_crop():
    """The three window algorithms on a crop of the cell-centroid mask."""
    img = synth.mask_u8(1024, 1024, synth.DEFAULT_SEED)[:200, :300]
    a = oracle.window_brute(img, 32, 32, 1, 1, outputs=("sum",))["sum"]
    b = oracle.window_sliding(img, 32, 32, 1, 1, outputs=("sum",))["sum"]
    c = oracle.window_sat(oracle.sat(img, with_sq=False)[0], None, 32, 32, 1, 1,
                          outputs=("sum",))["sum"]
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(a, numpy_window_sums(img, 32, 32, 1, 1))


def test_window_sat_rows_equals_full():
    img = rand_img(40, 33, np.uint16)
    S, Q = oracle.sat(img)
    full = oracle.window_sat(S, Q, 6, 5, 2, 3)
    rows = [0, 3, full["sum"].shape[0] - 1]
    part = oracle.window_sat_rows(S, Q, 6, 5, 2, 3, rows)
    for k in ("sum", "mean", "std"):
        np.testing.assert_array_equal(part[k], full[k][rows])


def test_window_rows_stream_equals_the_definition():
    """The streamed-rows oracle (only the table rows the corners lie on are
    kept) against the naive definition, on random subsets of output rows of
    ragged images: windows as tall as the image, strides larger than the
    window, first and last rows, both pixel types."""
    rng = np.random.default_rng(404)
    for it in range(300):
        r, c = (int(v) for v in rng.integers(1, 48, 2))
        dt = np.uint8 if it % 2 else np.uint16
        img = rng.integers(0, 256 if dt == np.uint8 else 65536, (r, c)).astype(dt)
        wh = int(rng.integers(1, r + 1)) if it % 7 else r
        ww = int(rng.integers(1, c + 1))
        sy, sx = (int(v) for v in rng.integers(1, 9, 2))
        R, C = oracle.window_shape(r, c, wh, ww, sy, sx)
        rows = sorted(set([0, R - 1] + rng.integers(0, R, int(rng.integers(0, R + 1))).tolist()))
        got = oracle.window_rows_stream(img, wh, ww, sy, sx, rows)
        want = oracle.window_brute(img, wh, ww, sy, sx)
        for k in ("sum", "mean", "std"):
            np.testing.assert_array_equal(got[k], want[k][rows], err_msg="%d %s" % (it, k))
    # sum only (no squared table is formed) and argument checks
    img = rng.integers(0, 256, (30, 40)).astype(np.uint8)
    got = oracle.window_rows_stream(img, 5, 6, 2, 3, [1, 4], outputs=("sum",))
    np.testing.assert_array_equal(got["sum"], oracle.window_brute(img, 5, 6, 2, 3)["sum"][[1, 4]])
    with pytest.raises(ValueError):
        oracle.window_rows_stream(img, 5, 6, 2, 3, [4, 1])
    with pytest.raises(ValueError):
        oracle.window_rows_stream(img, 5, 6, 2, 3, [13])          # R = 13 rows: 0..12


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_parallel_variants_equal_the_serial_oracle(threads):
    """The row-band parallel table build and the row-split window pass give
    the serial oracle's tables and outputs exactly, for band counts that do
    and do not divide the rows (including more bands than rows)."""
    rng = np.random.default_rng(505 + threads)
    oracle.par_threads(threads)
    try:
        for (r, c), dt in [((1, 1), np.uint8), ((2, 9), np.uint16), ((7, 13), np.uint8),
                           ((64, 33), np.uint16), ((301, 257), np.uint8),
                           ((1000, 77), np.uint16)]:
            img = rng.integers(0, 256 if dt == np.uint8 else 65536, (r, c)).astype(dt)
            S, Q = oracle.sat(img)
            Sp, Qp = oracle.sat_par(img)
            np.testing.assert_array_equal(Sp, S)
            np.testing.assert_array_equal(Qp, Q)
            Sp1, none = oracle.sat_par(img, with_sq=False)
            assert none is None
            np.testing.assert_array_equal(Sp1, S)
            for wh, ww, sy, sx in [(1, 1, 1, 1), (r, c, 1, 1), (max(1, r // 2), max(1, c // 3), 2, 3)]:
                want = oracle.window_sat(S, Q, wh, ww, sy, sx)
                got = oracle.window_sat_par(S, Q, wh, ww, sy, sx)
                for k in want:
                    np.testing.assert_array_equal(got[k], want[k])
    finally:
        oracle.par_threads(os.cpu_count() or 1)
