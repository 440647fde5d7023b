"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Summed-area tables and window sums must match bit for bit; mean and std are
formed from the same exact integer moments with correctly rounded IEEE
operations on both sides, so they are compared bit for bit as well (the
contract's bar is 1e-12 relative; a bit mismatch is still reported with its
relative error).
"""
import numpy as np
import pytest

import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12
RNG = np.random.default_rng(2024)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    from paper_2410_16291_gb300 import build
    build.build()
    yield
    import torch
    torch.cuda.synchronize()


def rand_img(r, c, dtype, hi=None):
    hi = hi if hi is not None else (256 if dtype == np.uint8 else 65536)
    return RNG.integers(0, hi, size=(r, c), dtype=np.int64).astype(dtype)


def assert_close_bits(got, want, what):
    """Bit-exact comparison; on failure report the worst relative error."""
    if np.array_equal(got, want):
        return
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    bad = np.argwhere(got != want)
    pytest.fail("%s: %d mismatches, worst rel %.3g at %s (got %r want %r)" % (
        what, len(bad), rel.max(), bad[0], got[tuple(bad[0])], want[tuple(bad[0])]))


def check_tables(sat, img, with_sq=True):
    S_ref, Q_ref = oracle.sat(img, with_sq=with_sq)
    S, Q = sat.tables()
    np.testing.assert_array_equal(u64(S), S_ref)
    if with_sq:
        np.testing.assert_array_equal(u64(Q), Q_ref)
    else:
        assert Q is None
    return S_ref, Q_ref


def check_windows(sat, S_ref, Q_ref, windows, outputs=("sum", "mean", "std")):
    res = sat.window_stats(windows, outputs=outputs)
    for (wh, ww, sy, sx), got in zip(windows, res):
        want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx, outputs=outputs)
        if "sum" in outputs:
            np.testing.assert_array_equal(u64(got["sum"]), want["sum"])
        for k in ("mean", "std"):
            if k in outputs:
                g = f64(got[k])
                assert np.allclose(g, want[k], rtol=REL_TOL, atol=0), k
                assert_close_bits(g, want[k], "%s w=%dx%d s=%dx%d" % (k, wh, ww, sy, sx))


SHAPES = [(1, 1), (1, 300), (300, 1), (7, 9), (128, 256), (129, 257), (255, 511),
          (383, 769), (1000, 1031)]


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("twopass", [False, True])
def test_tables_bitexact(dtype, shape, twopass):
    img = rand_img(*shape, dtype)
    sat = swa.build_sat(to_device(img), with_sq=True, twopass=twopass)
    check_tables(sat, img)
    sat.sync()
    sat.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("pad,offset", [(5, 1), (13, 0), (0, 3), (3, 8), (3, 4)])
@pytest.mark.parametrize("twopass", [False, True])
def test_tables_pitched_and_unaligned(dtype, pad, offset, twopass):
    """Row pitches larger than the width and base addresses that are aligned
    to 8 bytes, 2 bytes or not at all select the vector-load or the
    pixel-by-pixel path; results must not change."""
    img = rand_img(301, 517, dtype)
    dev = to_device(img, pad_cols=pad, offset_px=offset)
    sat = swa.build_sat(dev, with_sq=True, twopass=twopass)
    check_tables(sat, img)
    sat.free()


# Widths whose last column slice (256 pixels) holds 1..17 pixels, and the
# slice before it ending near a 16-byte boundary: the staging copies the
# 16-byte-aligned chunks covering each slice, so the chunks that straddle a
# row's start or end (first, second-to-last and last slices) and the zero
# fill past the row are exercised for every misalignment of the row start.
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("tail", [1, 2, 7, 8, 9, 15, 16, 17])
@pytest.mark.parametrize("pad,offset", [(0, 0), (1, 1), (3, 2), (5, 3), (8, 1)])
@pytest.mark.parametrize("twopass", [False, True])
def test_tables_row_ends_every_alignment(dtype, tail, pad, offset, twopass):
    img = rand_img(67, 2 * 256 + tail, dtype)
    dev = to_device(img, pad_cols=pad, offset_px=offset)
    sat = swa.build_sat(dev, with_sq=True, twopass=twopass)
    check_tables(sat, img)
    sat.free()


# The single pass takes its tiles along anti-diagonals in edge mode by
# default; corner mode (the corner term from the tile above-left) and
# row-major tickets are the alternatives the test hooks select.  All four
# combinations must give the same tables.
HOOKS = {"default": 0, "corner": swa.SWA_HOOK_CORNER_MODE, "row": swa.SWA_HOOK_ROW_ORDER,
         "corner+row": swa.SWA_HOOK_CORNER_MODE | swa.SWA_HOOK_ROW_ORDER}


@pytest.mark.parametrize("with_sq", [True, False], ids=["S+Q", "S"])
@pytest.mark.parametrize("hook", list(HOOKS))
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape,pad,offset", [((129, 32768), 0, 0), ((200, 32775), 3, 1),
                                              ((67, 40000), 0, 0), ((5, 33000), 8, 3),
                                              ((1000, 1031), 0, 2), ((300, 5000), 5, 0)])
def test_tables_lookback_modes(hook, dtype, shape, pad, offset, with_sq):
    """Tables of S and Q, and of S alone (whose uint8 tiles are staged in two
    parts), in all four look-back / ticket-order combinations, on wide,
    short, pitched and unaligned images."""
    img = rand_img(*shape, dtype)
    L = swa.lib()
    assert L.swa_set_test_hooks(HOOKS[hook]) == 0
    try:
        sat = swa.build_sat(to_device(img, pad_cols=pad, offset_px=offset), with_sq=with_sq)
        sat.sync()
    finally:
        L.swa_set_test_hooks(0)
    S_ref, Q_ref = check_tables(sat, img, with_sq=with_sq)
    check_windows(sat, S_ref, Q_ref, [(min(33, shape[0]), 1000, 4, 7), (shape[0], shape[1], 1, 1)],
                  outputs=("sum", "mean", "std") if with_sq else ("sum", "mean"))
    sat.free()


def test_sum_only_table_has_no_q():
    img = rand_img(200, 333, np.uint8)
    sat = swa.build_sat(to_device(img), with_sq=False)
    S_ref, _ = check_tables(sat, img, with_sq=False)
    check_windows(sat, S_ref, None, [(5, 7, 1, 1), (200, 333, 1, 1)], outputs=("sum", "mean"))
    with pytest.raises(swa.SwaError):
        sat.window_stats([(5, 5, 1, 1)], outputs=("std",))
    sat.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_windows_bitexact(dtype):
    img = rand_img(389, 611, dtype)
    sat = swa.build_sat(to_device(img))
    S_ref, Q_ref = check_tables(sat, img)
    windows = [(1, 1, 1, 1), (2, 3, 1, 1), (32, 32, 1, 1), (50, 50, 1, 1), (17, 29, 3, 5),
               (100, 100, 16, 16), (389, 611, 1, 1), (389, 1, 7, 1), (1, 611, 1, 9)]
    check_windows(sat, S_ref, Q_ref, windows)
    sat.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_windows_grouped_sparse_strides(dtype):
    """Sparse-stride queries with equal strides are evaluated in one sweep
    over their union grid, in column panels of 4 blocks: sizes from 1 to the
    whole image, more same-stride queries than one launch holds (21 > 16),
    groups with other strides in the same call, a ragged last panel."""
    img = rand_img(613, 9000, dtype)          # stride 4: 2,250 columns = 8.8 blocks
    sat = swa.build_sat(to_device(img))
    S_ref, Q_ref = check_tables(sat, img)
    windows = [(8, 8, 4, 4), (64, 64, 4, 4), (100, 36, 4, 4), (613, 40, 4, 4),
               (613, 9000, 4, 4), (1, 1, 4, 4), (33, 33, 16, 5), (256, 512, 16, 5),
               (5, 17, 1, 4), (12, 12, 1, 1)]
    windows += [(3 + 5 * k, 2 + 7 * k, 5, 7) for k in range(21)]
    # single queries of their strides whose width is a multiple of the
    # stride (right corners exchanged through shared memory without a
    # shared top-left load)
    windows += [(30, 30, 5, 5), (7, 21, 3, 3), (613, 600, 6, 6)]
    check_windows(sat, S_ref, Q_ref, windows)
    check_windows(sat, S_ref, Q_ref, windows[:4], outputs=("sum",))
    check_windows(sat, S_ref, Q_ref, windows[6:8], outputs=("mean", "std"))
    # Pitched outputs (row stride C + 5) for a group of four same-stride
    # queries; the padding must stay untouched.
    import torch
    group = windows[:4]
    out = []
    for wh, ww, sy, sx in group:
        R, C = swa.window_shape(*img.shape, wh, ww, sy, sx)
        out.append({k: torch.full((R, C + 5), -7, dtype=torch.int64 if k == "sum"
                                  else torch.float64, device="cuda") for k in ("sum", "mean", "std")})
    res = sat.window_stats(group, out=[{k: v[:, :v.shape[1] - 5] for k, v in o.items()} for o in out])
    for (wh, ww, sy, sx), got, full in zip(group, res, out):
        want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx)
        np.testing.assert_array_equal(u64(got["sum"]), want["sum"])
        np.testing.assert_array_equal(f64(got["mean"]), want["mean"])
        np.testing.assert_array_equal(f64(got["std"]), want["std"])
        for k in ("sum", "mean", "std"):
            pad = full[k][:, -5:].cpu()
            assert (pad == -7).all(), k
    sat.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_hand_worked_golden(dtype):
    """The CUDA path on the hand-worked cases of tests/golden/hand_worked.txt:
    tables and sums exact, means the correctly rounded quotient, stds within
    2 ulp of the exact root and equal to the oracle's bit for bit."""
    import golden_util
    for case in golden_util.load_cases():
        img = case["image"].astype(dtype)
        sat = swa.build_sat(to_device(img))
        S, Q = sat.tables()
        if "S" in case:
            np.testing.assert_array_equal(u64(S), case["S"])
            np.testing.assert_array_equal(u64(Q), case["Q"])
        S_ref, Q_ref = oracle.sat(img)
        shapes = [w["shape"] for w in case["windows"]]
        for w, got in zip(case["windows"], sat.window_stats(shapes)):
            R, C = swa.window_shape(*img.shape, *w["shape"])
            s, m, d = golden_util.expected(w, R, C)
            np.testing.assert_array_equal(u64(got["sum"]), s)
            np.testing.assert_array_equal(f64(got["mean"]), m)
            g = f64(got["std"])
            assert (np.abs(g - d) <= 2 * np.spacing(d)).all(), (case["name"], w["shape"])
            want = oracle.window_sat(S_ref, Q_ref, *w["shape"])
            np.testing.assert_array_equal(g, want["std"])
        sat.free()


def test_windows_closed_forms():
    """Constant image: mean exact, std exactly 0; checkerboard {0, a}, even w:
    std exactly a/2."""
    const = np.full((300, 300), 171, np.uint8)
    sat = swa.build_sat(to_device(const))
    (o,) = sat.window_stats([(25, 25, 1, 1)])
    assert (u64(o["sum"]) == 171 * 625).all()
    assert (f64(o["mean"]) == 171.0).all() and (f64(o["std"]) == 0.0).all()
    a = 60000
    cb = ((np.indices((300, 300)).sum(0) % 2) * a).astype(np.uint16)
    sat = swa.build_sat(to_device(cb))
    (o,) = sat.window_stats([(8, 8, 1, 1)])
    assert (f64(o["std"]) == a / 2).all() and (f64(o["mean"]) == a / 2).all()


def test_window_on_another_stream():
    """The build runs on one stream and the windows on another; the library
    orders them."""
    import torch
    img = rand_img(700, 900, np.uint8)
    dev = to_device(img)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        sat = swa.build_sat(dev, stream=s1)
    (o,) = sat.window_stats([(40, 40, 1, 1)], stream=s2)
    s2.synchronize()
    S_ref, Q_ref = oracle.sat(img)
    want = oracle.window_sat(S_ref, Q_ref, 40, 40, 1, 1)
    np.testing.assert_array_equal(u64(o["sum"]), want["sum"])
    sat.free()


def test_analyze_host_buffers_match_device_path():
    """swa_analyze with pinned host input and host outputs equals the device
    path."""
    import torch
    img = rand_img(513, 1025, np.uint16)
    wins = [(31, 31, 1, 1), (64, 64, 4, 4)]
    host = torch.from_numpy(img.view(np.int16)).pin_memory()
    res = swa.analyze(host, wins)
    S_ref, Q_ref = oracle.sat(img)
    for (wh, ww, sy, sx), got in zip(wins, res):
        want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx)
        assert not got["sum"].is_cuda
        np.testing.assert_array_equal(got["sum"].numpy().view(np.uint64), want["sum"])
        np.testing.assert_array_equal(got["mean"].numpy(), want["mean"])
        np.testing.assert_array_equal(got["std"].numpy(), want["std"])


def test_workload0_cell_mask():
    """1024x1024 cell-centroid mask, window 32 stride 1, sum only, against the
    naive definition."""
    (im,) = synth.workload(0)
    img = im.generate()
    sat = swa.build_sat(to_device(img), with_sq=False)
    (o,) = sat.window_stats([(32, 32, 1, 1)], outputs=("sum",))
    want = oracle.window_brute(img, 32, 32, 1, 1, outputs=("sum",))["sum"]
    np.testing.assert_array_equal(u64(o["sum"]), want)
    assert o["sum"].shape == (993, 993)
    sat.free()


OUTPUT_SETS = [("sum",), ("mean",), ("std",), ("sum", "mean"), ("sum", "std"), ("mean", "std"),
               ("sum", "mean", "std")]


@pytest.mark.parametrize("outputs", OUTPUT_SETS, ids=["+".join(o) for o in OUTPUT_SETS])
@pytest.mark.parametrize("stride", [1, 2, 4])
def test_every_output_selection(outputs, stride):
    """Each selection of outputs runs its own kernel instantiation (dense
    column strides 1-2, sparse from 3; the 64-bit-D and 128-bit-D rounding
    paths): all of them must equal the oracle.  On a uint16 image a 31 x 17
    window takes the 64-bit-D path (n * 65535 < 2^32), a 300 x 300 one the
    128-bit path."""
    img = rand_img(700, 1100, np.uint16)
    sat = swa.build_sat(to_device(img), with_sq=True)
    S_ref, Q_ref = oracle.sat(img)
    check_windows(sat, S_ref, Q_ref, [(31, 17, stride, stride), (300, 300, stride, stride)],
                  outputs=outputs)
    sat.free()
