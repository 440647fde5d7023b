"""Out-of-core analysis in row bands (swa_analyze_banded) against the oracle:
bands of 1 row up to the whole image, bands shorter than the window (the
table of a band then starts far above it), both dtypes, host and device
images and outputs, pitched outputs.  Sums, means and stds must equal the
oracle's bit for bit, like the one-table path."""
import numpy as np
import pytest

import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = pytest.mark.gpu

WINDOWS = [(5, 7, 1, 1), (64, 64, 3, 5), (150, 33, 7, 2), (1, 1, 4, 4)]


def _image(dtype, r, c, seed):
    if dtype == "u8":
        return synth.intensity_u8(r, c, seed, synth.cluster_count(r, c))
    return synth.intensity_u16(r, c, seed, synth.cluster_count(r, c))


def _check(img, res, windows):
    S, Q = oracle.sat(img)
    for (wh, ww, sy, sx), got in zip(windows, res):
        want = oracle.window_sat(S, Q, wh, ww, sy, sx)
        np.testing.assert_array_equal(u64(got["sum"]), want["sum"])
        np.testing.assert_array_equal(f64(got["mean"]), want["mean"])
        np.testing.assert_array_equal(f64(got["std"]), want["std"])


@pytest.mark.parametrize("dtype,band_rows", [("u8", 1), ("u8", 7), ("u8", 64), ("u8", 333),
                                             ("u8", 0), ("u16", 13), ("u16", 100000)])
def test_banded_host_in_host_out(dtype, band_rows):
    require_gpu()
    import torch
    img = _image(dtype, 517, 701, 41 + band_rows)
    h = torch.from_numpy(img.view(np.int16) if dtype == "u16" else img).pin_memory()
    res = swa.analyze(h, WINDOWS, band_rows=band_rows)
    _check(img, res, WINDOWS)


@pytest.mark.parametrize("dtype,cols,band_rows", [("u8", 733, 5), ("u8", 640, 64), ("u16", 733, 33),
                                                  ("u8", 733, 0), ("u16", 640, 150)])
def test_banded_two_buffer_mode(dtype, cols, band_rows):
    """A host image staged in two band buffers (the mode for images larger
    than a quarter of the free device memory), forced on a small image by a
    test hook: each band's rows shared with the previous band are copied on
    the device, the rest uploaded (linear copies when host and device rows
    have the same pitch, pitched ones otherwise)."""
    require_gpu()
    import torch
    L = swa.lib()
    img = _image(dtype, 611, cols, 19 + band_rows)
    h = torch.from_numpy(img.view(np.int16) if dtype == "u16" else img).pin_memory()
    assert L.swa_set_test_hooks(swa.SWA_HOOK_BAND_BUFFERS) == 0
    try:
        res = swa.analyze(h, WINDOWS, band_rows=band_rows)
    finally:
        L.swa_set_test_hooks(0)
    _check(img, res, WINDOWS)


@pytest.mark.parametrize("dtype", ["u8", "u16"])
def test_banded_pitched_host_image(dtype):
    """Host rows with padding (a column slice of a wider pinned array) go to
    back-to-back device rows with pitched copies."""
    require_gpu()
    import torch
    img = _image(dtype, 450, 519, 23)
    wide = np.zeros((450, 530), dtype=img.dtype)
    wide[:, 3:522] = img
    h = torch.from_numpy(wide.view(np.int16) if dtype == "u16" else wide).pin_memory()[:, 3:522]
    res = swa.analyze(h, WINDOWS, band_rows=40)
    _check(img, res, WINDOWS)


@pytest.mark.parametrize("band_rows", [9, 50, 0])
def test_banded_same_stride_queries_of_different_heights(band_rows):
    """Sparse-stride queries with equal strides share one sweep; in a band
    their first output rows start at different table rows (row0), so they
    do not share corner loads.  Heights 8..200, strides 4 and 16."""
    require_gpu()
    import torch
    img = _image("u8", 433, 1500, 5 + band_rows)
    wl = [(8, 8, 4, 4), (40, 24, 4, 4), (200, 96, 4, 4), (16, 256, 16, 16), (128, 16, 16, 16)]
    h = torch.from_numpy(img).pin_memory()
    res = swa.analyze(h, wl, band_rows=band_rows)
    _check(img, res, wl)


@pytest.mark.parametrize("dtype", ["u8", "u16"])
def test_banded_device_in_device_out_pitched(dtype):
    require_gpu()
    import torch
    img = _image(dtype, 389, 455, 77)
    d = to_device(img, pad_cols=13, offset_px=0)
    out = []
    for wh, ww, sy, sx in WINDOWS:
        R, C = swa.window_shape(*img.shape, wh, ww, sy, sx)
        out.append({k: torch.full((R, C + 3), -1, dtype=torch.int64 if k == "sum"
                                  else torch.float64, device="cuda")[:, :C]
                    for k in ("sum", "mean", "std")})
    res = swa.analyze(d, WINDOWS, out=out, band_rows=10)
    _check(img, res, WINDOWS)


def test_banded_pageable_host_image_matches_one_table_path():
    require_gpu()
    import torch
    img = _image("u8", 640, 480, 5)
    h = torch.from_numpy(img)                       # pageable
    banded = swa.analyze(h, WINDOWS, band_rows=50)
    whole = swa.analyze(h.pin_memory(), WINDOWS)
    for a, b in zip(banded, whole):
        for k in ("sum", "mean", "std"):
            assert torch.equal(a[k], b[k])


def test_banded_repeated_calls_and_sum_only():
    require_gpu()
    img = _image("u8", 300, 900, 9)
    import torch
    h = torch.from_numpy(img).pin_memory()
    wl = [(32, 32, 1, 1)]
    for _ in range(2):
        res = swa.analyze(h, wl, outputs=("sum",), band_rows=40)
        want = oracle.window_brute(img, 32, 32, 1, 1, outputs=("sum",))
        np.testing.assert_array_equal(u64(res[0]["sum"]), want["sum"])


@pytest.mark.slow
def test_analyze_routes_large_host_images_through_bands():
    """swa_analyze streams a host image of 256 MiB or more band by band; the
    results equal the one-table device path bit for bit, and sampled windows
    equal the definition."""
    require_gpu()
    import torch
    r, c = 16400, 16400
    img = _image("u8", r, c, 12)
    wl = [(100, 100, 7, 5), (1024, 512, 16, 16)]
    h = torch.from_numpy(img).pin_memory()
    streamed = swa.analyze(h, wl)
    sat = swa.build_sat(torch.from_numpy(img).cuda())
    direct = sat.window_stats(wl)
    for a, d in zip(streamed, direct):
        for k in ("sum", "mean", "std"):
            assert torch.equal(a[k], d[k].cpu()), k
    rng = np.random.default_rng(5)
    for (wh, ww, sy, sx), a in zip(wl, streamed):
        R, C = a["sum"].shape
        for i, j in zip(rng.integers(0, R, 20), rng.integers(0, C, 20)):
            s, _, m, d = oracle.window_one(img, int(i) * sy, int(j) * sx, wh, ww)
            assert int(u64(a["sum"][i:i + 1, j:j + 1])[0, 0]) == s
            assert f64(a["mean"][i:i + 1, j:j + 1])[0, 0] == m
            assert f64(a["std"][i:i + 1, j:j + 1])[0, 0] == d
    sat.free()


@pytest.mark.parametrize("dtype", ["u8", "u16"])
def test_banded_device_in_host_out(dtype):
    """Device image, pinned host outputs, many bands: the results of band t
    are downloaded from a staging set that band t+2 reuses."""
    require_gpu()
    import torch
    img = _image(dtype, 403, 389, 91)
    d = to_device(img)
    out = []
    for wh, ww, sy, sx in WINDOWS:
        R, C = swa.window_shape(*img.shape, wh, ww, sy, sx)
        out.append({k: torch.empty((R, C), dtype=torch.int64 if k == "sum" else torch.float64,
                                   pin_memory=True) for k in ("sum", "mean", "std")})
    res = swa.analyze(d, WINDOWS, out=out, band_rows=4)
    _check(img, res, WINDOWS)
