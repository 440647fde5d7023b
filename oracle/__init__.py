"""CPU oracle for parallel-integral-image sliding window analysis.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library's compute
path never does, and this package imports nothing from the library.

Thin numpy wrappers over ``oracle.c`` (plain serial C; see its header for the
definitions and the paper sections they follow):

- ``sat``            summed-area tables S and Q (Section II-B)
- ``sat_rows``       selected table rows, streamed (for images too large to
                     hold both tables in host memory)
- ``window_brute``   naive SWA, the definition (Sections II-A, III-A)
- ``window_sat``     integral-image SWA, four lookups (Sections II-B, III-B)
- ``window_sliding`` DP-naive-SWA read as separable moving sums (Section IV-A)
- ``window_one``     one window by the definition (sampled checks at any size)
- ``window_sat_rows`` integral-image SWA for selected output rows
- ``window_rows_stream`` the same from the image, streamed once, keeping only
                     the table rows the windows' corners lie on (full-size
                     checks without whole tables in host memory)
- ``stats_from_moments`` mean and population std from exact integer moments
- ``count_brute``    threshold count map by the definition (pixels > thr per
                     window, their fraction and the indicator's std)
- ``count_sat``      the same through the indicator image's tables

Row-parallel variants for timing the CPU baseline on all host cores
(``oracle_par.c``, OpenMP row bands; pinned equal to the serial functions):

- ``sat_par``, ``window_sat_par``; ``par_threads`` sets or reads the thread
  count
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_PAR = os.path.join(_HERE, "oracle_par.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

DT = {"u8": 1, "u16": 2, np.dtype(np.uint8): 1, np.dtype(np.uint16): 2}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, no fast-math, no contraction; OpenMP
    only in the row-parallel variants of ``oracle_par.c``)."""
    if force or not os.path.exists(_LIB_PATH) or any(
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(f) for f in (_SRC, _SRC_PAR)):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
            "-fPIC", "-shared", _SRC, _SRC_PAR, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, vp, dbl, ci = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                 ctypes.c_double, ctypes.c_int)
        P = ctypes.POINTER
        lib.oracle_fits_u64.argtypes = [i64, i64, ci, ci]
        lib.oracle_window_shape.argtypes = [i64, i64, i64, i64, i64, i64, P(i64), P(i64)]
        lib.oracle_u128_to_double.argtypes = [u64, u64]
        lib.oracle_u128_to_double.restype = dbl
        lib.oracle_stats_from_moments.argtypes = [u64, u64, u64, P(dbl), P(dbl)]
        lib.oracle_stats_from_moments.restype = None
        lib.oracle_sat.argtypes = [vp, i64, i64, i64, ci, vp, vp, i64]
        lib.oracle_sat_rows.argtypes = [vp, i64, i64, i64, ci, vp, i64, vp, vp]
        lib.oracle_window_one.argtypes = [vp, i64, i64, i64, ci, i64, i64, i64, i64,
                                          P(u64), P(u64), P(dbl), P(dbl)]
        lib.oracle_count_brute.argtypes = [vp, i64, i64, i64, ci, u64, i64, i64, i64, i64,
                                           vp, vp, vp, i64]
        for f in (lib.oracle_window_brute, lib.oracle_window_sliding):
            f.argtypes = [vp, i64, i64, i64, ci, i64, i64, i64, i64, vp, vp, vp, i64]
        lib.oracle_window_sat.argtypes = [vp, vp, i64, i64, i64, i64, i64, i64, i64,
                                          vp, vp, vp, i64]
        lib.oracle_total.argtypes = [vp, i64, i64, i64, ci, P(u64), P(u64)]
        lib.oracle_stats_bulk.argtypes = [vp, vp, vp, i64, vp, vp]
        lib.oracle_stats_bulk.restype = None
        lib.oracle_window_sat_rows.argtypes = [vp, vp, i64, i64, i64, i64, i64, i64, i64,
                                               vp, i64, vp, vp, vp, i64]
        lib.oracle_sat_par.argtypes = [vp, i64, i64, i64, ci, vp, vp, i64]
        lib.oracle_window_sat_par.argtypes = [vp, vp, i64, i64, i64, i64, i64, i64, i64,
                                              vp, vp, vp, i64]
        lib.oracle_par_threads.argtypes = [ci]
        lib.oracle_par_threads.restype = ci
        lib.oracle_window_rows_stream.argtypes = [vp, i64, i64, i64, ci, i64, i64, i64, i64,
                                                  vp, i64, vp, vp, vp, i64]
        _lib = lib
    return _lib


def _img(img):
    img = np.asarray(img)
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16):
        raise TypeError("image must be a 2-D uint8 or uint16 array")
    if img.strides[1] != img.itemsize:
        img = np.ascontiguousarray(img)
    return img, DT[img.dtype]


def _check(rc, what):
    if rc != 0:
        raise ValueError("%s failed with code %d" % (what, rc))


def fits_u64(rows: int, cols: int, dtype: str, with_sq: bool) -> bool:
    return bool(_load().oracle_fits_u64(rows, cols, DT[dtype], int(with_sq)))


def window_shape(rows, cols, wh, ww, sy, sx):
    R, C = ctypes.c_int64(), ctypes.c_int64()
    _check(_load().oracle_window_shape(rows, cols, wh, ww, sy, sx,
                                       ctypes.byref(R), ctypes.byref(C)), "window_shape")
    return R.value, C.value


def u128_to_double(v: int) -> float:
    return _load().oracle_u128_to_double((v >> 64) & (2**64 - 1), v & (2**64 - 1))


def stats_from_moments(n: int, sw: int, qw: int):
    m, s = ctypes.c_double(), ctypes.c_double()
    _load().oracle_stats_from_moments(n, sw, qw, ctypes.byref(m), ctypes.byref(s))
    return m.value, s.value


def stats_bulk(n, sw, qw):
    """stats_from_moments over uint64 arrays: (mean, std) float64 arrays."""
    n, sw, qw = (np.ascontiguousarray(a, dtype=np.uint64) for a in (n, sw, qw))
    m = np.empty(len(n), np.float64)
    s = np.empty(len(n), np.float64)
    _load().oracle_stats_bulk(n.ctypes.data, sw.ctypes.data, qw.ctypes.data, len(n),
                              m.ctypes.data, s.ctypes.data)
    return m, s


def sat(img, with_sq: bool = True):
    """(S, Q) as uint64 arrays of the image's shape (Q is None if not with_sq)."""
    img, dt = _img(img)
    r, c = img.shape
    S = np.empty((r, c), np.uint64)
    Q = np.empty((r, c), np.uint64) if with_sq else None
    _check(_load().oracle_sat(img.ctypes.data, r, c, img.strides[0], dt, S.ctypes.data,
                              Q.ctypes.data if with_sq else None, c), "sat")
    return S, Q


def sat_par(img, with_sq: bool = True):
    """``sat`` on all threads (row bands): the same tables."""
    img, dt = _img(img)
    r, c = img.shape
    S = np.empty((r, c), np.uint64)
    Q = np.empty((r, c), np.uint64) if with_sq else None
    _check(_load().oracle_sat_par(img.ctypes.data, r, c, img.strides[0], dt, S.ctypes.data,
                                  Q.ctypes.data if with_sq else None, c), "sat_par")
    return S, Q


def par_threads(n: int = 0) -> int:
    """Set (n > 0) and return the thread count of the parallel variants."""
    return int(_load().oracle_par_threads(int(n)))


def sat_rows(img, rows_wanted, with_sq: bool = True):
    """Table rows ``rows_wanted`` (strictly increasing) of S and Q, streamed."""
    img, dt = _img(img)
    r, c = img.shape
    req = np.ascontiguousarray(np.asarray(rows_wanted, dtype=np.int64))
    S = np.empty((len(req), c), np.uint64)
    Q = np.empty((len(req), c), np.uint64) if with_sq else None
    _check(_load().oracle_sat_rows(img.ctypes.data, r, c, img.strides[0], dt,
                                   req.ctypes.data, len(req), S.ctypes.data,
                                   Q.ctypes.data if with_sq else None), "sat_rows")
    return S, Q


def window_one(img, y0, x0, wh, ww):
    """(sum, sum of squares, mean, std) of one window by the definition."""
    img, dt = _img(img)
    r, c = img.shape
    s, q = ctypes.c_uint64(), ctypes.c_uint64()
    m, d = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_window_one(img.ctypes.data, r, c, img.strides[0], dt, y0, x0,
                                     wh, ww, ctypes.byref(s), ctypes.byref(q),
                                     ctypes.byref(m), ctypes.byref(d)), "window_one")
    return s.value, q.value, m.value, d.value


def _outputs(R, C, outputs):
    return (np.empty((R, C), np.uint64) if "sum" in outputs else None,
            np.empty((R, C), np.float64) if "mean" in outputs else None,
            np.empty((R, C), np.float64) if "std" in outputs else None)


def _p(a):
    return None if a is None else a.ctypes.data


def window_brute(img, wh, ww, sy=1, sx=1, outputs=("sum", "mean", "std")):
    """Naive SWA: dict of the requested outputs, each R x C."""
    img, dt = _img(img)
    r, c = img.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    s, m, d = _outputs(R, C, outputs)
    _check(_load().oracle_window_brute(img.ctypes.data, r, c, img.strides[0], dt, wh, ww,
                                       sy, sx, _p(s), _p(m), _p(d), C), "window_brute")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def window_sliding(img, wh, ww, sy=1, sx=1, outputs=("sum", "mean", "std")):
    """DP-naive-SWA (separable moving sums): dict of the requested outputs."""
    img, dt = _img(img)
    r, c = img.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    s, m, d = _outputs(R, C, outputs)
    _check(_load().oracle_window_sliding(img.ctypes.data, r, c, img.strides[0], dt, wh,
                                         ww, sy, sx, _p(s), _p(m), _p(d), C),
           "window_sliding")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def window_sat(S, Q, wh, ww, sy=1, sx=1, outputs=("sum", "mean", "std")):
    """Integral-image SWA on oracle tables: dict of the requested outputs."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    if Q is not None:
        Q = np.ascontiguousarray(Q, dtype=np.uint64)
    r, c = S.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    s, m, d = _outputs(R, C, outputs)
    _check(_load().oracle_window_sat(S.ctypes.data, _p(Q), c, r, c, wh, ww, sy, sx,
                                     _p(s), _p(m), _p(d), C), "window_sat")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def window_sat_par(S, Q, wh, ww, sy=1, sx=1, outputs=("sum", "mean", "std")):
    """``window_sat`` on all threads (output rows split): the same outputs."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    if Q is not None:
        Q = np.ascontiguousarray(Q, dtype=np.uint64)
    r, c = S.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    s, m, d = _outputs(R, C, outputs)
    _check(_load().oracle_window_sat_par(S.ctypes.data, _p(Q), c, r, c, wh, ww, sy, sx,
                                         _p(s), _p(m), _p(d), C), "window_sat_par")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def window_sat_rows(S, Q, wh, ww, sy, sx, out_rows, outputs=("sum", "mean", "std")):
    """Integral-image SWA for the selected output rows only."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    if Q is not None:
        Q = np.ascontiguousarray(Q, dtype=np.uint64)
    r, c = S.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    rr = np.ascontiguousarray(np.asarray(out_rows, dtype=np.int64))
    s, m, d = _outputs(len(rr), C, outputs)
    _check(_load().oracle_window_sat_rows(S.ctypes.data, _p(Q), c, r, c, wh, ww, sy, sx,
                                          rr.ctypes.data, len(rr), _p(s), _p(m), _p(d), C),
           "window_sat_rows")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def window_rows_stream(img, wh, ww, sy, sx, out_rows, outputs=("sum", "mean", "std")):
    """Integral-image SWA for the selected (strictly increasing) output rows,
    from the image streamed once: only the table rows the corners lie on are
    kept, so this works on images whose tables exceed host memory."""
    img, dt = _img(img)
    r, c = img.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    rr = np.ascontiguousarray(np.asarray(out_rows, dtype=np.int64))
    s, m, d = _outputs(len(rr), C, outputs)
    _check(_load().oracle_window_rows_stream(img.ctypes.data, r, c, img.strides[0], dt, wh, ww,
                                             sy, sx, rr.ctypes.data, len(rr), _p(s), _p(m),
                                             _p(d), C), "window_rows_stream")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def total(img):
    """(sum of pixels, sum of squared pixels) by a flat loop."""
    img, dt = _img(img)
    r, c = img.shape
    s, q = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_load().oracle_total(img.ctypes.data, r, c, img.strides[0], dt,
                                ctypes.byref(s), ctypes.byref(q)), "total")
    return s.value, q.value


def count_brute(img, thr, wh, ww, sy=1, sx=1, outputs=("sum", "mean", "std")):
    """Threshold count map by the definition: per window the number of pixels
    > thr ("sum"), their fraction ("mean") and the std of the 0/1 indicator."""
    img, dt = _img(img)
    r, c = img.shape
    R, C = window_shape(r, c, wh, ww, sy, sx)
    s, m, d = _outputs(R, C, outputs)
    _check(_load().oracle_count_brute(img.ctypes.data, r, c, img.strides[0], dt, int(thr), wh,
                                      ww, sy, sx, _p(s), _p(m), _p(d), C), "count_brute")
    return {k: v for k, v in (("sum", s), ("mean", m), ("std", d)) if v is not None}


def count_sat(img, thr, windows, outputs=("sum", "mean", "std")):
    """Threshold count maps for several windows through the tables of the
    0/1 indicator image (img > thr); its squared values are the values, so
    its S table serves as Q as well."""
    ind = (np.asarray(img) > thr).astype(np.uint8)
    S, _ = sat(ind, with_sq=False)
    return [window_sat(S, S, wh, ww, sy, sx, outputs=outputs) for wh, ww, sy, sx in windows]
