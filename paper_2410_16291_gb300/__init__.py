"""GB300 sliding-window analysis with parallel integral images (arXiv 2410.16291).

Python binding of ``libswa.so`` (declared in ``include/swa.h``).  The
functions named ``swa_*`` are the C entry points with their C arguments
(integers and raw pointers); ``build_sat`` / ``SAT.window_stats`` /
``analyze`` marshal torch tensors into those calls.  Every step of the
computation runs in the library's CUDA kernels: there is no CPU path, and
loading fails loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswa.so")

SWA_U8, SWA_U16 = 1, 2
SWA_OK, SWA_EINVAL, SWA_EOVERFLOW, SWA_ENOMEM, SWA_ECUDA, SWA_ETIMEOUT = range(6)
SWA_WITH_SQ, SWA_TWOPASS, SWA_COUNT = 1, 2, 4
SWA_LATTICE_SHIFT = 8
SWA_OUT_SUM, SWA_OUT_MEAN, SWA_OUT_STD = 1, 2, 4
SWA_MAX_WINDOWS = 64
SWA_HOOK_STALL_TILE0 = 1
SWA_HOOK_BAND_BUFFERS = 2
SWA_HOOK_CORNER_MODE = 4
SWA_HOOK_ROW_ORDER = 8

#: C function name -> (restype, argtypes)
_I64, _U64, _U32, _I32, _VP = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                               ctypes.c_int32, ctypes.c_void_p)
_P = ctypes.POINTER


class swa_window(ctypes.Structure):
    """Mirror of ``swa_window`` in swa.h."""
    _fields_ = [("wh", _I64), ("ww", _I64), ("sy", _I64), ("sx", _I64),
                ("outputs", _U32), ("reserved", _U32), ("sum", _VP), ("mean", _VP),
                ("std", _VP), ("out_ld", _I64)]


class swa_batch_item(ctypes.Structure):
    """Mirror of ``swa_batch_item`` in swa.h."""
    _fields_ = [("image", _VP), ("rows", _I64), ("cols", _I64), ("pitch_bytes", _I64),
                ("dtype", ctypes.c_int), ("n_windows", _I32), ("windows", _P(swa_window))]


class swa_batch_config(ctypes.Structure):
    """Mirror of ``swa_batch_config`` in swa.h."""
    _fields_ = [("u8_tile_rows", _I32), ("order", _I32), ("ticket_order", _I32),
                ("lookback", _I32), ("warps", _I32), ("interleave", _I32),
                ("reserved", _I32 * 2)]


class swa_kernel_time(ctypes.Structure):
    """Mirror of ``swa_kernel_time`` in swa.h."""
    _fields_ = [("name", ctypes.c_char * 48), ("launches", _I64), ("total_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


SIGNATURES = {
    "swa_build_sat": (ctypes.c_int, [_VP, _I64, _I64, _I64, ctypes.c_int, _U32, _VP, _P(_VP)]),
    "swa_build_count_sat": (ctypes.c_int, [_VP, _I64, _I64, _I64, ctypes.c_int, _U32, _VP,
                                           _P(_VP)]),
    "swa_window_shape": (ctypes.c_int, [_I64, _I64, _I64, _I64, _I64, _I64, _P(_I64), _P(_I64)]),
    "swa_window_stats": (ctypes.c_int, [_VP, _I64, _I64, _I64, _I64, _U32, _VP, _VP, _VP, _I64, _VP]),
    "swa_window_stats_multi": (ctypes.c_int, [_VP, _P(swa_window), _I32, _VP]),
    "swa_sat_data": (ctypes.c_int, [_VP, _P(_VP), _P(_VP), _P(_I64)]),
    "swa_sat_lattice": (ctypes.c_int, [_VP, _P(_VP), _P(_VP), _P(_I64), _P(_I64), _P(_I64),
                                       _P(_I32)]),
    "swa_sat_info": (ctypes.c_int, [_VP, _P(_I64), _P(_I64), _P(_I32), _P(_U32)]),
    "swa_sat_bytes": (ctypes.c_int, [_I64, _I64, ctypes.c_int, _U32, _P(_I64), _P(_I64)]),
    "swa_sync": (ctypes.c_int, [_VP]),
    "swa_sat_status": (ctypes.c_int, [_VP]),
    "swa_free": (None, [_VP]),
    "swa_analyze": (ctypes.c_int, [_VP, _I64, _I64, _I64, ctypes.c_int, _P(swa_window), _I32, _VP]),
    "swa_analyze_banded": (ctypes.c_int, [_VP, _I64, _I64, _I64, ctypes.c_int, _P(swa_window), _I32,
                                          _I64, _VP]),
    "swa_band_range": (ctypes.c_int, [_I64, _I64, _I64, _I64, _I64, _P(_I64), _P(_I64)]),
    "swa_set_memory_limit": (ctypes.c_int, [_I64]),
    "swa_memory_in_use": (_I64, []),
    "swa_trim": (ctypes.c_int, [_I64]),
    "swa_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "swa_last_error": (ctypes.c_char_p, []),
    "swa_launch_count": (_I64, []),
    "swa_version": (_I32, []),
    "swa_profile_begin": (ctypes.c_int, []),
    "swa_set_test_hooks": (ctypes.c_int, [_U32]),
    "swa_batch_create": (ctypes.c_int, [_P(swa_batch_item), _I32, _P(swa_batch_config), _VP,
                                        _P(_VP)]),
    "swa_batch_run": (ctypes.c_int, [_VP, _VP]),
    "swa_batch_sync": (ctypes.c_int, [_VP]),
    "swa_batch_tables": (ctypes.c_int, [_VP, _I32, _P(_VP), _P(_VP), _P(_I64)]),
    "swa_batch_bytes": (_I64, [_VP]),
    "swa_batch_free": (None, [_VP]),
    "swa_build_sat_noalloc": (ctypes.c_int, [_VP, _I64, _I64, _I64, ctypes.c_int, _U32, _VP, _VP,
                                             _I64, _VP, _VP]),
    "swa_profile_end": (_I32, [_P(swa_kernel_time), _I32]),
    "swa_verify_tables": (ctypes.c_int, [_VP, _I64, _I64, _I64, ctypes.c_int, _VP, _VP, _I64,
                                         _VP, _VP]),
}

_lib = None


def lib():
    """The loaded ``libswa.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libswa.so is not built (run __graft_entry__.build() or "
                "python paper_2410_16291_gb300/build.py); there is no fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def __getattr__(name):
    # swa_* entry points resolve to the C functions themselves.
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


class SwaError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = lib().swa_status_str(status).decode()
        last = lib().swa_last_error().decode()
        super().__init__("%s: %s%s" % (what, msg, (" (%s)" % last) if last else ""))


def check(status, what=""):
    if status != SWA_OK:
        raise SwaError(status, what)


def profile_begin():
    """Start bracketing every library kernel launch with CUDA events."""
    check(lib().swa_profile_begin(), "swa_profile_begin")


def profile_end():
    """Stop profiling; {kernel name: (launches, total_ms, max_ms)}."""
    buf = (swa_kernel_time * 64)()
    n = lib().swa_profile_end(buf, 64)
    if n < 0:
        raise SwaError(SWA_ECUDA, "swa_profile_end")
    return {buf[k].name.decode(): (buf[k].launches, buf[k].total_ms, buf[k].max_ms)
            for k in range(min(n, 64))}


def window_shape(rows, cols, wh, ww, sy=1, sx=1):
    R, C = _I64(), _I64()
    check(lib().swa_window_shape(rows, cols, wh, ww, sy, sx, ctypes.byref(R), ctypes.byref(C)),
          "swa_window_shape")
    return R.value, C.value


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dtype_code(t):
    """uint8 -> SWA_U8; uint16 (or int16 holding uint16 bit patterns) -> SWA_U16."""
    import torch
    if t.dtype == torch.uint8:
        return SWA_U8
    if t.dtype in (torch.uint16, torch.int16):
        return SWA_U16
    raise TypeError("image must be uint8 or uint16, got %s" % t.dtype)


class SAT:
    """A built table pair on the device (owns the C handle)."""

    def __init__(self, handle, rows, cols, with_sq, stream):
        self.handle = handle
        self.rows, self.cols, self.with_sq, self.stream = rows, cols, with_sq, stream

    def window_stats(self, windows, outputs=("sum", "mean", "std"), stream=None, out=None):
        """Evaluate windows [(wh, ww, sy, sx), ...] in one launch sequence.

        Returns a list of dicts of device tensors (R x C each): "sum" is an
        int64 tensor holding the uint64 sums' bit patterns (torch has few
        uint64 operations), "mean" and "std" are float64.  ``out`` may supply
        preallocated dicts of tensors (contiguous rows, any row stride).
        """
        import torch
        if len(windows) > SWA_MAX_WINDOWS:
            res = []
            for k in range(0, len(windows), SWA_MAX_WINDOWS):
                res += self.window_stats(windows[k:k + SWA_MAX_WINDOWS], outputs, stream,
                                         None if out is None else out[k:k + SWA_MAX_WINDOWS])
            return res
        arr = (swa_window * len(windows))()
        res = []
        mask = (SWA_OUT_SUM if "sum" in outputs else 0) | (
            SWA_OUT_MEAN if "mean" in outputs else 0) | (SWA_OUT_STD if "std" in outputs else 0)
        dev = torch.device("cuda", torch.cuda.current_device())
        for k, w in enumerate(windows):
            wh, ww, sy, sx = w
            R, C = window_shape(self.rows, self.cols, wh, ww, sy, sx)
            if out is not None:
                o = out[k]
            else:
                o = {}
                if mask & SWA_OUT_SUM:
                    o["sum"] = torch.empty((R, C), dtype=torch.int64, device=dev)
                if mask & SWA_OUT_MEAN:
                    o["mean"] = torch.empty((R, C), dtype=torch.float64, device=dev)
                if mask & SWA_OUT_STD:
                    o["std"] = torch.empty((R, C), dtype=torch.float64, device=dev)
            ld = next(iter(o.values())).stride(0)
            for t in o.values():
                assert t.shape == (R, C) and t.stride(1) == 1 and t.stride(0) == ld and t.is_cuda
            arr[k] = swa_window(wh, ww, sy, sx, mask, 0,
                                o["sum"].data_ptr() if "sum" in o else None,
                                o["mean"].data_ptr() if "mean" in o else None,
                                o["std"].data_ptr() if "std" in o else None, ld)
            res.append(o)
        check(lib().swa_window_stats_multi(self.handle, arr, len(windows), _stream_ptr(stream)),
              "swa_window_stats_multi")
        return res

    def tables(self):
        """(S, Q) as device tensors viewing the handle's memory (rows x cols).

        Views are int64 tensors (uint64 bit patterns) over ld-strided rows;
        they are only valid while this object lives.
        """
        import torch
        S, Q, ld = _VP(), _VP(), _I64()
        check(lib().swa_sat_data(self.handle, ctypes.byref(S), ctypes.byref(Q), ctypes.byref(ld)))
        return _view_u64(S.value, self.rows, self.cols, ld.value), (
            _view_u64(Q.value, self.rows, self.cols, ld.value) if Q.value else None)

    def lattice(self):
        """(stride, LS, LQ): the corner lattice of a build with ``lattice=s``
        (int64 views, uint64 bit patterns; entry (a, b) is the table entry at
        row s*(a+1)-1, column s*(b+1)-1), or (0, None, None) without one."""
        LS, LQ, r, c, ld, st = _VP(), _VP(), _I64(), _I64(), _I64(), _I32()
        check(lib().swa_sat_lattice(self.handle, ctypes.byref(LS), ctypes.byref(LQ),
                                    ctypes.byref(r), ctypes.byref(c), ctypes.byref(ld),
                                    ctypes.byref(st)), "swa_sat_lattice")
        if not st.value:
            return 0, None, None
        return (st.value, _view_u64(LS.value, r.value, c.value, ld.value),
                _view_u64(LQ.value, r.value, c.value, ld.value))

    def sync(self):
        check(lib().swa_sync(self.handle), "swa_sync")

    def status(self):
        """The build's status code (SWA_OK or SWA_ETIMEOUT) without waiting:
        call it only once the build is known to have finished."""
        return int(lib().swa_sat_status(self.handle))

    def free(self):
        if self.handle:
            lib().swa_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def verify_tables(image, S, Q=None, stream=None):
    """Check tables against a 2-D uint8/uint16 CUDA image on the device by
    the summed-area recurrence (see swa_verify_tables): returns (S entries
    failing, Q entries failing, smallest failing flat index or None).  S and
    Q are int64 views (uint64 bit patterns) with unit column stride, e.g.
    from SAT.tables() or Batch.tables()."""
    import torch
    assert image.is_cuda and image.dim() == 2 and image.stride(1) == 1
    rows, cols = image.shape
    assert S.shape == (rows, cols) and S.stride(1) == 1
    if Q is not None:
        assert Q.shape == (rows, cols) and Q.stride(1) == 1 and Q.stride(0) == S.stride(0)
    counts = torch.empty(3, dtype=torch.int64, device=image.device)
    check(lib().swa_verify_tables(image.data_ptr(), rows, cols,
                                  image.stride(0) * image.element_size(), _dtype_code(image),
                                  S.data_ptr(), None if Q is None else Q.data_ptr(), S.stride(0),
                                  counts.data_ptr(), _stream_ptr(stream)), "swa_verify_tables")
    c = counts.cpu().tolist()
    return c[0], c[1], (None if c[2] == -1 else c[2])


def _view_u64(ptr, rows, cols, ld):
    """A torch view of device memory the library owns: int64 elements holding
    the uint64 bit patterns (torch has few uint64 operations)."""
    import torch

    class _Arr:
        def __init__(self):
            self.__cuda_array_interface__ = {
                "shape": (rows, cols), "typestr": "<i8", "data": (ptr, False),
                "strides": (ld * 8, 8), "version": 3}
    return torch.as_tensor(_Arr(), device="cuda")


def build_sat(image, with_sq=True, twopass=False, stream=None, lattice=0) -> SAT:
    """Build S (and Q) of a 2-D uint8/uint16 CUDA tensor (row stride may exceed
    its width).  ``lattice=s`` (8..255) also keeps the corner lattice of
    stride s, which serves window queries at strides (s, s) whose sides are
    multiples of s (see SWA_LATTICE in swa.h)."""
    assert image.is_cuda and image.dim() == 2 and image.stride(1) == 1
    rows, cols = image.shape
    h = _VP()
    flags = (SWA_WITH_SQ if with_sq else 0) | (SWA_TWOPASS if twopass else 0) | (
        int(lattice) << SWA_LATTICE_SHIFT)
    check(lib().swa_build_sat(image.data_ptr(), rows, cols, image.stride(0) * image.element_size(),
                              _dtype_code(image), flags, _stream_ptr(stream), ctypes.byref(h)),
          "swa_build_sat")
    return SAT(h.value, rows, cols, with_sq, stream)


def build_count_sat(image, threshold, stream=None) -> SAT:
    """The table of the 0/1 indicator "pixel > threshold" of a 2-D
    uint8/uint16 CUDA tensor: window_stats on it gives per window the count of
    pixels above the threshold ("sum"), their fraction ("mean") and the
    indicator's std ("std")."""
    assert image.is_cuda and image.dim() == 2 and image.stride(1) == 1
    rows, cols = image.shape
    h = _VP()
    check(lib().swa_build_count_sat(image.data_ptr(), rows, cols,
                                    image.stride(0) * image.element_size(), _dtype_code(image),
                                    int(threshold), _stream_ptr(stream), ctypes.byref(h)),
          "swa_build_count_sat")
    return SAT(h.value, rows, cols, True, stream)


def analyze(image, windows, outputs=("sum", "mean", "std"), out=None, stream=None,
            band_rows=None):
    """One request end to end through ``swa_analyze``: image and outputs may
    live in host (ideally pinned) or device memory.  Returns the output dicts
    (allocated like the image when ``out`` is None).  With ``band_rows`` (0
    for automatic) the request goes through ``swa_analyze_banded`` instead:
    tables are built band by band, for images whose tables exceed device
    memory or the uint64 bound."""
    import torch
    rows, cols = image.shape
    mask = (SWA_OUT_SUM if "sum" in outputs else 0) | (
        SWA_OUT_MEAN if "mean" in outputs else 0) | (SWA_OUT_STD if "std" in outputs else 0)
    arr = (swa_window * len(windows))()
    res = []
    for k, (wh, ww, sy, sx) in enumerate(windows):
        R, C = window_shape(rows, cols, wh, ww, sy, sx)
        if out is not None:
            o = out[k]
        else:
            kw = dict(device=image.device, pin_memory=not image.is_cuda)
            o = {}
            if mask & SWA_OUT_SUM:
                o["sum"] = torch.empty((R, C), dtype=torch.int64, **kw)
            if mask & SWA_OUT_MEAN:
                o["mean"] = torch.empty((R, C), dtype=torch.float64, **kw)
            if mask & SWA_OUT_STD:
                o["std"] = torch.empty((R, C), dtype=torch.float64, **kw)
        ld = next(iter(o.values())).stride(0)
        arr[k] = swa_window(wh, ww, sy, sx, mask, 0,
                            o["sum"].data_ptr() if "sum" in o else None,
                            o["mean"].data_ptr() if "mean" in o else None,
                            o["std"].data_ptr() if "std" in o else None, ld)
        res.append(o)
    if band_rows is None:
        check(lib().swa_analyze(image.data_ptr(), rows, cols,
                                image.stride(0) * image.element_size(), _dtype_code(image), arr,
                                len(windows), _stream_ptr(stream)), "swa_analyze")
    else:
        check(lib().swa_analyze_banded(image.data_ptr(), rows, cols,
                                       image.stride(0) * image.element_size(),
                                       _dtype_code(image), arr, len(windows), int(band_rows),
                                       _stream_ptr(stream)), "swa_analyze_banded")
    return res


def band_range(rows, wh, sy, band_rows, b):
    """Output rows [i_begin, i_end) that band b of swa_analyze_banded serves
    (host only)."""
    ib, ie = _I64(), _I64()
    check(lib().swa_band_range(rows, wh, sy, band_rows, b, ctypes.byref(ib), ctypes.byref(ie)),
          "swa_band_range")
    return ib.value, ie.value


class Batch:
    """A batched plan: many images with their window queries, built and
    queried by one persistent launch per ``run`` (see swa_batch_create).

    images: list of 2-D uint8/uint16 (or int16 bit-pattern) CUDA tensors.
    windows: list (per image) of [(wh, ww, sy, sx), ...].
    Outputs are allocated here (device tensors, like SAT.window_stats) unless
    ``out`` supplies them.
    """

    def __init__(self, images, windows, outputs=("sum", "mean", "std"), u8_tile_rows=64,
                 order=0, stream=None, out=None, ticket_order=0, lookback=0, warps=0,
                 interleave=0):
        import torch
        mask = (SWA_OUT_SUM if "sum" in outputs else 0) | (
            SWA_OUT_MEAN if "mean" in outputs else 0) | (SWA_OUT_STD if "std" in outputs else 0)
        self.images = list(images)
        self.outputs = []
        self._wins = []
        items = (swa_batch_item * len(self.images))()
        for k, (img, wl) in enumerate(zip(self.images, windows)):
            assert img.is_cuda and img.dim() == 2 and img.stride(1) == 1
            rows, cols = img.shape
            arr = (swa_window * max(1, len(wl)))()
            res = []
            for q, (wh, ww, sy, sx) in enumerate(wl):
                R, C = window_shape(rows, cols, wh, ww, sy, sx)
                if out is not None:
                    o = out[k][q]
                else:
                    o = {}
                    if mask & SWA_OUT_SUM:
                        o["sum"] = torch.empty((R, C), dtype=torch.int64, device=img.device)
                    if mask & SWA_OUT_MEAN:
                        o["mean"] = torch.empty((R, C), dtype=torch.float64, device=img.device)
                    if mask & SWA_OUT_STD:
                        o["std"] = torch.empty((R, C), dtype=torch.float64, device=img.device)
                ld = next(iter(o.values())).stride(0)
                arr[q] = swa_window(wh, ww, sy, sx, mask, 0,
                                    o["sum"].data_ptr() if "sum" in o else None,
                                    o["mean"].data_ptr() if "mean" in o else None,
                                    o["std"].data_ptr() if "std" in o else None, ld)
                res.append(o)
            self._wins.append(arr)
            self.outputs.append(res)
            items[k] = swa_batch_item(img.data_ptr(), rows, cols,
                                      img.stride(0) * img.element_size(), _dtype_code(img),
                                      len(wl), arr)
        cfg = swa_batch_config(u8_tile_rows, order, ticket_order, lookback, warps, interleave)
        h = _VP()
        self.stream = stream
        check(lib().swa_batch_create(items, len(self.images), ctypes.byref(cfg),
                                     _stream_ptr(stream), ctypes.byref(h)), "swa_batch_create")
        self.handle = h.value

    def run(self, stream=None):
        check(lib().swa_batch_run(self.handle, _stream_ptr(stream if stream is not None
                                                           else self.stream)), "swa_batch_run")

    def sync(self):
        check(lib().swa_batch_sync(self.handle), "swa_batch_sync")

    def nbytes(self):
        return int(lib().swa_batch_bytes(self.handle))

    def tables(self, k):
        """(S, Q) int64 views (uint64 bit patterns) of image k's tables."""
        S, Q, ld = _VP(), _VP(), _I64()
        check(lib().swa_batch_tables(self.handle, k, ctypes.byref(S), ctypes.byref(Q),
                                     ctypes.byref(ld)), "swa_batch_tables")
        rows, cols = self.images[k].shape
        return _view_u64(S.value, rows, cols, ld.value), _view_u64(Q.value, rows, cols, ld.value)

    def free(self):
        if self.handle:
            lib().swa_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
