"""Seeded synthetic inputs shaped like the paper's workloads (Section IV-A).

The paper's pancreatic ductal adenocarcinoma immunofluorescence images are not
available; these generators stand in for them with the shapes, sizes and value
distributions of the five workloads listed in ``WORKLOADS``.  The module holds
input generation only (no summed-area table or window arithmetic) and is the
one piece of code shared by the CPU oracle's tests, the CUDA path's tests and
the benchmark.

The generators are written in C (``synth.c``) with a counter-based RNG, so an
image is a function of (seed, shape, parameters) only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

DEFAULT_SEED = 20241016


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, vp, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double
        lib.synth_mask_u8.argtypes = [vp, i64, i64, i64, u64, i64, dbl, dbl]
        lib.synth_mask_u8.restype = i64
        lib.synth_intensity_u8.argtypes = [vp, i64, i64, i64, u64, i64]
        lib.synth_intensity_u8.restype = ctypes.c_int
        lib.synth_intensity_u16.argtypes = [vp, i64, i64, i64, u64, i64]
        lib.synth_intensity_u16.restype = ctypes.c_int
        lib.synth_draws.argtypes = [u64, u64, u64, i64, vp]
        lib.synth_draws.restype = None
        lib.synth_exp.argtypes = [dbl]
        lib.synth_exp.restype = dbl
        lib.synth_log.argtypes = [dbl]
        lib.synth_log.restype = dbl
        lib.synth_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _out(rows, cols, dtype, out):
    if out is None:
        return np.empty((rows, cols), dtype=dtype)
    assert out.dtype == dtype and out.shape == (rows, cols) and out.strides[1] == out.itemsize
    return out


def mask_u8(rows: int, cols: int, seed: int, frac_ones: float = 0.03,
            sigma: float = 8.0, mean_children: float = 20.0, out=None) -> np.ndarray:
    """Binary cell-centroid mask: Thomas cluster process (Poisson(20) children
    per uniform parent, normal offsets of ``sigma`` px), exactly
    round(frac_ones * rows * cols) ones."""
    a = _out(rows, cols, np.uint8, out)
    n = int(round(frac_ones * rows * cols))
    got = _load().synth_mask_u8(a.ctypes.data, rows, cols, a.strides[0], seed, n,
                                sigma, mean_children)
    if got != n:
        raise RuntimeError("synth_mask_u8 produced %d ones, wanted %d" % (got, n))
    return a


def intensity_u8(rows: int, cols: int, seed: int, n_clusters: int, out=None) -> np.ndarray:
    """Gamma(2, 20) background plus Gaussian clusters (sigma 10-60 px,
    amplitude 60-200), clipped to 255."""
    a = _out(rows, cols, np.uint8, out)
    rc = _load().synth_intensity_u8(a.ctypes.data, rows, cols, a.strides[0], seed, n_clusters)
    if rc != 0:
        raise RuntimeError("synth_intensity_u8 failed (%d)" % rc)
    return a


def intensity_u16(rows: int, cols: int, seed: int, n_clusters: int, out=None) -> np.ndarray:
    """Log-normal(6, 1.5) background plus Gaussian clusters with amplitudes
    scaled by 256, clipped to 65535."""
    a = _out(rows, cols, np.uint16, out)
    rc = _load().synth_intensity_u16(a.ctypes.data, rows, cols, a.strides[0], seed, n_clusters)
    if rc != 0:
        raise RuntimeError("synth_intensity_u16 failed (%d)" % rc)
    return a


def draws(seed: int, stream: int, n: int, first: int = 0) -> np.ndarray:
    """n uniform 64-bit words of a named stream (counter-based)."""
    out = np.empty(n, dtype=np.uint64)
    _load().synth_draws(seed, stream, first, n, out.ctypes.data)
    return out


def uniforms(seed: int, stream: int, n: int, first: int = 0) -> np.ndarray:
    """n uniforms in (0, 1) from ``draws``."""
    d = draws(seed, stream, n, first)
    return ((d >> np.uint64(11)).astype(np.float64) + 0.5) / 9007199254740992.0


def num_threads() -> int:
    return int(_load().synth_num_threads())


def portable_exp(x: float) -> float:
    return float(_load().synth_exp(x))


def portable_log(x: float) -> float:
    return float(_load().synth_log(x))


# --------------------------------------------------------------- workloads --

@dataclass(frozen=True)
class Window:
    """A square or rectangular window with its strides."""
    wh: int
    ww: int
    sy: int
    sx: int


@dataclass
class Image:
    """One synthetic image of a workload: its generator and window list."""
    rows: int
    cols: int
    dtype: str                 # "u8" or "u16"
    kind: str                  # "mask" or "intensity"
    seed: int
    n_clusters: int = 0
    windows: list = field(default_factory=list)
    with_sq: bool = True       # build the squared-pixel table too
    outputs: tuple = ("sum", "mean", "std")

    @property
    def pixels(self) -> int:
        return self.rows * self.cols

    def generate(self, out=None) -> np.ndarray:
        if self.kind == "mask":
            return mask_u8(self.rows, self.cols, self.seed, out=out)
        if self.dtype == "u8":
            return intensity_u8(self.rows, self.cols, self.seed, self.n_clusters, out=out)
        return intensity_u16(self.rows, self.cols, self.seed, self.n_clusters, out=out)


def cluster_count(rows: int, cols: int) -> int:
    """Clusters per image at the density of the 20,000 x 20,000 workload
    (5,000 clusters per 4e8 px), at least one."""
    return max(1, int(round(5000 * rows * cols / 4.0e8)))


def workload(index: int, seed: int | None = None):
    """The images of workload ``index`` (0-4), in order.

    0: 1024x1024 u8 cell-centroid mask, 3% ones, window 32 stride 1, sum only.
    1: 20,000x20,000 u8 intensity, 5,000 clusters, windows 50/100/200 stride 1.
    2: 70,000x85,000 u8 intensity, 50,000 clusters, windows 256/1024 stride 16.
    3: 256 images, sides U[512, 8192] and aspect U[0.5, 2], u8/u16 50/50,
       1-4 windows of U{16..512} px with strides U{1..8}.
    4: see ``serve_requests``.
    """
    s = (DEFAULT_SEED + index) if seed is None else seed
    if index == 0:
        return [Image(1024, 1024, "u8", "mask", s, 0, [Window(32, 32, 1, 1)],
                      with_sq=False, outputs=("sum",))]
    if index == 1:
        return [Image(20000, 20000, "u8", "intensity", s, 5000,
                      [Window(w, w, 1, 1) for w in (50, 100, 200)])]
    if index == 2:
        return [Image(70000, 85000, "u8", "intensity", s, 50000,
                      [Window(w, w, 16, 16) for w in (256, 1024)])]
    if index == 3:
        return batch_images(256, s)
    raise ValueError("workload %d has no fixed image list (see serve_requests)" % index)


def batch_images(n: int, seed: int, side_lo: int = 512, side_hi: int = 8192,
                 win_lo: int = 16, win_hi: int = 512, stride_hi: int = 8):
    """Uneven images for the batched workload (configuration 3)."""
    u = uniforms(seed, 0, n * 16)
    imgs = []
    for i in range(n):
        r = u[16 * i:16 * (i + 1)]
        W = side_lo + int(r[0] * (side_hi - side_lo + 1))
        a = 0.5 + 1.5 * r[1]
        H = min(side_hi, max(side_lo, int(round(W * a))))
        dt = "u8" if r[2] < 0.5 else "u16"
        nw = 1 + int(r[3] * 4)
        wins = []
        for k in range(nw):
            w = win_lo + int(r[4 + 2 * k] * (win_hi - win_lo + 1))
            w = min(w, H, W)
            st = 1 + int(r[5 + 2 * k] * stride_hi)
            wins.append(Window(w, w, st, st))
        imgs.append(Image(H, W, dt, "intensity", seed * 1000003 + i,
                          cluster_count(H, W), wins))
    return imgs


def serve_requests(n: int, seed: int, rate_hz: float = 200.0, pool: int = 64,
                   side_lo: int = 1000, side_hi: int = 40000, zipf_s: float = 1.1,
                   max_windows: int = 8, win_lo: int = 16, win_hi: int = 1024,
                   stride_lo: int = 4, stride_hi: int = 16):
    """Poisson request stream for the served workload (configuration 4).

    Returns (pool_images, requests) where each request is
    (arrival_s, pool_index, [Window, ...]).  Pool images have square sides
    U[side_lo, side_hi], u8/u16 50/50; popularity is Zipf(zipf_s) over the
    pool; each request asks 1..max_windows windows of U{win_lo..win_hi} px
    with strides U{stride_lo..stride_hi}.
    """
    u = uniforms(seed, 1, pool * 4)
    imgs = []
    for i in range(pool):
        side = side_lo + int(u[4 * i] * (side_hi - side_lo + 1))
        dt = "u8" if u[4 * i + 1] < 0.5 else "u16"
        imgs.append(Image(side, side, dt, "intensity", seed * 7919 + i,
                          cluster_count(side, side), []))
    weights = 1.0 / np.arange(1, pool + 1) ** zipf_s
    cdf = np.cumsum(weights) / weights.sum()
    v = uniforms(seed, 2, n * (3 + 2 * max_windows))
    per = 3 + 2 * max_windows
    t = 0.0
    reqs = []
    for k in range(n):
        r = v[per * k:per * (k + 1)]
        t += -np.log(r[0]) / rate_hz
        idx = int(np.searchsorted(cdf, r[1]))
        img = imgs[idx]
        nw = 1 + int(r[2] * max_windows)
        wins = []
        for j in range(nw):
            w = win_lo + int(r[3 + 2 * j] * (win_hi - win_lo + 1))
            w = min(w, img.rows, img.cols)
            st = stride_lo + int(r[4 + 2 * j] * (stride_hi - stride_lo + 1))
            wins.append(Window(w, w, st, st))
        reqs.append((t, idx, wins))
    return imgs, reqs
