"""The device's rounding paths for the standard deviation, over the ordinary
window call, bit for bit against the oracle:

- D = n*Qw - Sw^2 formed in 64 bits (n times the largest pixel value below
  2^32), in 128 bits, and the FP64 path of windows of 2^32 pixels or more;
- images drawn log-normal (uint16), two-valued {0, 65535} (D above 2^64) and
  from the uint8 generator, 4096 x 4096, windows of 1 to 1024 px at column
  strides on both sides of the dense/sparse split (1-16);
- windows built so that D lands exactly on 2^53 - 1, 2^53, 2^53 + 1,
  2^64 - 1, 2^64, 2^64 + 1 and on exact squares s^2 - 1, s^2, s^2 + 1 (the
  edges of the integer-to-double rounding and of the square root's floor).

The constructed windows rest on D = sum over pixel pairs of (v_i - v_j)^2:
pixels start as even as the sum allows, then pairs at one level are spread
symmetrically (v - d, v + d adds 2 d^2 to the sum of squares) until the sum
of squares is the one the target D asks for.
"""
import math

import numpy as np
import pytest

import full_parity
import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _release_device_memory():
    yield
    try:
        import torch
        if torch.cuda.is_available():
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            swa.lib().swa_trim(0)
    except ImportError:
        pass


def pixels_with_D(n, T, A):
    """n integers in [0, A] with n * sum(v^2) - (sum v)^2 == T, or None."""
    base = n * A // 2
    res = np.arange(n, dtype=np.int64)               # Sw mod n with Sw^2 = -T (mod n)
    for rr in np.flatnonzero((res * res + T % n) % n == 0):
        sw = base + (int(rr) - base) % n
        qt = (T + sw * sw) // n                      # the sum of squares T asks for
        if (qt - sw) % 2:                            # sum v^2 = sum v (mod 2)
            continue
        q, r = divmod(sw, n)
        e = qt - (r * (q + 1) ** 2 + (n - r) * q * q)
        if e < 0:
            continue
        vals = [q + 1] * r + [q] * (n - r)
        pairs = [(i, q + 1) for i in range(0, r - 1, 2)] + [(i, q) for i in range(r, n - 1, 2)]
        for i, L in pairs:                           # level L -> L - d, L + d: +2 d^2
            if e == 0:
                break
            d = min(L, A - L, math.isqrt(e // 2))
            if d == 0:
                break
            vals[i], vals[i + 1] = L - d, L + d
            e -= 2 * d * d
        if e == 0:
            s1 = sum(vals)
            assert n * sum(v * v for v in vals) - s1 * s1 == T and 0 <= min(vals) <= max(vals) <= A
            return vals
    return None


def window_with_D(T, A, shapes, seed):
    """A wh x ww image (the first shape that admits T) whose single window
    has D == T; pixels in a seeded random order."""
    for wh, ww in shapes:
        vals = pixels_with_D(wh * ww, T, A)
        if vals is not None:
            img = np.array(vals, dtype=np.uint8 if A == 255 else np.uint16)
            np.random.default_rng(seed).shuffle(img)
            return img.reshape(wh, ww)
    raise AssertionError("no window shape admits D = %d" % T)


def near(lo, hi):
    """Window shapes of lo..hi pixels high and up to 8 pixels wider."""
    return [(h, h + k) for h in range(lo, hi + 1) for k in range(9)]


def check_one_window(img):
    sat = swa.build_sat(to_device(img))
    r, c = img.shape
    (o,) = sat.window_stats([(r, c, 1, 1)])
    s, q, m, d = oracle.window_one(img, 0, 0, r, c)
    assert int(u64(o["sum"])[0, 0]) == s
    assert f64(o["mean"])[0, 0] == m
    assert f64(o["std"])[0, 0] == d, (img.shape, f64(o["std"])[0, 0], d)
    sat.free()
    return s, q


SQ = [2**26 + 12345, 3 * 2**28 + 1, 2**33 + 7, 2**35 + 1]


# (pixel type, target D, smallest and largest window height to try).  An odd
# D needs an even window area (for odd n, D = n Qw - Sw^2 is even) and -D a
# square modulo n, so a range of shapes is searched for one that admits it.
CASES = [
    # uint16, D in 64 bits (n * 65535 < 2^32: n <= 65536)
    ("u16", 2**53 - 1, 60, 100), ("u16", 2**53, 60, 100), ("u16", 2**53 + 1, 60, 100),
    ("u16", SQ[0] ** 2 - 1, 60, 100), ("u16", SQ[0] ** 2, 60, 100),
    ("u16", SQ[0] ** 2 + 1, 60, 100),
    ("u16", SQ[1] ** 2 - 1, 160, 240), ("u16", SQ[1] ** 2, 160, 240),
    ("u16", SQ[1] ** 2 + 1, 160, 240),
    # uint16, D in 128 bits (n > 65536)
    ("u16", 2**53 - 1, 260, 300), ("u16", 2**53 + 1, 260, 300),
    ("u16", 2**64 - 1, 370, 420), ("u16", 2**64, 370, 420), ("u16", 2**64 + 1, 370, 420),
    ("u16", SQ[2] ** 2 - 1, 520, 560), ("u16", SQ[2] ** 2, 520, 560),
    ("u16", SQ[2] ** 2 + 1, 520, 560),
    ("u16", SQ[3] ** 2 - 1, 1030, 1060), ("u16", SQ[3] ** 2 + 1, 1030, 1060),
    # uint8, D in 64 bits (every window up to 4096 x 4096)
    ("u8", 2**53 - 1, 870, 920), ("u8", 2**53 + 1, 870, 920),
    ("u8", SQ[0] ** 2 - 1, 730, 780), ("u8", SQ[0] ** 2 + 1, 730, 780),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-D%#x" % (c[0], c[1]))
def test_constructed_D_edges(case):
    require_gpu()
    dt, T, lo, hi = case
    A = 255 if dt == "u8" else 65535
    img = window_with_D(T, A, near(lo, hi), seed=T % 1000)
    n = img.size
    assert (n * A < 2**32) == (dt == "u8" or hi <= 240)    # the path the case is meant for
    s, q = check_one_window(img)
    assert n * q - s * s == T


def near_midpoint_D(count, seed, scale):
    """Integers D = Mx * 4^scale whose square root lies within 1/32 of a
    midpoint between two doubles (Mx * 2^52 close to (R + 1/2)^2 for a
    53-bit R): where the square root's last Newton step can stop on the
    wrong neighbour and the final step to the nearest has to move it."""
    import random
    from fractions import Fraction
    r = random.Random(seed)
    out = []
    while len(out) < count:
        R = r.randrange(2**52, 2**53)
        Mx = round(Fraction((2 * R + 1) ** 2, 2**54))
        if 2**52 <= Mx < 2**54 and abs(Mx * 2**52 - (R * R + R)) < 2**49:
            out.append(Mx << (2 * scale))
    return out


@pytest.mark.parametrize("path,scale,lo,hi", [("int64", 0, 64, 100), ("int128", 4, 300, 340)])
def test_sqrt_near_rounding_midpoints(path, scale, lo, hi):
    """Windows whose D has a square root next to a rounding midpoint, through
    the device's rsqrtf-seeded square root, bit for bit against the oracle."""
    require_gpu()
    for k, T in enumerate(near_midpoint_D(8, 61 + scale, scale)):
        img = window_with_D(T, 65535, near(lo, hi), seed=k)
        assert (img.size * 65535 < 2**32) == (path == "int64")
        s, q = check_one_window(img)
        assert img.size * q - s * s == T


def two_valued(r, c, seed):
    """{0, 65535} pixels with the share of 65535 varying across the image."""
    rng = np.random.default_rng(seed)
    p = np.linspace(0.02, 0.98, c)[None, :] * np.ones((r, 1))
    return np.where(rng.random((r, c)) < p, 65535, 0).astype(np.uint16)


WINDOWS = [(1, 1, 1, 1), (2, 3, 1, 2), (3, 3, 3, 3), (7, 5, 2, 4), (16, 16, 1, 1),
           (64, 64, 3, 3), (255, 257, 1, 2), (256, 256, 8, 8), (257, 255, 16, 16),
           (512, 512, 5, 5), (1000, 1000, 16, 16), (1024, 1024, 1, 1), (1024, 1024, 2, 16)]


@pytest.mark.parametrize("kind", ["u16_lognormal", "u16_two_valued", "u8"])
def test_every_window_4096(kind):
    """Every window of 13 sizes and strides on a 4096 x 4096 image, bit for
    bit: the 64-bit-D path (uint16 windows up to 256 x 256, every uint8
    window here), the 128-bit-D path (larger uint16 windows; two-valued
    images push D above 2^64) and both column-stride kernels."""
    require_gpu()
    if kind == "u16_lognormal":
        img = synth.intensity_u16(4096, 4096, 9001, synth.cluster_count(4096, 4096))
    elif kind == "u16_two_valued":
        img = two_valued(4096, 4096, 9002)
    else:
        img = synth.intensity_u8(4096, 4096, 9003, synth.cluster_count(4096, 4096))
    sat = swa.build_sat(to_device(img))
    res = sat.window_stats(WINDOWS)
    n = full_parity.check_all_windows(img, WINDOWS, res, rows_per_chunk=512)
    assert n == sum(swa.window_shape(4096, 4096, *w)[0] * swa.window_shape(4096, 4096, *w)[1]
                    for w in WINDOWS)
    sat.free()


@pytest.mark.slow
def test_fp64_path_for_windows_of_2_pow_32_pixels():
    """Windows of 65536 x 65536 = 2^32 pixels and more take the FP64
    division and square root: a 65,536 x 65,600 uint8 image (4.3e9 px, 69 GB
    of tables), every window of three such queries against the oracle's
    streamed rows."""
    require_gpu()
    import torch
    block = synth.intensity_u8(4096, 4100, 9004, synth.cluster_count(4096, 4100))
    img = np.tile(block, (16, 16))                   # 65,536 x 65,600
    img[::977, ::1013] = 255                          # break the tiling's periodicity
    wins = [(65536, 65536, 1, 1), (65536, 65537, 1, 7), (65535, 65599, 1, 1)]
    sat = swa.build_sat(torch.from_numpy(img).cuda())
    res = sat.window_stats(wins)
    for (wh, ww, sy, sx), got in zip(wins, res):
        want = oracle.window_rows_stream(img, wh, ww, sy, sx, np.arange(got["sum"].shape[0]))
        np.testing.assert_array_equal(u64(got["sum"]), want["sum"])
        np.testing.assert_array_equal(f64(got["mean"]), want["mean"])
        np.testing.assert_array_equal(f64(got["std"]), want["std"])
    sat.free()
