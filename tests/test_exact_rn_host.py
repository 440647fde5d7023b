"""The CUDA path's integer round-to-nearest helpers (exact_rn.cuh), built for
the host and compared bit for bit with the oracle's IEEE double arithmetic
(CPU only).  The same code runs in the window kernel on the GPU."""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_rn(seed_ulps=None):
    """The helpers built for the host; seed_ulps pushes the square root's
    reciprocal-square-root seed by that many ulp (the device's rsqrtf is
    within 2 ulp)."""
    tag = "" if seed_ulps is None else "_%+d" % seed_ulps
    out = os.path.join(tempfile.mkdtemp(), "exact_rn_host%s.so" % tag)
    extra = [] if seed_ulps is None else ["-DSWA_RSQRT_TEST_ULPS=(%d)" % seed_ulps]
    subprocess.check_call([
        "g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
        *extra, "-I", os.path.join(ROOT, "paper_2410_16291_gb300", "csrc"),
        os.path.join(ROOT, "tests", "exact_rn_host.cpp"), "-o", out])
    L = ctypes.CDLL(out)
    vp = ctypes.c_void_p
    L.rn_stats_bulk.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    L.rn_std64_bulk.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
    L.rn_u128.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.rn_u128.restype = ctypes.c_double
    L.rn_sqrt.argtypes = [ctypes.c_double]
    L.rn_sqrt.restype = ctypes.c_double
    L.rn_div.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
    L.rn_div.restype = ctypes.c_double
    return L


@pytest.fixture(scope="module")
def rn():
    return build_rn()


def run_bulk(rn, n, sw, qw):
    n, sw, qw = (np.ascontiguousarray(a, dtype=np.uint64) for a in (n, sw, qw))
    m = np.empty(len(n))
    s = np.empty(len(n))
    rn.rn_stats_bulk(n.ctypes.data, sw.ctypes.data, qw.ctypes.data, len(n), m.ctypes.data,
                     s.ctypes.data)
    return m, s


def moments(rng, count, nmax, vmax):
    """Random valid (n, Sw, Qw): Qw in [ceil(Sw^2/n), Sw*vmax]."""
    n = rng.integers(1, nmax + 1, count, dtype=np.uint64)
    sw = (rng.random(count) * n.astype(float) * vmax).astype(np.uint64)
    lo = np.array([-(-int(a) * int(a) // int(b)) for a, b in zip(sw, n)], dtype=object)
    hi = np.array([max(int(a) * vmax, l) for a, l in zip(sw, lo)], dtype=object)
    f = rng.random(count)
    qw = np.array([int(l + (h - l) * x) for l, h, x in zip(lo, hi, f)], dtype=np.uint64)
    return n, sw, qw


@pytest.mark.parametrize("nmax,vmax", [(1024 ** 2, 255), (1024 ** 2, 65535), (2 ** 32 - 1, 255),
                                       (2 ** 32 - 1, 65535), (64, 65535), (4, 3)])
def test_stats_bitexact_random(rn, nmax, vmax):
    rng = np.random.default_rng(nmax ^ vmax)
    n, sw, qw = moments(rng, 20000, nmax, vmax)
    m0, s0 = oracle.stats_bulk(n, sw, qw)
    m1, s1 = run_bulk(rn, n, sw, qw)
    np.testing.assert_array_equal(m1, m0)
    np.testing.assert_array_equal(s1, s0)


def test_stats_window_areas_and_edges(rn):
    """Square windows of every side 1..1024 with constant, two-valued and
    extreme moments."""
    ns, sws, qws = [], [], []
    for w in range(1, 1025):
        n = w * w
        for v in (0, 1, 255, 65535):
            ns.append(n); sws.append(n * v); qws.append(n * v * v)          # constant: D = 0
        for k in (1, n // 3, n // 2, n - 1):
            if 0 < k < n:                                                      # k of 65535, rest 0
                ns.append(n); sws.append(k * 65535); qws.append(k * 65535 ** 2)
                ns.append(n); sws.append(k * 255 + (n - k)); qws.append(k * 255 ** 2 + (n - k))
    m0, s0 = oracle.stats_bulk(ns, sws, qws)
    m1, s1 = run_bulk(rn, ns, sws, qws)
    np.testing.assert_array_equal(m1, m0)
    np.testing.assert_array_equal(s1, s0)


def test_u128_rounding_ties_to_even(rn):
    vals = [1, 2**53 - 1, 2**53 + 1, 2**53 + 3, 2**54 + 2, 2**54 + 6, 2**64 - 1, 2**64 + 2**11,
            2**64 + 3 * 2**11, 2**64 + 2**11 + 1, 2**100 + 2**47, 2**100 + 3 * 2**47,
            2**127 + 2**74, 2**127 + 2**74 + 1, 2**128 - 1]
    rng = np.random.default_rng(3)
    for _ in range(20000):
        b = int(rng.integers(1, 128))
        vals.append(int.from_bytes(rng.bytes(16), "little") >> (128 - b))
    for v in vals:
        assert rn.rn_u128(v >> 64, v & (2**64 - 1)) == float(v), v


def test_sqrt_correctly_rounded(rn):
    rng = np.random.default_rng(11)
    xs = list(rng.random(20000) * 2.0 ** rng.integers(-60, 120, 20000))
    xs += [float(k * k) for k in range(1, 3000)] + [float(k * k + 1) for k in range(1, 3000)]
    xs += [2.0 ** e for e in range(-60, 120)] + [math.nextafter(2.0 ** e, 0) for e in range(-50, 100)]
    for x in xs:
        if x > 0:
            assert rn.rn_sqrt(x) == math.sqrt(x), x


def test_division_correctly_rounded(rn):
    rng = np.random.default_rng(12)
    for _ in range(30000):
        n = int(rng.integers(1, 2**32))
        a = int(rng.integers(0, 2**63)) >> int(rng.integers(0, 63))
        want = float(a) / float(n)
        assert rn.rn_div(a, n) == want, (a, n)


def test_division_by_powers_of_two_is_exact(rn):
    rng = np.random.default_rng(13)
    for k in range(32):
        n = 1 << k
        for _ in range(300):
            a = int(rng.integers(0, 2**63)) >> int(rng.integers(0, 63))
            assert rn.rn_div(a, n) == float(a) / float(n), (a, n)


@pytest.mark.parametrize("vmax", [1, 255, 65535])
def test_std_64bit_variant_equals_128bit_path(rn, vmax):
    """std_rn64 (D formed in 64 bits, used when n * vmax < 2^32) gives the
    same bits as std_rn and the oracle for windows up to that bound,
    including the largest n it is used for."""
    rng = np.random.default_rng(vmax)
    nmax = (2 ** 32 - 1) // vmax
    n, sw, qw = moments(rng, 20000, nmax, vmax)
    n[:3] = nmax
    sw[:3] = [0, nmax * vmax, nmax * vmax // 2]
    qw[:3] = [0, nmax * vmax * vmax, (nmax * vmax // 2) * vmax]
    s64 = np.empty(len(n))
    rn.rn_std64_bulk(np.ascontiguousarray(n).ctypes.data, np.ascontiguousarray(sw).ctypes.data,
                     np.ascontiguousarray(qw).ctypes.data, len(n), s64.ctypes.data)
    _, s128 = run_bulk(rn, n, sw, qw)
    np.testing.assert_array_equal(s64, s128)
    _, want = oracle.stats_bulk(n, sw, qw)
    np.testing.assert_array_equal(s64, want)


def near_midpoints(count, seed):
    """Doubles whose square root lies within 1/32 of a midpoint between two
    doubles: sig * 2^52 close to (R + 1/2)^2 for a 53-bit R.  There the last
    Newton step can stop on the wrong neighbour and the final step to the
    nearest integer has to move it (with a seed 2-4 ulp off, dropping either
    direction of that step fails on these inputs)."""
    import random
    from fractions import Fraction
    r = random.Random(seed)
    xs = []
    while len(xs) < count:
        R = r.randrange(2**52, 2**53)
        Mx = round(Fraction((2 * R + 1) ** 2, 2**54))
        if 2**52 <= Mx < 2**54 and abs(Mx * 2**52 - (R * R + R)) < 2**49:
            xs.append(math.ldexp(float(Mx), r.randrange(-40, 40) * 2 - 52))
    return xs


@pytest.mark.parametrize("ulps", [-4, -2, 2, 4])
def test_sqrt_and_std_with_a_perturbed_seed(ulps):
    """The square root stays correctly rounded, and std bit-exact, when the
    reciprocal-square-root seed is off by 2 or 4 ulp either way (the device's
    rsqrtf is within 2): the Newton corrections and the final step to the
    nearest integer absorb it, also on inputs next to rounding midpoints."""
    L = build_rn(ulps)
    for x in near_midpoints(20000, 7):
        assert L.rn_sqrt(x) == math.sqrt(x), x
    rng = np.random.default_rng(100 + ulps)
    xs = list(rng.random(20000) * 2.0 ** rng.integers(-60, 120, 20000))
    xs += [float(k * k) for k in range(1, 3000)] + [float(k * k + 1) for k in range(1, 3000)]
    xs += [float(k * k - 1) for k in range(2, 3000)]
    xs += [2.0 ** e for e in range(-60, 120)] + [math.nextafter(2.0 ** e, 0) for e in range(-50, 100)]
    xs += [math.nextafter(2.0 ** e, math.inf) for e in range(-50, 100)]
    for x in xs:
        if x > 0:
            assert L.rn_sqrt(x) == math.sqrt(x), x
    for nmax, vmax in [(1024 ** 2, 255), (2 ** 32 - 1, 65535), (64, 65535)]:
        n, sw, qw = moments(rng, 20000, nmax, vmax)
        m0, s0 = oracle.stats_bulk(n, sw, qw)
        m1, s1 = run_bulk(L, n, sw, qw)
        np.testing.assert_array_equal(m1, m0)
        np.testing.assert_array_equal(s1, s0)
