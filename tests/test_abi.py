"""The C ABI: the library builds, loads and exports every declared entry
point, and host-side argument checks answer without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2410_16291_gb300 as swa
from paper_2410_16291_gb300 import build as swa_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swa.h")


@pytest.fixture(scope="module")
def L():
    swa_build.build()
    return swa.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swa_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ("swa_build_sat", "swa_window_stats", "swa_free", "swa_window_shape",
              "swa_sat_data", "swa_sync", "swa_status_str"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.check_output(["nm", "-D", "--defined-only", swa.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # only the ABI is exported (the static CUDA runtime stays hidden)
    assert all(n.startswith("swa_") for n in exported if not n.startswith("_")), \
        sorted(n for n in exported if not n.startswith("swa_"))[:10]
    assert set(swa.SIGNATURES) <= set(declared_functions())


def test_status_strings_and_version(L):
    for s in range(6):
        assert L.swa_status_str(s)
    assert L.swa_version() == 10000


def test_window_shape_host_only(L):
    assert swa.window_shape(1024, 1024, 32, 32, 1, 1) == (993, 993)
    assert swa.window_shape(70000, 85000, 1024, 1024, 16, 16) == (4312, 5249)
    R, C = ctypes.c_int64(), ctypes.c_int64()
    for bad in [(10, 10, 11, 1, 1, 1), (10, 10, 1, 11, 1, 1), (10, 10, 2, 2, 0, 1),
                (0, 10, 1, 1, 1, 1), (10, 10, 0, 1, 1, 1)]:
        assert L.swa_window_shape(*bad, ctypes.byref(R), ctypes.byref(C)) == swa.SWA_EINVAL


def test_build_argument_checks_before_any_device_work(L):
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails first
    assert L.swa_build_sat(None, 10, 10, 10, swa.SWA_U8, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 0, 10, 10, swa.SWA_U8, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 10, 10, 9, swa.SWA_U8, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 10, 10, 19, swa.SWA_U16, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 10, 10, 10, 3, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 10, 10, 21, swa.SWA_U16, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    odd = ctypes.c_void_p(0x1001)
    assert L.swa_build_sat(odd, 10, 10, 20, swa.SWA_U16, 0, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 10, 10, 10, swa.SWA_U8, 8, None, ctypes.byref(h)) == swa.SWA_EINVAL
    assert L.swa_build_sat(fake, 10, 10, 10, swa.SWA_U8, 0, None, None) == swa.SWA_EINVAL
    # the u16 squared table of a 70,000 x 85,000 image could overflow uint64
    assert L.swa_build_sat(fake, 70000, 85000, 170000, swa.SWA_U16, swa.SWA_WITH_SQ, None,
                           ctypes.byref(h)) == swa.SWA_EOVERFLOW
    assert L.swa_build_sat(fake, 184252, 23311, 2 * 23311, swa.SWA_U16, swa.SWA_WITH_SQ, None,
                           ctypes.byref(h)) == swa.SWA_EOVERFLOW
    # a memory limit of zero refuses the build before allocating
    L.swa_set_memory_limit(0)
    try:
        assert L.swa_build_sat(fake, 100, 100, 100, swa.SWA_U8, 1, None,
                               ctypes.byref(h)) == swa.SWA_ENOMEM
    finally:
        L.swa_set_memory_limit(-1)
    assert h.value is None


def test_handle_checks(L):
    assert L.swa_window_stats(None, 2, 2, 1, 1, 1, None, None, None, 1, None) == swa.SWA_EINVAL
    assert L.swa_sync(None) == swa.SWA_EINVAL
    assert L.swa_sat_status(None) == swa.SWA_EINVAL
    assert L.swa_sat_data(None, None, None, None) == swa.SWA_EINVAL
    bogus = ctypes.c_void_p(0xdeadbeef)
    assert L.swa_sync(bogus) == swa.SWA_EINVAL          # not a live handle: never read
    L.swa_free(None)
    L.swa_free(bogus)                                      # ignored, not dereferenced


def test_sat_bytes(L):
    t, s = ctypes.c_int64(), ctypes.c_int64()
    assert L.swa_sat_bytes(70000, 85000, swa.SWA_U8, swa.SWA_WITH_SQ, ctypes.byref(t),
                           ctypes.byref(s)) == swa.SWA_OK
    ld = (85000 + 31) // 32 * 32
    assert t.value == 2 * 8 * 70000 * ld
    assert s.value < t.value // 16


def test_test_hooks_validate(L):
    assert L.swa_set_test_hooks(0) == swa.SWA_OK
    assert L.swa_set_test_hooks(swa.SWA_HOOK_BAND_BUFFERS) == swa.SWA_OK
    assert L.swa_set_test_hooks(0) == swa.SWA_OK
    assert L.swa_set_test_hooks(swa.SWA_HOOK_CORNER_MODE | swa.SWA_HOOK_ROW_ORDER) == swa.SWA_OK
    assert L.swa_set_test_hooks(0) == swa.SWA_OK
    assert L.swa_set_test_hooks(16) == swa.SWA_EINVAL


def test_batch_config_checked_on_the_host(L):
    """A batch configuration out of range is refused before any device work."""
    item = swa.swa_batch_item(ctypes.c_void_p(0x1000), 4, 4, 4, swa.SWA_U8, 0, None)
    items = (swa.swa_batch_item * 1)(item)
    h = ctypes.c_void_p()
    for bad in [dict(u8_tile_rows=48), dict(order=2), dict(ticket_order=-1), dict(lookback=2),
                dict(warps=7), dict(interleave=-1), dict(reserved=(ctypes.c_int32 * 2)(0, 1))]:
        cfg = swa.swa_batch_config(**bad)
        assert L.swa_batch_create(items, 1, ctypes.byref(cfg), None, ctypes.byref(h)) == \
            swa.SWA_EINVAL, bad
        assert h.value is None


def test_lattice_flag_checks_on_the_host(L):
    """The corner-lattice build flag is refused without Q, with the two-pass
    build or with a stride outside 8..255, before any device work; the table
    byte count includes the two lattice arrays."""
    h = ctypes.c_void_p()
    img = ctypes.c_void_p(0x1000)
    for flags in [8 << 8, swa.SWA_WITH_SQ | (7 << 8), swa.SWA_WITH_SQ | swa.SWA_TWOPASS | (16 << 8),
                  swa.SWA_WITH_SQ | (1 << 16)]:
        assert L.swa_build_sat(img, 100, 100, 100, swa.SWA_U8, flags, None,
                               ctypes.byref(h)) == swa.SWA_EINVAL, hex(flags)
        assert h.value is None
    t0, t1, sc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert L.swa_sat_bytes(70000, 85000, swa.SWA_U8, swa.SWA_WITH_SQ, ctypes.byref(t0),
                           ctypes.byref(sc)) == swa.SWA_OK
    assert L.swa_sat_bytes(70000, 85000, swa.SWA_U8, swa.SWA_WITH_SQ | (16 << 8), ctypes.byref(t1),
                           ctypes.byref(sc)) == swa.SWA_OK
    ld = (85000 // 16 + 31) // 32 * 32
    assert t1.value - t0.value == 2 * (70000 // 16) * ld * 8


def test_verify_tables_argument_checks(L):
    """Bad arguments are refused before any device work."""
    img, S = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000)
    cnt = ctypes.c_void_p(0x3000)
    assert L.swa_verify_tables(None, 4, 4, 4, swa.SWA_U8, S, None, 4, cnt, None) == swa.SWA_EINVAL
    assert L.swa_verify_tables(img, 4, 4, 4, swa.SWA_U8, S, None, 3, cnt, None) == swa.SWA_EINVAL
    assert L.swa_verify_tables(img, 4, 4, 3, swa.SWA_U8, S, None, 4, cnt, None) == swa.SWA_EINVAL
    assert L.swa_verify_tables(img, 4, 4, 8, swa.SWA_U8, S, None, 4, None, None) == swa.SWA_EINVAL
    assert L.swa_verify_tables(ctypes.c_void_p(0x1001), 4, 4, 8, swa.SWA_U16, S, None, 4, cnt,
                               None) == swa.SWA_EINVAL
