"""swa_build_sat_noalloc: the single-pass build without device allocation.

Some callers cannot allocate device memory (an application whose memory
manager owns the whole device, or code in a callback or a latency-bound loop
where an allocation is not acceptable).  For them the library builds the
tables into buffers the caller passes, with its scratch in a fixed array.
This test calls that entry point through the C ABI and checks its tables
against the regular swa_build_sat on two calls in a row (the second call
reuses the scratch the first one left behind), and that an image too large
for the fixed scratch is refused.  It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

import paper_2410_16291_gb300 as swa
from gpu_util import require_gpu, to_device, u64

pytestmark = pytest.mark.gpu


def noalloc_tables(img_dev, rows, cols, dtype_code, with_sq, with_status=True, want=0):
    """Caller-allocated tables (torch) filled by swa_build_sat_noalloc; the
    status word (starting at 7, which the call must reset) must end as
    `want`."""
    import torch
    ld = (cols + 15) // 16 * 16
    S = torch.empty((rows, ld), dtype=torch.int64, device="cuda")
    Q = torch.empty((rows, ld), dtype=torch.int64, device="cuda") if with_sq else None
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = swa.lib().swa_build_sat_noalloc(
        img_dev.data_ptr(), rows, cols, img_dev.stride(0) * img_dev.element_size(), dtype_code,
        swa.SWA_WITH_SQ if with_sq else 0, S.data_ptr(), Q.data_ptr() if with_sq else None, ld,
        status.data_ptr() if with_status else None, st)
    assert rc == swa.SWA_OK, swa.lib().swa_last_error()
    torch.cuda.synchronize()
    if with_status:
        assert int(status.item()) == want
    return S[:, :cols], (Q[:, :cols] if with_sq else None)


def test_noalloc_build_matches_regular_build_twice():
    require_gpu()
    from paper_2410_16291_gb300 import build
    build.build()
    rng = np.random.default_rng(77)
    cases = [(np.uint8, (1000, 2049), True), (np.uint16, (777, 1500), True),
             (np.uint8, (300, 513), False)]
    for dtype, (r, c), with_sq in cases:
        img = rng.integers(0, 256 if dtype == np.uint8 else 65536, (r, c)).astype(dtype)
        dev = to_device(img)
        code = swa.SWA_U8 if dtype == np.uint8 else swa.SWA_U16
        ref = swa.build_sat(dev, with_sq=with_sq)
        S_ref, Q_ref = ref.tables()
        S, Q = noalloc_tables(dev, r, c, code, with_sq)
        np.testing.assert_array_equal(u64(S), u64(S_ref))
        if with_sq:
            np.testing.assert_array_equal(u64(Q), u64(Q_ref))
        ref.free()


def test_noalloc_rejects_images_beyond_its_scratch():
    require_gpu()
    import torch
    L = swa.lib()
    dev = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    S = torch.empty((16, 16), dtype=torch.int64, device="cuda")
    # a 20,000 x 20,000 build needs far more than the fixed scratch; the call
    # refuses it before touching the (deliberately small) buffers
    rc = L.swa_build_sat_noalloc(dev.data_ptr(), 20000, 20000, 20000, swa.SWA_U8, 0,
                                 S.data_ptr(), None, 20000, None,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == swa.SWA_EINVAL
    assert b"scratch" in L.swa_last_error()


def test_noalloc_reports_an_expired_wait_and_runs_without_a_status_word():
    """With the stall hook (the first tile never publishes, so every bounded
    look-back wait runs out after about 2 s; nothing faults) the status word
    gets bit 0.  Then, hook cleared, a build with no status word at all is
    still correct."""
    require_gpu()
    rng = np.random.default_rng(78)
    img = rng.integers(0, 256, (300, 700)).astype(np.uint8)
    dev = to_device(img)
    L = swa.lib()
    L.swa_set_test_hooks(swa.SWA_HOOK_STALL_TILE0)
    try:
        noalloc_tables(dev, 300, 700, swa.SWA_U8, True, want=1)
    finally:
        L.swa_set_test_hooks(0)
    ref = swa.build_sat(dev)
    S_ref, Q_ref = ref.tables()
    S, Q = noalloc_tables(dev, 300, 700, swa.SWA_U8, True, with_status=False)
    np.testing.assert_array_equal(u64(S), u64(S_ref))
    np.testing.assert_array_equal(u64(Q), u64(Q_ref))
    ref.free()
