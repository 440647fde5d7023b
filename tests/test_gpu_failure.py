"""Failure detection without a GPU fault: the single-pass build's bounded
look-back waits expire when a predecessor never publishes (a test hook keeps
the first tile silent), the kernel exits, and the status is reported."""
import numpy as np
import pytest

import paper_2410_16291_gb300 as swa
from gpu_util import require_gpu, to_device, u64

pytestmark = pytest.mark.gpu


def test_lookback_timeout_reports_etimeout_and_recovers():
    require_gpu()
    import torch
    from paper_2410_16291_gb300 import build
    build.build()
    img = np.random.default_rng(5).integers(0, 256, (300, 700)).astype(np.uint8)
    dev = to_device(img)
    L = swa.lib()
    L.swa_set_test_hooks(swa.SWA_HOOK_STALL_TILE0)
    try:
        sat = swa.build_sat(dev)
        with pytest.raises(swa.SwaError) as ei:
            sat.sync()
        assert ei.value.status == swa.SWA_ETIMEOUT
        sat.free()
    finally:
        L.swa_set_test_hooks(0)
    # the context is still usable and the next build is correct
    torch.cuda.synchronize()
    sat = swa.build_sat(dev)
    sat.sync()
    S, _ = sat.tables()
    assert int(u64(S[-1:, -1:])[0, 0]) == int(img.astype(np.uint64).sum())
    sat.free()
