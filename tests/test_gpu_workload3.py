"""The batched workload at its stated size: 256 uneven images (sides
512-8192, aspect 0.5-2, uint8/uint16 half and half), each with 1-4 windows of
16-512 px at strides 1-8, built and queried by the batched engine with the
autotuned configuration, replayed from a captured CUDA graph.

- On the device, every table entry and every output equals a per-image
  ``swa_build_sat`` + ``swa_window_stats`` run, bit for bit, and every
  table entry satisfies the summed-area recurrence with the image
  (``swa_verify_tables``).
- Against the oracle: each image's last table entries equal its totals,
  four table rows per image equal the oracle's streamed rows, and every one
  of the 2.29e9 window outputs (sum, mean, std) equals the oracle's
  streamed-rows windows, bit for bit.
"""
import numpy as np
import pytest

import full_parity
import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import require_gpu, u64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def test_workload3_batch_every_table_and_window():
    require_gpu()
    import torch
    from paper_2410_16291_gb300 import build, tune
    build.build()
    imgs = synth.workload(3)
    assert len(imgs) == 256
    host = [im.generate() for im in imgs]
    devs = [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
            for a in host]
    wins = [[(w.wh, w.ww, w.sy, w.sx) for w in im.windows] for im in imgs]
    cfg = tune.tune(devs, wins, use_cache=False)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = swa.Batch(devs, wins, stream=s, **cfg)
        b.run(s)                                   # warm-up outside the capture
    s.synchronize()
    b.sync()
    for o in b.outputs:                            # every output must be rewritten
        for d in o:
            for t in d.values():
                t.fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    g.replay()
    torch.cuda.synchronize()
    b.sync()

    # Device: the batch equals the per-image path, table entry by table entry
    # and output by output.
    n_out = 0
    for k, dev in enumerate(devs):
        sat = swa.build_sat(dev)
        S, Q = sat.tables()
        bS, bQ = b.tables(k)
        assert torch.equal(S, bS) and torch.equal(Q, bQ), k
        assert swa.verify_tables(dev, bS, bQ) == (0, 0, None), k
        for q, (got, ref) in enumerate(zip(b.outputs[k], sat.window_stats(wins[k]))):
            for key in ("sum", "mean", "std"):
                assert torch.equal(got[key], ref[key]), (k, q, key)
            n_out += ref["sum"].numel()
        del S, Q, bS, bQ
        sat.free()
    torch.cuda.synchronize()

    # Oracle: totals, four streamed table rows per image, every window.
    rng = np.random.default_rng(303)
    for k, a in enumerate(host):
        r = a.shape[0]
        rows = sorted(set([0, r - 1] + rng.integers(0, r, 2).tolist()))
        S_ref, Q_ref = oracle.sat_rows(a, rows)
        bS, bQ = b.tables(k)
        np.testing.assert_array_equal(u64(bS[rows]), S_ref, err_msg=str(k))
        np.testing.assert_array_equal(u64(bQ[rows]), Q_ref, err_msg=str(k))
        tot_s, tot_q = oracle.total(a)
        assert int(S_ref[-1, -1]) == tot_s and int(Q_ref[-1, -1]) == tot_q, k
    checked = full_parity.check_many(list(zip(host, wins, b.outputs)), rows_per_chunk=512)
    assert checked == n_out == sum(
        ((im.rows - w.wh) // w.sy + 1) * ((im.cols - w.ww) // w.sx + 1)
        for im in imgs for w in im.windows)
    b.free()
