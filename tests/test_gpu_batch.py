"""The batched engine: many uneven uint8/uint16 images with their queries in
one persistent launch, bit-exact against the oracle, on repeated runs and
from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(31)


def make_case():
    shapes = [((300, 700), np.uint8, 0, 0), ((129, 257), np.uint16, 0, 0),
              ((1000, 513), np.uint8, 5, 0), ((64, 4097), np.uint16, 0, 1),
              ((777, 1300), np.uint8, 0, 8), ((5, 5), np.uint8, 0, 0),
              ((256, 256), np.uint16, 0, 0), ((2049, 300), np.uint8, 3, 1),
              ((33, 33), np.uint16, 2, 0), ((1500, 1024), np.uint8, 0, 0)]
    imgs, devs, wins = [], [], []
    for k, ((r, c), dt, pad, off) in enumerate(shapes):
        if k == 6:
            img = np.full((r, c), 65535, np.uint16)
        elif dt == np.uint8:
            img = synth.intensity_u8(r, c, 100 + k, synth.cluster_count(r, c))
        else:
            img = synth.intensity_u16(r, c, 100 + k, synth.cluster_count(r, c))
        imgs.append(img)
        devs.append(to_device(img, pad_cols=pad, offset_px=off))
        wl = []
        for _ in range(int(RNG.integers(1, 4))):
            wh = int(RNG.integers(1, min(r, 200) + 1))
            ww = int(RNG.integers(1, min(c, 200) + 1))
            st = int(RNG.integers(1, 9))
            wl.append((wh, ww, st, int(RNG.integers(1, 9))))
        wins.append(wl)
    wins[5] = [(5, 5, 1, 1)]
    return imgs, devs, wins


def check_batch(batch, imgs, wins):
    for k, img in enumerate(imgs):
        S_ref, Q_ref = oracle.sat(img)
        S, Q = batch.tables(k)
        np.testing.assert_array_equal(u64(S), S_ref)
        np.testing.assert_array_equal(u64(Q), Q_ref)
        for (wh, ww, sy, sx), got in zip(wins[k], batch.outputs[k]):
            want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx)
            np.testing.assert_array_equal(u64(got["sum"]), want["sum"])
            np.testing.assert_array_equal(f64(got["mean"]), want["mean"])
            np.testing.assert_array_equal(f64(got["std"]), want["std"])


@pytest.mark.parametrize("cfg", [
    dict(u8_tile_rows=64, order=0), dict(u8_tile_rows=32, order=1, interleave=1),
    dict(u8_tile_rows=64, order=0, ticket_order=1, lookback=1, warps=8),
    dict(u8_tile_rows=32, order=0, ticket_order=1, lookback=0, warps=9),
    dict(u8_tile_rows=64, order=1, ticket_order=0, lookback=1, warps=9),
    dict(u8_tile_rows=32, order=1, ticket_order=0, lookback=0, warps=8),
    dict(u8_tile_rows=64, order=0, interleave=4),
    dict(u8_tile_rows=64, order=1, ticket_order=1, lookback=1, interleave=1000),
    dict(u8_tile_rows=32, order=0, ticket_order=0, lookback=0, warps=8, interleave=3)],
    ids=lambda c: "-".join("%s%d" % (k[:2], v) for k, v in c.items()))
def test_batch_bitexact_and_repeatable(cfg):
    """Every configuration the autotuner may pick gives the same, exact
    tables and outputs."""
    require_gpu()
    import torch
    from paper_2410_16291_gb300 import build
    build.build()
    imgs, devs, wins = make_case()
    b = swa.Batch(devs, wins, **cfg)
    b.run()
    b.sync()
    check_batch(b, imgs, wins)
    for o in b.outputs:
        for d in o:
            for t in d.values():
                t.zero_()
    b.run()
    b.sync()
    check_batch(b, imgs, wins)
    b.free()
    torch.cuda.synchronize()


def test_batch_replayed_from_a_cuda_graph():
    require_gpu()
    import torch
    imgs, devs, wins = make_case()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = swa.Batch(devs, wins, stream=s)
        b.run(s)                      # warm-up outside capture
    s.synchronize()
    for o in b.outputs:
        for d in o:
            for t in d.values():
                t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    b.sync()
    check_batch(b, imgs, wins)
    b.free()
