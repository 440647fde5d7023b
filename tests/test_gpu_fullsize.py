"""Parity at the workloads' full sizes, in the benchmark's launch
configuration: full tables where host memory allows, otherwise sampled rows
and windows the oracle computes one by one, plus invariants that hold at any
size."""
import numpy as np
import pytest

import full_parity
import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
RNG = np.random.default_rng(99)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    from paper_2410_16291_gb300 import build
    build.build()
    yield
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    swa.lib().swa_trim(0)


def sampled_windows(img, res, windows, n):
    for (wh, ww, sy, sx), got in zip(windows, res):
        R, C = got["sum"].shape
        ii = np.concatenate([[0, R - 1], RNG.integers(0, R, n)])
        jj = np.concatenate([[0, C - 1], RNG.integers(0, C, n)])
        gs = u64(got["sum"][ii, jj])
        gm, gd = f64(got["mean"][ii, jj]), f64(got["std"][ii, jj])
        for k, (i, j) in enumerate(zip(ii, jj)):
            s, _, m, d = oracle.window_one(img, int(i) * sy, int(j) * sx, wh, ww)
            assert gs[k] == s and gm[k] == m and gd[k] == d, (wh, i, j)


def test_workload1_20k():
    """20,000 x 20,000 u8: full S and Q, and every one of the 1,186,171,803
    windows (w = 50, 100, 200 at stride 1) with its sum, mean and std, bit
    for bit against the oracle; random windows also by the definition."""
    (im,) = synth.workload(1)
    img = im.generate()
    dev = to_device(img)
    sat = swa.build_sat(dev)
    wins = [(w.wh, w.ww, w.sy, w.sx) for w in im.windows]
    res = sat.window_stats(wins)
    S_ref, Q_ref = oracle.sat(img)
    S, Q = sat.tables()
    np.testing.assert_array_equal(u64(S), S_ref)
    np.testing.assert_array_equal(u64(Q), Q_ref)
    assert swa.verify_tables(dev, S, Q) == (0, 0, None)
    del S_ref, Q_ref, S, Q
    assert full_parity.check_all_windows(img, wins, res) == 1186171803
    sampled_windows(img, res, wins, 200)
    sat.free()


def test_workload2_70k_by_85k():
    """70,000 x 85,000 u8 (5.95e9 px, 95 GB of tables), built with the corner
    lattice of stride 16 as the benchmark does: every table entry checked on
    the device by the summed-area recurrence, sampled table rows streamed by
    the oracle, last entries equal the totals, the lattice equal to the
    sampled rows at its columns, every one of the 45,728,608 windows (256 and
    1024 at stride 16, served from the lattice) against the oracle's
    streamed-rows windows, sampled windows and a whole output row by the
    definition."""
    (im,) = synth.workload(2)
    img = im.generate()
    dev = to_device(img)
    sat = swa.build_sat(dev, lattice=16)       # as the benchmark builds it
    wins = [(w.wh, w.ww, w.sy, w.sx) for w in im.windows]
    res = sat.window_stats(wins)
    sat.sync()
    S, Q = sat.tables()
    # every entry of both 47.6 GB tables, on the device, by the recurrence
    assert swa.verify_tables(dev, S, Q) == (0, 0, None)
    rows = [0, 1, 127, 128, 4095, 35001, 35007, 69998, 69999]
    S_ref, Q_ref = oracle.sat_rows(img, rows)
    np.testing.assert_array_equal(u64(S[rows]), S_ref)
    np.testing.assert_array_equal(u64(Q[rows]), Q_ref)
    tot_s, tot_q = oracle.total(img)
    assert int(S_ref[-1, -1]) == tot_s and int(Q_ref[-1, -1]) == tot_q
    st, LS, LQ = sat.lattice()
    assert st == 16 and LS.shape == (4375, 5312)
    for k, y in enumerate(rows):
        if (y + 1) % 16 == 0:
            a = (y + 1) // 16 - 1
            np.testing.assert_array_equal(u64(LS[a:a + 1]), S_ref[k:k + 1, 15::16][:, :5312])
            np.testing.assert_array_equal(u64(LQ[a:a + 1]), Q_ref[k:k + 1, 15::16][:, :5312])
    assert full_parity.check_all_windows(img, wins, res, rows_per_chunk=128) == 45728608
    sampled_windows(img, res, wins, 100)
    # one whole output row of the 256 window by the definition
    got = res[0]
    i = got["sum"].shape[0] - 1
    want = oracle.window_brute(img[i * 16:i * 16 + 256], 256, 256, 16, 16)
    np.testing.assert_array_equal(u64(got["sum"][i:i + 1]), want["sum"])
    np.testing.assert_array_equal(f64(got["mean"][i:i + 1]), want["mean"])
    np.testing.assert_array_equal(f64(got["std"][i:i + 1]), want["std"])
    del S, Q
    sat.free()


def test_u16_all_max_at_the_overflow_edge():
    """The largest uint16 image whose squared table fits (7809 x 550019 px,
    all 65535): last entries are r c 65535 and r c 65535^2 (just below 2^64),
    and sampled entries are (y+1)(x+1) times the pixel (square)."""
    import torch
    r, c = 7809, 550019
    dev = torch.full((r, c), -1, dtype=torch.int16, device="cuda")   # 0xFFFF
    sat = swa.build_sat(dev)
    S, Q = sat.tables()
    assert swa.verify_tables(dev, S, Q) == (0, 0, None)          # every entry
    v = 65535
    assert int(u64(S[-1:, -1:])[0, 0]) == r * c * v
    assert int(u64(Q[-1:, -1:])[0, 0]) == r * c * v * v
    ys = RNG.integers(0, r, 50)
    xs = RNG.integers(0, c, 50)
    gs, gq = u64(S[ys, xs]), u64(Q[ys, xs])
    for k in range(50):
        n = (int(ys[k]) + 1) * (int(xs[k]) + 1)
        assert int(gs[k]) == n * v and int(gq[k]) == n * v * v
    (o,) = sat.window_stats([(7809, 550019, 1, 1)])
    assert int(u64(o["sum"])[0, 0]) == r * c * v
    assert f64(o["std"])[0, 0] == 0.0 and f64(o["mean"])[0, 0] == float(v)
    del S, Q, dev
    sat.free()


def test_u16_70k_by_85k_banded():
    """70,000 x 85,000 uint16 (5.95e9 px): the squared-pixel table of the
    whole image could overflow uint64, so the one-table build refuses it; the
    banded path (pinned host image in, host outputs out, 5,000-row bands)
    gives every sampled window equal to the definition, with extra samples
    on windows that end just past a band edge (their tables start in the
    band above)."""
    import torch
    r, c, B = 70000, 85000, 5000
    img = synth.intensity_u16(r, c, synth.DEFAULT_SEED + 5, 50000)
    h = torch.from_numpy(img.view(np.int16)).pin_memory()
    wins = [(256, 256, 16, 16), (1024, 1024, 16, 16)]
    dev = h.to("cuda")
    with pytest.raises(swa.SwaError) as ei:
        swa.build_sat(dev)                  # the one-table build refuses it
    assert ei.value.status == swa.SWA_EOVERFLOW
    del dev
    res = swa.analyze(h, wins, band_rows=B)
    for (wh, ww, sy, sx), got in zip(wins, res):
        R, C = got["sum"].shape
        edge = [max(0, -(-(b * B - wh + 1) // sy)) for b in range(1, r // B)]
        ii = np.concatenate([[0, R - 1], edge, [e + 1 for e in edge], RNG.integers(0, R, 40)])
        ii = np.minimum(ii, R - 1)
        jj = RNG.integers(0, C, len(ii))
        for i, j in zip(ii, jj):
            s, _, m, d = oracle.window_one(img, int(i) * sy, int(j) * sx, wh, ww)
            assert int(u64(got["sum"][i:i + 1, j:j + 1])[0, 0]) == s, (wh, i, j)
            assert f64(got["mean"][i:i + 1, j:j + 1])[0, 0] == m
            assert f64(got["std"][i:i + 1, j:j + 1])[0, 0] == d
    del h, res
