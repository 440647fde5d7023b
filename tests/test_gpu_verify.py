"""swa_verify_tables: the device check of tables against their image by the
summed-area recurrence.  Correct builds pass everywhere; an entry changed
after the build is found, with the number of recurrences it takes part in
and its position."""
import numpy as np
import pytest

import paper_2410_16291_gb300 as swa
import synth
from gpu_util import require_gpu, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    from paper_2410_16291_gb300 import build
    build.build()


def image(r, c, dtype, seed):
    if dtype == np.uint8:
        return synth.intensity_u8(r, c, seed, synth.cluster_count(r, c))
    return synth.intensity_u16(r, c, seed, synth.cluster_count(r, c))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape,pad,off", [((1, 1), 0, 0), ((1, 700), 0, 0), ((700, 1), 0, 0),
                                           ((513, 1031), 0, 0), ((1000, 2049), 5, 3)])
def test_correct_builds_pass(dtype, shape, pad, off):
    img = image(*shape, dtype, 3)
    dev = to_device(img, pad_cols=pad, offset_px=off)
    for twopass in (False, True):
        sat = swa.build_sat(dev, twopass=twopass)
        S, Q = sat.tables()
        assert swa.verify_tables(dev, S, Q) == (0, 0, None)
        assert swa.verify_tables(dev, S) == (0, 0, None)
        sat.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_a_changed_entry_is_found(dtype):
    """Entry (y, x) takes part in the recurrences at (y, x), (y, x+1),
    (y+1, x) and (y+1, x+1) that lie inside the table."""
    r, c = 300, 517
    img = image(r, c, dtype, 4)
    dev = to_device(img)
    rng = np.random.default_rng(5)
    cases = [(0, 0), (r - 1, c - 1), (0, c - 1), (r - 1, 0), (150, 200)] + [
        (int(rng.integers(0, r)), int(rng.integers(0, c))) for _ in range(5)]
    for y, x in cases:
        for table in ("S", "Q"):
            sat = swa.build_sat(dev)
            S, Q = sat.tables()
            T = S if table == "S" else Q
            T[y, x] += 1
            want = (1 + (x + 1 < c)) * (1 + (y + 1 < r))
            got = swa.verify_tables(dev, S, Q)
            assert got == ((want, 0, y * c + x) if table == "S" else (0, want, y * c + x)), \
                (table, y, x, got)
            sat.free()


def test_batch_tables_pass():
    import torch
    imgs = [image(300, 700, np.uint8, 6), image(129, 257, np.uint16, 7),
            image(1000, 513, np.uint8, 8)]
    devs = [to_device(a) for a in imgs]
    b = swa.Batch(devs, [[] for _ in imgs])
    b.run()
    b.sync()
    for k, d in enumerate(devs):
        S, Q = b.tables(k)
        assert swa.verify_tables(d, S, Q) == (0, 0, None)
    b.free()
    torch.cuda.synchronize()
