"""The band partition of the out-of-core path (swa_band_range, host only):
every output row belongs to exactly one band, in order, and the band that
serves a window ends it: its bottom row lies in the band's rows.  A band's
tables start at the top row of its first window, which the four-corner
lookup (Section II-B) needs at or above every window it serves; that row is
never more than wh - 1 rows above the band."""
import numpy as np
import pytest

import paper_2410_16291_gb300 as swa
from paper_2410_16291_gb300 import build as swa_build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    swa_build.build()


CASES = [(1, 1, 1, 1), (10, 3, 1, 1), (10, 10, 3, 4), (97, 5, 3, 7), (100, 64, 16, 1),
         (100, 64, 16, 200), (1000, 200, 7, 64), (1000, 1, 9, 33), (513, 512, 1, 2),
         (70000, 1024, 16, 12345)]


@pytest.mark.parametrize("rows,wh,sy,B", CASES)
def test_bands_partition_the_output_rows(rows, wh, sy, B):
    R = (rows - wh) // sy + 1
    nb = -(-rows // B)
    seen = np.zeros(R, dtype=np.int64)
    prev_end = 0
    for b in range(nb):
        ib, ie = swa.band_range(rows, wh, sy, B, b)
        assert ib == prev_end and ie >= ib
        prev_end = ie
        lo, hi = b * B, min(rows, (b + 1) * B)
        for i in range(ib, ie):
            seen[i] += 1
            y1 = i * sy + wh - 1
            assert lo <= y1 < hi
            assert i * sy >= lo - (wh - 1)
    assert prev_end == R and (seen == 1).all()
    assert swa.band_range(rows, wh, sy, B, nb) == (R, R)
    assert swa.band_range(rows, wh, sy, B, nb + 5) == (R, R)


def test_random_partitions():
    rng = np.random.default_rng(3)
    for _ in range(300):
        rows = int(rng.integers(1, 400))
        wh = int(rng.integers(1, rows + 1))
        sy = int(rng.integers(1, 20))
        B = int(rng.integers(1, 2 * rows + 2))
        test_bands_partition_the_output_rows(rows, wh, sy, B)


@pytest.mark.parametrize("args", [(0, 1, 1, 1, 0), (10, 0, 1, 1, 0), (10, 11, 1, 1, 0),
                                  (10, 2, 0, 1, 0), (10, 2, 1, 0, 0), (10, 2, 1, 1, -1)])
def test_band_range_rejects_bad_arguments(args):
    with pytest.raises(swa.SwaError):
        swa.band_range(*args)
