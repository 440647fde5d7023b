"""The corner lattice (SWA_LATTICE): a single-pass build that also keeps the
table entries at rows and columns one below a multiple of a stride s, and
window queries at strides (s, s) with sides that are multiples of s served
from it.  The lattice must equal the tables at those points, and every
window -- served from the lattice or not, in the same call -- must equal the
oracle bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, to_device, u64

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(1616)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    from paper_2410_16291_gb300 import build
    build.build()


def image(r, c, dtype, seed):
    if dtype == np.uint8:
        return synth.intensity_u8(r, c, seed, synth.cluster_count(r, c))
    return synth.intensity_u16(r, c, seed, synth.cluster_count(r, c))


def check_windows(img, dev, s, wins):
    S_ref, Q_ref = oracle.sat(img)
    sat = swa.build_sat(dev, lattice=s)
    S, Q = sat.tables()
    np.testing.assert_array_equal(u64(S), S_ref)
    np.testing.assert_array_equal(u64(Q), Q_ref)
    st, LS, LQ = sat.lattice()
    r, c = img.shape
    if r // s and c // s:
        assert st == s and LS.shape == (r // s, c // s)
        np.testing.assert_array_equal(u64(LS), S_ref[s - 1::s, s - 1::s][:r // s, :c // s])
        np.testing.assert_array_equal(u64(LQ), Q_ref[s - 1::s, s - 1::s][:r // s, :c // s])
    else:
        assert st == 0 and LS is None
    wins = [w for w in wins if w[0] <= r and w[1] <= c]
    res = sat.window_stats(wins)
    for (wh, ww, sy, sx), got in zip(wins, res):
        want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx)
        np.testing.assert_array_equal(u64(got["sum"]), want["sum"], err_msg=str((wh, ww, sy, sx)))
        np.testing.assert_array_equal(f64(got["mean"]), want["mean"])
        np.testing.assert_array_equal(f64(got["std"]), want["std"])
    sat.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape", [(1000, 1031), (777, 2048), (300, 4100), (64, 64), (7, 9)])
@pytest.mark.parametrize("s", [8, 13, 16, 255])
def test_lattice_equals_tables_and_windows_equal_oracle(dtype, shape, s):
    img = image(*shape, dtype, 11 + s)
    # served from the lattice: (s, s) strides, sides multiples of s (square
    # and rectangular, as tall as the image allows); not served: a side or a
    # stride off the lattice, stride 1.
    wins = [(s, s, s, s), (2 * s, 3 * s, s, s), (4 * s, 4 * s, s, s),
            (shape[0] // s * s, s, s, s), (2 * s + 1, 2 * s, s, s), (2 * s, 2 * s, s, s + 1),
            (5, 5, 1, 1)]
    wins = [w for w in wins if w[0] > 0]
    check_windows(img, to_device(img), s, wins)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_lattice_on_unaligned_pitched_rows(dtype):
    img = image(513, 1500, dtype, 5)
    dev = to_device(img, pad_cols=7, offset_px=3)
    check_windows(img, dev, 16, [(16, 32, 16, 16), (256, 256, 16, 16), (17, 16, 16, 16)])


def test_analyze_chooses_a_lattice_and_matches_the_oracle():
    """swa_analyze builds the lattice of the stride most of its queries can
    use; results are those of the definition."""
    import torch
    img = image(900, 1300, np.uint16, 77)
    wins = [(64, 64, 16, 16), (128, 256, 16, 16), (50, 50, 16, 16), (32, 32, 8, 8)]
    host = torch.from_numpy(img.view(np.int16)).pin_memory()
    res = swa.analyze(host, wins)
    S_ref, Q_ref = oracle.sat(img)
    for (wh, ww, sy, sx), got in zip(wins, res):
        want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx)
        np.testing.assert_array_equal(got["sum"].numpy().view(np.uint64), want["sum"])
        np.testing.assert_array_equal(got["mean"].numpy(), want["mean"])
        np.testing.assert_array_equal(got["std"].numpy(), want["std"])
