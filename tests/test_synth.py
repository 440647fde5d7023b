"""The seeded input generators: shapes, distributions and determinism."""
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_mask_has_exact_ones_and_is_clustered():
    m = synth.mask_u8(1024, 1024, synth.DEFAULT_SEED)
    assert m.dtype == np.uint8 and set(np.unique(m)) <= {0, 1}
    assert int(m.sum()) == round(0.03 * 1024 * 1024) == 31457
    # clustered: 32x32 block counts are overdispersed relative to a uniform field
    blocks = m.reshape(32, 32, 32, 32).sum(axis=(1, 3)).astype(float)
    assert blocks.var() > 3 * blocks.mean()


def test_intensity_u8_distribution():
    a = synth.intensity_u8(2000, 2000, 5, synth.cluster_count(2000, 2000))
    # Gamma(2, 20) background has mean 40; clusters add brightness, clip at 255
    assert 35 < a.mean() < 90
    assert a.max() == 255 and a.min() == 0


def test_intensity_u16_distribution():
    a = synth.intensity_u16(1000, 1200, 9, 0)
    assert 390 <= np.median(a) <= 416          # log-normal median e^6 = 403
    assert 1.45 < np.log(a.astype(float) + 0.5).std() < 1.55
    b = synth.intensity_u16(1000, 1200, 9, 3)  # clusters only brighten
    assert (b >= a).all() and b.max() == 65535


def test_generators_are_seeded():
    a = synth.intensity_u8(300, 400, 1, 5)
    b = synth.intensity_u8(300, 400, 1, 5)
    c = synth.intensity_u8(300, 400, 2, 5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_thread_count_independent():
    code = ("import synth,hashlib;"
            "a=synth.intensity_u8(257,999,3,40);b=synth.intensity_u16(130,77,4,3);"
            "print(hashlib.sha256(a.tobytes()+b.tobytes()).hexdigest())")
    outs = []
    for n in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=n, PYTHONPATH=ROOT)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env, cwd=ROOT))
    assert outs[0] == outs[1]


def test_workload_shapes():
    (w0,) = synth.workload(0)
    assert (w0.rows, w0.cols, w0.dtype, w0.with_sq) == (1024, 1024, "u8", False)
    (w1,) = synth.workload(1)
    assert [w.wh for w in w1.windows] == [50, 100, 200]
    (w2,) = synth.workload(2)
    assert (w2.rows, w2.cols) == (70000, 85000) and w2.windows[0].sy == 16
    b = synth.workload(3)
    assert len(b) == 256
    assert all(512 <= im.cols <= 8192 and 512 <= im.rows <= 8192 for im in b)
    assert {im.dtype for im in b} == {"u8", "u16"}
    assert all(1 <= len(im.windows) <= 4 for im in b)
    pool, reqs = synth.serve_requests(100, 4)
    assert len(pool) == 64 and len(reqs) == 100
    assert all(1 <= len(w) <= 8 for _, _, w in reqs)
    ts = [t for t, _, _ in reqs]
    assert ts == sorted(ts) and 0.2 < ts[-1] < 1.0   # ~200 req/s
