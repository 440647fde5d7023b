"""Every-window parity at full size: device outputs are compared with the
oracle's streamed-rows windows (``oracle.window_rows_stream``) chunk by chunk
of output rows, on host threads (the oracle's C calls and torch's copies
release the GIL).  No arithmetic of the method lives here."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
from gpu_util import f64, u64


def threads():
    return max(1, min(16, os.cpu_count() or 1))


def _chunks(R, rows_per_chunk):
    return [(i, min(R, i + rows_per_chunk)) for i in range(0, R, rows_per_chunk)]


def check_all_windows(img, windows, results, outputs=("sum", "mean", "std"),
                      rows_per_chunk=256):
    """Compare every output of every (wh, ww, sy, sx) query in ``windows``
    with the oracle, bit for bit.  ``results`` are the device output dicts in
    the same order.  Returns the number of windows compared."""
    return check_many([(img, windows, results)], outputs, rows_per_chunk)


def check_many(jobs, outputs=("sum", "mean", "std"), rows_per_chunk=256):
    """check_all_windows over several (image, windows, results) jobs, all
    chunks sharing one pool of host threads."""
    tasks = []
    for img, windows, results in jobs:
        for (wh, ww, sy, sx), got in zip(windows, results):
            R = next(iter(got.values())).shape[0]
            for i0, i1 in _chunks(R, rows_per_chunk):
                tasks.append((img, wh, ww, sy, sx, got, i0, i1))

    def run(t):
        img, wh, ww, sy, sx, got, i0, i1 = t
        want = oracle.window_rows_stream(img, wh, ww, sy, sx, np.arange(i0, i1),
                                         outputs=outputs)
        for k in outputs:
            g = u64(got[k][i0:i1]) if k == "sum" else f64(got[k][i0:i1])
            if not np.array_equal(g, want[k]):
                bad = np.argwhere(g != want[k])[0]
                raise AssertionError("%s w=%dx%d s=%dx%d row %d col %d: got %r want %r" % (
                    k, wh, ww, sy, sx, i0 + bad[0], bad[1], g[tuple(bad)], want[k][tuple(bad)]))
        return (i1 - i0) * want[outputs[0]].shape[1]

    def cost(t):        # image rows streamed plus windows evaluated
        img, wh, ww, sy, sx, got, i0, i1 = t
        return (i1 * sy + wh) * img.shape[1] + (i1 - i0) * got[outputs[0]].shape[1]

    tasks.sort(key=cost, reverse=True)       # largest first: a short tail
    with ThreadPoolExecutor(threads()) as pool:
        return sum(pool.map(run, tasks))
