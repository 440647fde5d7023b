"""Serving: requests admitted while others run, overlapping on several
streams, with a table cache small enough to evict.  Every result must equal
the same request run alone (bit for bit: the arithmetic is exact), and the
oracle for a sample."""
import numpy as np
import pytest

import oracle
import paper_2410_16291_gb300 as swa
import synth
from gpu_util import f64, require_gpu, u64

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    require_gpu()
    import torch
    from paper_2410_16291_gb300 import build
    from paper_2410_16291_gb300.serve import Request, Server, output_bytes, table_bytes
    build.build()
    rng = np.random.default_rng(8)
    pool_np, pool = [], []
    for k in range(6):
        r, c = int(rng.integers(300, 1200)), int(rng.integers(300, 1200))
        if k % 2:
            a = synth.intensity_u16(r, c, 500 + k, synth.cluster_count(r, c))
            pool.append(torch.from_numpy(a.view(np.int16)).pin_memory())
        else:
            a = synth.intensity_u8(r, c, 500 + k, synth.cluster_count(r, c))
            pool.append(torch.from_numpy(a).pin_memory())
        pool_np.append(a)
    reqs = []
    for rid in range(30):
        k = int(rng.choice(6, p=[0.35, 0.25, 0.15, 0.1, 0.1, 0.05]))
        r, c = pool_np[k].shape
        wl = []
        for _ in range(int(rng.integers(1, 4))):
            w = int(rng.integers(4, min(r, c, 120)))
            st = int(rng.integers(2, 9))
            wl.append((w, w, st, st))
        reqs.append(Request(rid, k, pool[k], wl))
    need = max(sum(table_bytes(*pool_np[q.image_id].shape, 1 + (q.image_id % 2)))
               + output_bytes(*pool_np[q.image_id].shape, q.windows)
               + pool_np[q.image_id].nbytes for q in reqs)
    tab = [table_bytes(*a.shape, 1 + (k % 2))[0] for k, a in enumerate(pool_np)]
    # The budget holds the largest request plus half the largest table, well
    # under the tables of all requested images together, so building them all
    # must evict.
    requested = {q.image_id for q in reqs}
    budget = need + max(tab) // 2
    assert sum(tab[k] for k in requested) > budget
    server = Server(budget_bytes=budget, streams=3, slots=6)
    server.run(reqs, realtime=False)
    assert len(server.completed) == 30
    assert server.hits > 0 and server.misses > 0 and server.evictions > 0
    s = torch.cuda.Stream()
    for q in reqs:
        with torch.cuda.stream(s):
            dev = q.host_image.to("cuda")
            sat = swa.build_sat(dev, stream=s)
            alone = sat.window_stats(q.windows, stream=s)
        s.synchronize()
        for got, ref in zip(q.result, alone):
            for key in ("sum", "mean", "std"):
                assert torch.equal(got[key], ref[key]), (q.rid, key)
        sat.free()
    for q in reqs[:5]:
        S_ref, Q_ref = oracle.sat(pool_np[q.image_id])
        for (wh, ww, sy, sx), got in zip(q.windows, q.result):
            want = oracle.window_sat(S_ref, Q_ref, wh, ww, sy, sx)
            np.testing.assert_array_equal(u64(got["sum"]), want["sum"])
            np.testing.assert_array_equal(f64(got["std"]), want["std"])
    server.close()


def test_failed_build_is_reported_and_its_table_not_reused():
    """A build whose look-back wait expires (the stall hook keeps the first
    tile silent, so the bounded waits run out; nothing faults) is reported as
    a failed request, leaves the cache, and the next request for the same
    image builds again and gets the correct result."""
    require_gpu()
    import torch
    from paper_2410_16291_gb300.serve import Request, Server
    img = synth.intensity_u8(600, 900, 77, synth.cluster_count(600, 900))
    host = torch.from_numpy(img).pin_memory()
    wins = [(32, 32, 4, 4)]
    server = Server(budget_bytes=1 << 30, streams=2, slots=4)
    L = swa.lib()
    L.swa_set_test_hooks(swa.SWA_HOOK_STALL_TILE0)
    try:
        a = Request(0, "img", host, wins)
        server.run([a], realtime=False)
    finally:
        L.swa_set_test_hooks(0)
    assert a.failed and "build failed" in a.error and a.result is None
    assert server.failed == [a] and server.cache.get("img") is None
    assert server.cache.used == 0
    b = Request(1, "img", host, wins)
    server.run([b], realtime=False)
    assert not b.failed and not b.hit and server.misses == 2
    S_ref, Q_ref = oracle.sat(img)
    want = oracle.window_sat(S_ref, Q_ref, 32, 32, 4, 4)
    np.testing.assert_array_equal(u64(b.result[0]["sum"]), want["sum"])
    np.testing.assert_array_equal(f64(b.result[0]["std"]), want["std"])
    server.close()
