"""The server's resident-table cache and memory budget (CPU, fake tables)."""
import pytest

from paper_2410_16291_gb300.serve import TableCache, _Entry


class FakeSat:
    freed = []

    def __init__(self, name):
        self.name = name

    def free(self):
        FakeSat.freed.append(self.name)


def test_reserve_evicts_least_recently_used_unreferenced():
    FakeSat.freed = []
    c = TableCache(100, policy="lru")
    for k in "abc":
        assert c.reserve(30)
        c.insert(k, _Entry(FakeSat(k), 30))
    assert c.used == 90
    c.get("a")                       # a becomes most recent: LRU order b, c, a
    c.entries["b"].refs = 1          # b is in use
    assert c.reserve(40)             # evicts c (b is referenced) -> 60 + 40
    assert FakeSat.freed == ["c"] and c.used == 100 and c.evictions == 1
    assert c.reserve(1)              # full: evicts a (unreferenced), not b
    assert FakeSat.freed == ["c", "a"] and c.used == 71 and list(c.entries) == ["b"]


def test_lfu_evicts_the_least_asked_for_first_then_the_least_recent():
    FakeSat.freed = []
    c = TableCache(100)                  # policy "lfu"
    for k in "abc":
        assert c.reserve(30)
        c.insert(k, _Entry(FakeSat(k), 30))
    for k, n in (("a", 1), ("b", 3), ("c", 2)):
        for _ in range(n):
            c.count(k)
    c.get("b")
    c.get("c")                           # LRU order now a, b, c
    c.get("a")                           # ... b, c, a: LRU would evict b first
    assert c.reserve(40)                 # a was asked for least often: a goes
    assert FakeSat.freed == ["a"] and c.used == 100
    c.count("b")                         # b: 4, c: 2
    assert c.reserve(30)                 # c next (fewer requests than b)
    assert FakeSat.freed == ["a", "c"] and list(c.entries) == ["b"]
    c.insert("a", _Entry(FakeSat("a2"), 30))     # counts outlive an eviction
    assert c.freq["a"] == 1 and c.freq["c"] == 2
    with pytest.raises(ValueError):
        TableCache(10, policy="fifo")


def test_reserve_fails_when_everything_is_referenced():
    FakeSat.freed = []
    c = TableCache(50)
    assert c.reserve(40)
    c.insert("x", _Entry(FakeSat("x"), 40, refs=1))
    assert not c.reserve(20)
    assert FakeSat.freed == [] and c.used == 40
    c.entries["x"].refs = 0
    assert c.reserve(20) and FakeSat.freed == ["x"] and c.used == 20
    c.release(20)
    assert c.used == 0


def test_failed_reserve_evicts_nothing():
    FakeSat.freed = []
    c = TableCache(100)
    for k, refs in (("a", 0), ("b", 1)):
        assert c.reserve(40)
        c.insert(k, _Entry(FakeSat(k), 40, refs=refs))
    # 80 used, only a (40) can go: 80 - 40 + 70 > 100, so nothing is evicted
    assert not c.reserve(70)
    assert FakeSat.freed == [] and c.used == 80 and list(c.entries) == ["a", "b"]
    assert c.reserve(50) and FakeSat.freed == ["a"] and c.used == 90


def _fake_server(fits, slots=8, lookahead=8, max_bypass=16):
    """A Server whose admission test is `fits(request)`; no device needed."""
    import collections
    from paper_2410_16291_gb300.serve import Request, Server
    sv = object.__new__(Server)
    sv.slots, sv.lookahead, sv.max_bypass = slots, lookahead, max_bypass
    sv.inflight, sv.waiting = [], collections.deque()
    order = []

    def try_admit(req, now):
        if not fits(req):
            return False
        order.append(req.rid)
        sv.inflight.append(req)
        return True
    sv._try_admit = try_admit
    return sv, order, Request


def test_admission_lets_fitting_requests_pass_a_blocked_head():
    sv, order, Request = _fake_server(lambda r: r.rid != 0)
    sv.waiting.extend(Request(i, i, None, []) for i in range(4))
    assert sv._admit(0.0)
    assert order == [1, 2, 3] and sv.waiting[0].rid == 0 and sv.waiting[0].bypassed == 3


def test_admission_bypass_is_bounded():
    sv, order, Request = _fake_server(lambda r: r.rid != 0, max_bypass=2)
    sv.waiting.extend(Request(i, i, None, []) for i in range(5))
    sv._admit(0.0)
    assert order == [1, 2] and [r.rid for r in sv.waiting] == [0, 3, 4]


def test_admission_respects_slots_and_order():
    sv, order, Request = _fake_server(lambda r: True, slots=3)
    sv.waiting.extend(Request(i, i, None, []) for i in range(5))
    sv._admit(0.0)
    assert order == [0, 1, 2] and [r.rid for r in sv.waiting] == [3, 4]


def test_dropped_entry_is_freed_when_its_last_user_finishes():
    """A failed build leaves the cache at once (no later hit finds it) and
    gives its bytes back only when no in-flight request uses it."""
    FakeSat.freed = []
    c = TableCache(100)
    assert c.reserve(40)
    e = _Entry(FakeSat("bad"), 40, refs=2)
    c.insert("img", e)
    c.drop("img", e)
    assert c.get("img") is None and FakeSat.freed == [] and c.used == 40
    e.refs = 1
    c.release_dropped(e)
    assert FakeSat.freed == [] and c.used == 40
    e.refs = 0
    c.release_dropped(e)
    assert FakeSat.freed == ["bad"] and c.used == 0
    c.release_dropped(e)                 # idempotent
    assert FakeSat.freed == ["bad"] and c.used == 0


def test_request_that_can_never_fit_fails_alone():
    """A request larger than the whole budget is reported failed by itself;
    the requests behind it are still admitted."""
    sv, order, Request = _fake_server(lambda r: True)
    sv.completed, sv.failed, sv.on_complete = [], [], None
    inner = sv._try_admit

    def try_admit(req, now):
        if req.rid == 1:
            req.error = "needs more than the budget"
            return None
        return inner(req, now)
    sv._try_admit = try_admit
    sv.keep_results = True
    sv.waiting.extend(Request(i, i, None, []) for i in range(4))
    assert sv._admit(0.0)
    assert order == [0, 2, 3] and not sv.waiting
    assert [r.rid for r in sv.failed] == [1] and sv.failed[0].done == 0.0


def test_latency_summary_skips_failed_requests():
    from paper_2410_16291_gb300.serve import Request, latency_summary
    rs = [Request(i, 0, None, [], arrival=0.0, done=0.01 * (i + 1)) for i in range(4)]
    rs[3].error = "table build failed"
    out = latency_summary(rs)
    assert out["requests"] == 3 and out["failed"] == 1 and out["max_ms"] == 30.0


def _replay(policy, budget):
    """The served workload's 200-request trace in order through the cache
    (each table freed before the next request): misses and table bytes
    built."""
    import paper_2410_16291_gb300 as swa
    import synth
    from paper_2410_16291_gb300 import build, serve
    build.build()                            # table sizes come from the library (host only)
    pool, trace = synth.serve_requests(200, synth.DEFAULT_SEED + 4)
    c = TableCache(budget, policy=policy)
    misses = built = 0
    for _, idx, _ in trace:
        im = pool[idx]
        if c.get(idx) is None:
            code = swa.SWA_U8 if im.dtype == "u8" else swa.SWA_U16
            tab = serve.table_bytes(im.rows, im.cols, code)[0]
            assert c.reserve(tab)
            c.insert(idx, _Entry(FakeSat(idx), tab))
            misses += 1
            built += tab
        c.count(idx)
    return misses, built


def test_frequency_aware_eviction_rebuilds_less_on_the_served_trace():
    """The served workload's images have far more table bytes than the
    budget; keeping the tables asked for most often rebuilds fewer of them
    than keeping the most recent ones."""
    for budget in (90 * 10**9, 100 * 10**9):
        lfu, lru = _replay("lfu", budget), _replay("lru", budget)
        assert lfu[0] < lru[0] and lfu[1] < lru[1], (budget, lfu, lru)
