"""The server's resident-table cache and memory budget (CPU, fake tables)."""
from paper_2410_16291_gb300.serve import TableCache, _Entry


class FakeSat:
    freed = []

    def __init__(self, name):
        self.name = name

    def free(self):
        FakeSat.freed.append(self.name)


def test_reserve_evicts_least_recently_used_unreferenced():
    FakeSat.freed = []
    c = TableCache(100)
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
