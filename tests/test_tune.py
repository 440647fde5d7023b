"""The batch autotuner's host logic (CPU): candidate choice, sampling, cache
keys and the cache file."""
import json

from paper_2410_16291_gb300 import tune


def test_candidates_cover_every_combination_defaults_first():
    assert len(tune.CANDIDATES) == 64
    assert tune.CANDIDATES[0] == {"u8_tile_rows": 64, "order": 0, "ticket_order": 0,
                                  "lookback": 0, "warps": 9, "interleave": 8}
    assert len({tuple(sorted(c.items())) for c in tune.CANDIDATES}) == 64


def test_choose_picks_fastest_and_breaks_ties_in_order():
    assert tune.choose({0: 5.0, 1: 3.0, 2: 4.0, 3: 3.0}) == tune.CANDIDATES[1]
    assert tune.choose({2: 1.0}) == tune.CANDIDATES[2]


def test_sample_indices_spread():
    assert tune.sample_indices(5, 24) == [0, 1, 2, 3, 4]
    s = tune.sample_indices(256, 24)
    assert len(s) == 24 and s[0] == 0 and s[-1] >= 240 and s == sorted(set(s))


def test_key_buckets():
    k1 = tune.batch_key("GB300", [(1000, 2000)] * 256, ["u8"] * 128 + ["u16"] * 128)
    k2 = tune.batch_key("GB300", [(1100, 1900)] * 300, ["u8"] * 150 + ["u16"] * 150)
    assert k1 == k2 and "u16q2" in k1
    assert tune.batch_key("GB300", [(100, 100)], ["u8"]) != k1


class FakeImg:
    def __init__(self, r, c, dt):
        self.shape = (r, c)
        self.dtype = "torch.uint8" if dt == "u8" else "torch.uint16"


def test_tune_uses_timer_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("SWA_TUNE_CACHE", str(tmp_path / "t.json"))
    imgs = [FakeImg(512 + i, 600, "u8" if i % 2 else "u16") for i in range(40)]
    wins = [[(16, 16, 1, 1)]] * 40
    calls = []

    want = {"u8_tile_rows": 32, "order": 1, "ticket_order": 0, "lookback": 1, "warps": 8,
            "interleave": 1}

    def timer(cfg, ii, ww):
        calls.append((dict(cfg), len(ii)))
        return 1.0 if cfg == want else 2.0
    best = tune.tune(imgs, wins, sample=8, timer=timer)
    assert best == want
    assert len(calls) == 64 and all(n == 8 for _, n in calls)
    data = json.load(open(tmp_path / "t.json"))
    assert list(data.values())[0]["config"] == best
    calls.clear()
    assert tune.tune(imgs, wins, sample=8, timer=timer) == best
    assert calls == []                      # served from the cache
