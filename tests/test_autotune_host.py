"""Host logic of the autotuner (CPU): the fastest candidate is kept, results are
cached per key and reused without timing, and the cache file is replaced
atomically.  The device calls are replaced by a fake library whose "time" is a
function of the schedule it was given."""
import json
import types

import pytest

from paper_2405_11671_gb300 import autotune


class FakeByo:
    BYO_SCHED_HEURISTIC = 0

    def __init__(self, cost):
        self.cost = cost
        self.last = None
        self.calls = 0

    def make_sched(self, mode, thr_thread, thr_warp, alpha=15.0):
        return (thr_thread, thr_warp, alpha)

    def byo_bfs(self, g, sources, sched=None, want_parents=True):
        self.last = sched
        self.calls += 1

    def byo_msbfs(self, g, sources, num_sources, levels, sched=None):
        self.last = sched
        self.calls += 1


@pytest.fixture
def fake(monkeypatch, tmp_path):
    state = types.SimpleNamespace(byo=None)
    monkeypatch.setenv("BYO_AUTOTUNE_CACHE", str(tmp_path / "cache" / "autotune.json"))
    monkeypatch.setattr(autotune, "_key", lambda byo, g, op, extra="": f"gpu|{op}|g={g}{extra}")

    def fake_time(fn, repeats):
        fn()
        return state.byo.cost(state.byo.last)

    monkeypatch.setattr(autotune, "_time", fake_time)
    return state


def test_bfs_picks_the_fastest_bins_and_caches(fake, tmp_path):
    fake.byo = FakeByo(lambda s: abs(s[0] - 8) + abs(s[1] - 512) / 64)  # fastest at (8, 512)
    res = autotune.tune_bfs(fake.byo, 7, [0, 1])
    assert (res["thr_thread"], res["thr_warp"]) == (8, 512)
    assert res["ms"] == min(res["table_ms"].values()) and len(res["table_ms"]) == len(autotune.BFS_BINS)
    calls = fake.byo.calls
    again = autotune.tune_bfs(fake.byo, 7, [0, 1])  # cached: nothing is timed
    assert again == res and fake.byo.calls == calls
    stored = json.loads((tmp_path / "cache" / "autotune.json").read_text())
    assert stored["gpu|bfs|g=7|S=2"]["thr_thread"] == 8
    assert not list((tmp_path / "cache").glob("*.tmp*"))  # written through a temporary, then replaced


def test_bfs_cache_can_be_bypassed(fake):
    fake.byo = FakeByo(lambda s: s[0])
    autotune.tune_bfs(fake.byo, 3, [5])
    fake.byo.cost = lambda s: -s[0]  # now the largest bins win
    res = autotune.tune_bfs(fake.byo, 3, [5], use_cache=False)
    assert res["thr_thread"] == max(t for t, _ in autotune.BFS_BINS)


def test_msbfs_picks_the_fastest_alpha_per_key(fake):
    fake.byo = FakeByo(lambda s: abs(s[2] - 40.0))
    res = autotune.tune_msbfs(fake.byo, 11, [0] * 64, 64)
    assert res["alpha"] == 40.0 and set(res["table_ms"]) == {str(a) for a in autotune.MSBFS_ALPHAS}
    fake.byo.cost = lambda s: abs(s[2] - 1.0)
    other = autotune.tune_msbfs(fake.byo, 11, [0] * 32, 32)  # another key: timed afresh
    assert other["alpha"] == 1.0
    assert autotune.tune_msbfs(fake.byo, 11, [0] * 64, 64)["alpha"] == 40.0  # first key still cached


def test_unreadable_cache_is_ignored(fake, tmp_path):
    p = tmp_path / "cache" / "autotune.json"
    p.parent.mkdir(parents=True)
    p.write_text("{not json")
    fake.byo = FakeByo(lambda s: s[1])
    res = autotune.tune_bfs(fake.byo, 1, [0])
    assert res["thr_warp"] == min(w for _, w in autotune.BFS_BINS)
    assert json.loads(p.read_text())  # rewritten as valid JSON
