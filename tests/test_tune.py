"""Autotuner selection and cache logic (CPU only; the timing itself needs a GPU)."""
import json

import pytest

from paper_2405_01420_gb300.tune import TuneCache, select_best


def test_select_best_picks_minimum_and_skips_invalid():
    timings = {"a": 3.0, "b": None, "c": 1.5, "d": 2.0}
    best, times = select_best(["a", "b", "c", "d"], lambda k: timings[k])
    assert best == "c"
    assert times["'b'"] is None and times["'c'"] == 1.5


def test_select_best_all_invalid():
    with pytest.raises(RuntimeError):
        select_best([1, 2], lambda k: None)


def test_cache_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    c = TuneCache(str(path))
    assert c.get("GB300", "sig") is None
    c.put("GB300", "sig", {"shape": [256, 16, 0]})
    c2 = TuneCache(str(path))
    assert c2.get("GB300", "sig") == {"shape": [256, 16, 0]}
    assert json.loads(path.read_text())["GB300|sig"]["shape"] == [256, 16, 0]


def test_cache_without_path_is_in_memory(monkeypatch):
    monkeypatch.delenv("NB_TUNE_CACHE", raising=False)
    c = TuneCache()
    c.put("dev", "s", 1)
    assert c.get("dev", "s") == 1 and c.path is None


class _FakeEngine:
    """Stands in for NonbondedEngine: a schedule whose lists go stale when the
    prune interval outruns the margin (a displacement of 0.004 nm per frame)."""

    def __init__(self, r_inner, interval, rc):
        self.margin, self.interval = r_inner - rc, interval
        self.closed = False

    def check(self):
        return 0x10 if self.interval * 0.004 > self.margin else 0

    def close(self):
        self.closed = True


def test_tune_trajectory_rejects_stale_schedules_and_picks_the_fastest(monkeypatch):
    from paper_2405_01420_gb300 import tune
    made = []

    def make_engine(r_inner, interval):
        e = _FakeEngine(r_inner, interval, 1.0)
        made.append(e)
        return e

    # time per trajectory: fewer prunes (long intervals) and thin margins (short lists) are faster
    current = {}
    monkeypatch.setattr(tune, "_median_ms", lambda fn, reps: 10.0 / current["e"].interval + 100.0 * current["e"].margin)
    best, times = tune.tune_trajectory(make_engine, lambda e: current.update(e=e), rc=1.0)
    interval, margin = best
    assert interval * 0.004 <= margin  # a valid schedule
    valid = {(i, m): 10.0 / i + 100.0 * m for i in (5, 10, 20) for m in (0.02, 0.04, 0.06) if i * 0.004 <= m}
    assert best == min(valid, key=valid.get)
    assert times[repr((20, 0.02))] is None  # stale: rejected
    assert all(e.closed for e in made)


def test_tune_force_shape_sets_the_winner_and_uses_the_cache(monkeypatch):
    from paper_2405_01420_gb300 import nb, tune
    calls = []
    monkeypatch.setattr(nb, "nb_set_force_shape", lambda h, *shape: calls.append(shape))
    monkeypatch.setattr(tune, "_device_name", lambda: "GB300")
    speed = {(256, 16, 0): 1.4, (256, 8, 0): 1.35, (128, 16, 0): 1.3, (128, 8, 0): 1.2, (256, 16, 3): 1.33,
             (128, 16, 6): 1.25}
    monkeypatch.setattr(tune, "_median_ms", lambda fn, reps: speed[calls[-1]])

    class PL:
        handle = object()

    cache = tune.TuneCache(None)
    best, times = tune.tune_force_shape(PL(), lambda: None, signature="w96k", cache=cache)
    assert best == (128, 8, 0) and calls[-1] == (128, 8, 0)
    assert cache.get("GB300", "force_shape|w96k")["shape"] == [128, 8, 0]
    calls.clear()
    best2, _ = tune.tune_force_shape(PL(), lambda: pytest.fail("a cache hit measures nothing"), signature="w96k",
                                     cache=cache)
    assert best2 == (128, 8, 0) and calls == [(128, 8, 0)]
