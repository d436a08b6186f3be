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
