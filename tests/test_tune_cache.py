"""Host logic of the autotuner's cache (no GPU): the choice is keyed by the
device and the level's patch-size histogram, written to the cache file and
read back by a later process without timing again; an unreadable file is
ignored; SWA_TUNE_CACHE="" keeps the cache in the process."""
import json

from paper_1605_05320_gb300 import tune


class FakeSet:
    def __init__(self, sizes, level=1):
        self.patches = [(level, 0.0, 0.0, nx, ny, 1.0, 1.0) for nx, ny in sizes]
        self.levels = [level]
        self.h = object()

    def step(self, level, n):
        pass


def fresh(monkeypatch, path, times):
    monkeypatch.setenv("SWA_TUNE_CACHE", str(path) if path is not None else "")
    monkeypatch.setattr(tune, "_cache", {})
    monkeypatch.setattr(tune, "_loaded_from", None)
    monkeypatch.setattr(tune, "_device", lambda: "GPU-under-test")
    applied, timed = [], []
    monkeypatch.setattr(tune.S, "swa_patches_set_tile_rows",
                        lambda h, lv, rows: applied.append((lv, rows)))

    def fake_time(fn, steps):
        rows = applied[-1][1]
        timed.append(rows)
        return times[rows]

    monkeypatch.setattr(tune, "_time", fake_time)
    return applied, timed


def test_choice_is_written_and_read_back(monkeypatch, tmp_path):
    path = tmp_path / "sub" / "tune.json"
    ps = FakeSet([(40, 40), (100, 60), (200, 250)])
    applied, timed = fresh(monkeypatch, path, {32: 2.0, 16: 1.0})
    assert tune.tune_patches(ps) == {1: 16}
    assert sorted(timed) == [16, 32] and applied[-1] == (1, 16)
    data = json.loads(path.read_text())
    assert list(data.values()) == [16]
    assert "GPU-under-test" in list(data)[0]
    # a later process: read from the file, no timing
    applied, timed = fresh(monkeypatch, path, {32: 0.5, 16: 9.0})
    assert tune.tune_patches(ps) == {1: 16}
    assert timed == [] and applied == [(1, 16)]
    # another histogram is tuned afresh and added
    other = FakeSet([(16, 16)] * 5)
    assert tune.tune_patches(other) == {1: 32}
    assert len(json.loads(path.read_text())) == 2


def test_unreadable_cache_is_ignored_and_empty_name_keeps_it_in_process(monkeypatch, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    ps = FakeSet([(64, 64)])
    applied, timed = fresh(monkeypatch, path, {32: 1.0, 16: 2.0})
    assert tune.tune_patches(ps) == {1: 32} and sorted(timed) == [16, 32]
    assert json.loads(path.read_text())   # rewritten
    fresh(monkeypatch, None, {32: 1.0, 16: 2.0})
    assert tune.cache_path() is None
    assert tune.tune_patches(ps) == {1: 32}
