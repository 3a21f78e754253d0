"""Host logic of the tile-size autotuner of the batched form (no GPU): the
view-class buckets, the batch's tile and the switching margin, the JSON cache
and its refresh.  Device timing is replaced by a fake so that only the bookkeeping
runs."""
import json
import types

import pytest

from paper_1806_05385_gb300 import autotune as A


def _view(W, H, mode=3):
    return types.SimpleNamespace(W=W, H=H, mode=mode)


def test_view_class_buckets():
    # Same mode and buckets -> same class; a mode, a x1.5 resolution step or
    # a x4 triangle step apart -> another class.
    a = A.view_class(_view(1440, 1600), 266_000)
    assert a == A.view_class(_view(1440, 1601), 266_001)
    assert a != A.view_class(_view(1440, 1600, mode=1), 266_000)
    assert a != A.view_class(_view(2160, 2400), 266_000)
    assert a != A.view_class(_view(1440, 1600), 4 * 266_000)
    # Degenerate sizes stay well defined.
    assert A.view_class(_view(0, 0), 0) == A.view_class(_view(1, 1), 1)


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    calls = []
    fake = {8: 3.0, 16: 1.0, 32: 2.0}

    def time_tile(scene, view, tile, reps=10, params=None):
        calls.append((scene, view.W, tile))
        return fake[tile]

    monkeypatch.setattr(A, "time_tile", time_tile)
    path = str(tmp_path / "tiles.json")
    v0, v1 = _view(512, 512), _view(2160, 2160, mode=0)
    # Two views of one class and one of another: each class is timed once.
    tiles = A.tune([("s0", v0, 1000), ("s1", _view(512, 513), 1001), ("s2", v1, 500_000)], cache_path=path)
    assert tiles == [16, 16, 16]
    assert len(calls) == 2 * len(A.TILES)
    with open(path) as f:
        cache = json.load(f)
    assert set(cache) == {A.view_class(v0, 1000), A.view_class(v1, 500_000)}
    assert all(e["tile"] == 16 for e in cache.values())

    # A second run reads the cache and times nothing.
    calls.clear()
    fake.update({8: 0.5})
    assert A.tune([("s0", v0, 1000)], cache_path=path) == [16]
    assert not calls
    # refresh re-times and rewrites the entry.
    assert A.tune([("s0", v0, 1000)], cache_path=path, refresh=True) == [8]
    assert len(calls) == len(A.TILES)
    with open(path) as f:
        assert json.load(f)[A.view_class(v0, 1000)]["tile"] == 8


def test_batch_tile_and_margin(tmp_path, monkeypatch):
    """The batch takes the tile with the least summed time; a class leaves
    it only for a tile faster by more than the margin."""
    fake = {512: {8: 0.95, 16: 1.0, 32: 1.2},    # 5 % faster at 8: stays at 16
            1024: {8: 1.5, 16: 1.0, 32: 1.1},    # 16 is its own best
            2048: {8: 2.0, 16: 1.0, 32: 0.8}}    # 20 % faster at 32: leaves

    def time_tile(scene, view, tile, reps=10, params=None):
        return fake[view.W][tile]

    monkeypatch.setattr(A, "time_tile", time_tile)
    cases = [("a", _view(512, 512), 1000), ("b", _view(1024, 1024), 1000), ("c", _view(2048, 2048), 1000)]
    path = str(tmp_path / "tiles.json")
    assert A.tune(cases, cache_path=path) == [16, 16, 32]
    assert A.tune(cases, cache_path=path, margin=0.25) == [16, 16, 16]
    assert A.tune(cases, cache_path=path, margin=0.0) == [8, 16, 32]
    # the cache keeps every class's timings: later calls re-time nothing
    monkeypatch.setattr(A, "time_tile", lambda *a, **k: pytest.fail("re-timed a cached class"))
    assert A.tune(cases, cache_path=path) == [16, 16, 32]
    # an entry without its timings (an older cache) is re-timed
    with open(path) as f:
        cache = json.load(f)
    del cache[A.view_class(_view(512, 512), 1000)]["ms"]
    with open(path, "w") as f:
        json.dump(cache, f)
    monkeypatch.setattr(A, "time_tile", time_tile)
    assert A.tune(cases, cache_path=path) == [16, 16, 32]
    assert "ms" in json.load(open(path))[A.view_class(_view(512, 512), 1000)]


@pytest.mark.parametrize("content", ["", "{not json", "[]", '{"%s": {"tile": 12}}'])
def test_tune_tolerates_damaged_cache(tmp_path, monkeypatch, content):
    """An unreadable cache, one that is not a mapping, or an entry with a
    tile size outside {8, 16, 32} is re-timed and replaced."""
    monkeypatch.setattr(A, "time_tile", lambda scene, view, tile, reps=10, params=None: float(tile))
    path = tmp_path / "tiles.json"
    path.write_text(content.replace("%s", A.view_class(_view(256, 256), 100)))
    assert A.tune([("s", _view(256, 256), 100)], cache_path=str(path)) == [8]
    assert json.loads(path.read_text())[A.view_class(_view(256, 256), 100)]["tile"] == 8


def test_cache_path_from_environment(tmp_path, monkeypatch):
    monkeypatch.setenv("PR_AUTOTUNE_CACHE", str(tmp_path / "x.json"))
    assert A.default_cache_path() == str(tmp_path / "x.json")
    monkeypatch.setenv("PR_AUTOTUNE_CACHE", str(tmp_path))
    assert A.default_cache_path() == str(tmp_path / "tiles.json")
