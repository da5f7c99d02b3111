"""Host logic of the tile-shape autotuner's cache (no GPU): one entry per
(device, lattice, precision, walls); a hit sets the cached shape without a
search; a cached shape the library rejects falls back to a new search."""
import json

from paper_1711_10984_gb300 import autotune

T = autotune.kernels_tag() + "|"  # keys start with the hash of the CUDA sources


class FakeParams:
    def __init__(self, precision, flags):
        self.precision, self.flags = precision, flags


class FakeSim:
    """Stands in for lbd.Sim: records set_tile calls, counts searches."""

    def __init__(self, nx=64, ny=32, precision=1, flags=0, best=(118, 64), reject=()):
        self.nx, self.ny = nx, ny
        self.params = FakeParams(precision, flags)
        self.best, self.reject = best, set(reject)
        self.tiles, self.searches = [], 0

    def set_tile(self, bx, by):
        if (bx, by) in self.reject:
            raise RuntimeError("LBD_EINVAL: shape not valid here")
        self.tiles.append((bx, by))

    def autotune(self, reps):
        self.searches += 1
        self.tiles.append(self.best)
        return self.best


def test_search_then_cache_hit(tmp_path):
    path = str(tmp_path / "cache.json")
    a = FakeSim()
    assert autotune.tune(a, "GB300", path=path) == (118, 64)
    assert a.searches == 1
    b = FakeSim(best=(32, 8))  # a second context of the same kind: cache hit
    assert autotune.tune(b, "GB300", path=path) == (118, 64)
    assert b.searches == 0 and b.tiles == [(118, 64)]
    assert autotune.tune(b, "GB300", path=path, refresh=True) == (32, 8)
    assert json.load(open(path)) == {T + "GB300|64x32|fp32": [32, 8]}


def test_keys_separate_precision_walls_device_and_size(tmp_path):
    path = str(tmp_path / "cache.json")
    autotune.tune(FakeSim(precision=1), "GB300", path=path)
    autotune.tune(FakeSim(precision=0, best=(118, 128)), "GB300", path=path)
    autotune.tune(FakeSim(flags=16, best=(32, 16)), "GB300", path=path)
    autotune.tune(FakeSim(nx=65, best=(32, 8)), "GB300", path=path)
    autotune.tune(FakeSim(best=(246, 64)), "other", path=path)
    assert json.load(open(path)) == {
        T + "GB300|64x32|fp32": [118, 64],
        T + "GB300|64x32|fp64": [118, 128],
        T + "GB300|64x32|fp32|walls": [32, 16],
        T + "GB300|65x32|fp32": [32, 8],
        T + "other|64x32|fp32": [246, 64],
    }


def test_rejected_cached_shape_searches_again(tmp_path):
    path = str(tmp_path / "cache.json")
    autotune.store(autotune._key("GB300", 64, 32, 1, 16), (116, 64), path)
    s = FakeSim(flags=16, best=(32, 16), reject={(116, 64)})
    assert autotune.tune(s, "GB300", path=path) == (32, 16)
    assert s.searches == 1
    assert json.load(open(path))[T + "GB300|64x32|fp32|walls"] == [32, 16]


def test_unreadable_cache_is_empty(tmp_path):
    path = tmp_path / "cache.json"
    path.write_text("{not json")
    assert autotune.load_cache(str(path)) == {}
    assert autotune.tune(FakeSim(), "GB300", path=str(path)) == (118, 64)


def test_key_changes_with_the_kernel_sources(tmp_path, monkeypatch):
    """A winner stored for other kernel sources is not reused."""
    path = str(tmp_path / "cache.json")
    autotune.tune(FakeSim(), "GB300", path=path)
    monkeypatch.setattr(autotune, "kernels_tag", lambda: "other-sources")
    s = FakeSim(best=(32, 8))
    assert autotune.tune(s, "GB300", path=path) == (32, 8) and s.searches == 1
