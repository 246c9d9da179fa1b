"""Host logic of the launch-shape cache (paper_1806_09403_gb300.autotune):
a miss runs the native autotuner once and stores its choice under a key of
GPU, shape, storage, layout, delta, marker count and library version; a hit
applies the stored choice without timing; the file survives a corrupt write
of another process."""
import json
from types import SimpleNamespace

from paper_1806_09403_gb300 import autotune as T


class FakeLattice:
    def __init__(self, nx=1600, ny=800, storage=0, markers=126):
        self.cfg = SimpleNamespace(nx=nx, ny=ny, storage=storage, layout=1, delta=3, nf=1)
        self.marker_count = markers
        self.timed = 0
        self.applied = None

    def autotune(self, steps, flush_l2):
        self.timed += 1
        self.applied = 2
        return 2, {1: 0.030, 2: 0.025, 3: 0.031}

    def tune(self, variant, grid=0):
        self.applied = variant


def test_miss_then_hit(tmp_path):
    path = str(tmp_path / "tune.json")
    a = FakeLattice()
    e = T.tune_lattice(a, T.TuneCache(path), device="GB300")
    assert a.timed == 1 and e["variant"] == 2 and not e["cached"]
    b = FakeLattice()
    e = T.tune_lattice(b, T.TuneCache(path), device="GB300")
    assert b.timed == 0 and b.applied == 2 and e["cached"]
    stored = json.load(open(path))
    assert len(stored) == 1 and list(stored.values())[0]["ms_per_step"]["2"] == 0.025


def test_key_separates_configurations(tmp_path):
    path = str(tmp_path / "tune.json")
    cache = T.TuneCache(path)
    T.tune_lattice(FakeLattice(), cache, device="GB300")
    for other, dev in ((FakeLattice(storage=1), "GB300"), (FakeLattice(nx=800), "GB300"),
                       (FakeLattice(markers=0), "GB300"), (FakeLattice(), "B200")):
        T.tune_lattice(other, cache, device=dev)
        assert other.timed == 1
    assert len(json.load(open(path))) == 5


def test_retune_and_corrupt_file(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    a = FakeLattice()
    T.tune_lattice(a, T.TuneCache(str(path)), device="GB300")
    assert a.timed == 1
    T.tune_lattice(a, T.TuneCache(str(path)), device="GB300", retune=True)
    assert a.timed == 2
    assert json.load(open(path))


def test_cache_path_from_environment(tmp_path, monkeypatch):
    monkeypatch.setenv(T.CACHE_ENV, str(tmp_path / "x.json"))
    assert T.default_cache_path() == str(tmp_path / "x.json")
