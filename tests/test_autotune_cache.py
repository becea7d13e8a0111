"""Host logic of the tile-shape autotuner's cache (no GPU): the first call
times and stores the winner, the second retiles from the cache without
timing, retune=True times again; the file is valid JSON keyed by device,
operation and problem."""
import json

import paper_2204_06083_gb300 as pkg
from paper_2204_06083_gb300 import autotune


class FakeEB:
    def __init__(self):
        import eb_inputs as ei
        self.grid = ei.box_grid(2, 64)
        self.info = type("I", (), {"num_cp": 777})()
        self.retiled = []
        self.tuned = 0

    def retile(self, shape):
        self.retiled.append(tuple(shape))

    def autotune(self, prec, reps, op=0):
        self.tuned += 1
        return pkg.TuneResult([(32, 8, 1), (64, 4, 1), (16, 16, 1)], [5.0, 3.0, 4.0], 1)


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_device", lambda: "FakeGPU")
    path = str(tmp_path / "tiles.json")
    eb = FakeEB()
    shape, res = autotune.tune_eb(eb, path=path)
    assert shape == (64, 4, 1) and res is not None and eb.tuned == 1 and eb.retiled == []
    shape2, res2 = autotune.tune_eb(eb, path=path)
    assert shape2 == (64, 4, 1) and res2 is None and eb.tuned == 1 and eb.retiled == [(64, 4, 1)]
    autotune.tune_eb(eb, path=path, retune=True)
    assert eb.tuned == 2
    d = json.load(open(path))
    (key,) = d.keys()
    assert key.startswith("FakeGPU | apply prec=0 | 2D 64x64 cp=777")
    assert d[key]["tile"] == [64, 4, 1] and d[key]["us"]["64x4x1"] == 3.0


def test_cache_path_env(monkeypatch, tmp_path):
    monkeypatch.setenv("EB_TUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.cache_path() == str(tmp_path / "x.json")


class FakeAMG:
    def __init__(self):
        self.eb = FakeEB()
        self.vcycle_prec = 1
        self.tuned = 0
        self.set_to = []

    def tune_csr(self, reps):
        self.tuned += 1
        return 4, {1: 9.0, 2: 7.0, 4: 5.0, 8: 6.0}

    def set_csr_epl(self, epl):
        self.set_to.append(epl)


def test_csr_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_device", lambda: "FakeGPU")
    path = str(tmp_path / "tiles.json")
    amg = FakeAMG()
    assert autotune.tune_csr(amg, path=path) == (4, {1: 9.0, 2: 7.0, 4: 5.0, 8: 6.0})
    assert amg.tuned == 1 and amg.set_to == []
    assert autotune.tune_csr(amg, path=path) == (4, None)
    assert amg.tuned == 1 and amg.set_to == [4]
    d = json.load(open(path))
    (key,) = d.keys()
    assert key.startswith("FakeGPU | csr vcycle prec=1 | 2D 64x64 cp=777") and d[key]["epl"] == 4
