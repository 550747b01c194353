"""The planner autotuner's search and cache on the CPU: a fake handle whose
product time is a known function of the parameters stands in for the GPU
timing, so the coordinate search can be checked against the known optimum."""
import json

import pytest


class _Params:
    def __init__(self, d):
        self.d = dict(d)

    def as_dict(self):
        return dict(self.d)


class _FakeHandle:
    DEFAULTS = {"hash_kind": 2, "max_load": 0.5, "group_shift": 4, "dense_ratio": 4, "sym_dense_ratio": 64,
                "bitmap_ratio": 4, "dense_blocks": 0, "dense_owner": 0, "row_window_tbits": 7}

    def __init__(self):
        self.params = _Params(self.DEFAULTS)
        self.sets = 0

    def set_params(self, **kw):
        self.params.d.update(kw)
        self.sets += 1


# separable cost with a unique optimum inside the search space
BEST = {"group_shift": 5, "max_load": 0.5, "dense_ratio": 16, "sym_dense_ratio": 16, "bitmap_ratio": 1,
        "dense_blocks": 2, "dense_owner": 1, "row_window_tbits": 6}


def _cost(d):
    ms = 4.0
    for k, v in BEST.items():
        if d.get(k) != v:
            ms += 0.25
    return ms


@pytest.fixture
def tuner(monkeypatch):
    from paper_2105_14156_gb300 import autotune
    calls = []

    def fake_time(handle, dA, dB, reps=2):
        calls.append(dict(handle.params.d))
        return _cost(handle.params.d)

    monkeypatch.setattr(autotune, "_time", fake_time)
    monkeypatch.setattr(autotune, "gpu_key", lambda: "FakeGPU/152")
    return autotune, calls


def test_coordinate_search_finds_the_separable_optimum(tuner, tmp_path):
    autotune, calls = tuner
    h = _FakeHandle()
    params, ms = autotune.tune(h, None, None, "wl", cache_path=str(tmp_path / "cache.json"))
    assert params == BEST
    assert ms == 4.0
    assert {k: h.params.d[k] for k in BEST} == BEST          # applied to the handle
    # the starting point, then at most every candidate of every parameter once
    assert len(calls) <= 1 + sum(len(vals) for _, vals in autotune.SPACE)


def test_cache_hit_skips_timing(tuner, tmp_path):
    autotune, calls = tuner
    path = str(tmp_path / "cache.json")
    autotune.tune(_FakeHandle(), None, None, "wl", cache_path=path)
    n = len(calls)
    cache = json.load(open(path))
    assert cache["FakeGPU/152"]["wl"]["params"] == BEST
    h = _FakeHandle()
    params, ms = autotune.tune(h, None, None, "wl", cache_path=path)
    assert len(calls) == n                                    # no product timed
    assert params == BEST and ms == 4.0
    assert {k: h.params.d[k] for k in BEST} == BEST
    autotune.tune(_FakeHandle(), None, None, "other workload", cache_path=path)
    assert len(calls) > n                                     # another key is tuned afresh
    assert set(json.load(open(path))["FakeGPU/152"]) == {"wl", "other workload"}


def test_small_gains_are_not_taken(tuner, monkeypatch):
    autotune, calls = tuner
    # every change gains only 1 %: below the 2 % the search asks for
    monkeypatch.setattr(autotune, "_time",
                        lambda h, a, b, reps=2: 4.0 * (0.99 if h.params.d != _FakeHandle.DEFAULTS else 1.0))
    h = _FakeHandle()
    params, _ = autotune.tune(h, None, None, "wl")
    assert params == {k: _FakeHandle.DEFAULTS[k] for k, _ in autotune.SPACE}
