"""Host logic of the tile autotuner on CPU, with a stand-in batch whose
V-cycle time is a known function of its tiles: the coordinate-descent pass
of tune_batch, the candidates the library refuses, and the JSON cache."""
import json
import types

import pytest

import paper_2412_05082_gb300 as bh
from paper_2412_05082_gb300 import autotune


class FakeBatch:
    """vcycle_time = sum over degrees of (pb - best[k])^2 + 1; set_tile refuses
    tiles above `limit[k]` the way the library refuses a tile that does not
    fit in shared memory."""

    def __init__(self, best, limit, precision=0):
        self.best, self.limit = best, limit
        self.params = [types.SimpleNamespace(precision=precision)]
        self.tiles = {}
        self.timings = 0

    def set_tile(self, k, pb):
        if pb > self.limit.get(k, 99):
            raise bh.BiharmError(bh.BH_EINVAL, "tile does not fit")
        self.tiles[k] = pb

    def vcycle_time(self, reps=5):
        self.timings += 1
        return 1.0 + sum((self.tiles[k] - b) ** 2 for k, b in self.best.items())


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    monkeypatch.setenv("BIHARM_TUNE_CACHE", str(tmp_path / "tiles.json"))
    monkeypatch.setattr(autotune, "_arch", lambda: "sm_103_fake")
    # per-degree starting tiles, as tiles_for would measure them
    monkeypatch.setattr(autotune, "tiles_for", lambda degrees, refresh=False, verbose=False,
                        precision=0: {k: 4 for k in degrees})
    return tmp_path / "tiles.json"


def test_coordinate_descent_finds_each_degrees_best_candidate(tuner):
    problems = [(2, 2, 6), (2, 5, 4), (2, 7, 3), (2, 5, 5)]
    batch = FakeBatch(best={2: 12, 5: 6, 7: 24}, limit={7: 16})
    tiles = autotune.tune_batch(batch, problems)
    # k = 7 is limited to 16 by the (fake) shared-memory check
    assert tiles == {2: 12, 5: 6, 7: 16}
    assert batch.tiles == tiles  # applied to the batch
    # one timing of the start, then every other allowed candidate per degree
    allowed = {k: [pb for pb in autotune.CANDIDATES if pb <= batch.limit.get(k, 99)]
               for k in (2, 5, 7)}
    assert batch.timings == 1 + sum(len(v) - 1 for v in allowed.values())


def test_cache_is_keyed_by_the_problem_list_and_reused(tuner):
    problems = [(2, 3, 5), (2, 4, 4)]
    first = FakeBatch(best={3: 8, 4: 2}, limit={})
    tiles = autotune.tune_batch(first, problems)
    assert tiles == {3: 8, 4: 2}
    cache = json.load(open(tuner))
    key = "batch_p0_2.3.5-2.4.4_sm_103_fake"
    assert cache[key]["tiles"] == {"3": 8, "4": 2}
    # the FP32 V-cycle's kernels are tuned apart from the FP64 ones
    mixed = FakeBatch(best={3: 2, 4: 16}, limit={}, precision=2)
    assert autotune.tune_batch(mixed, problems) == {3: 2, 4: 16}
    assert "batch_p2_2.3.5-2.4.4_sm_103_fake" in json.load(open(tuner))
    # same problems in another order: no timing, cached tiles applied
    again = FakeBatch(best={3: 1, 4: 1}, limit={})
    assert autotune.tune_batch(again, list(reversed(problems))) == tiles
    assert again.timings == 0 and again.tiles == tiles
    # refresh re-tunes
    fresh = FakeBatch(best={3: 1, 4: 1}, limit={})
    assert autotune.tune_batch(fresh, problems, refresh=True) == {3: 1, 4: 1}


def test_unreadable_cache_is_treated_as_empty(tuner):
    tuner.write_text("{ not json")
    assert autotune.load_cache() == {}
    batch = FakeBatch(best={2: 3}, limit={})
    assert autotune.tune_batch(batch, [(2, 2, 4)]) == {2: 3}
    assert json.load(open(tuner))  # rewritten as valid JSON
