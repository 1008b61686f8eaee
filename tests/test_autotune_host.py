"""Host logic of the tile autotuner (no GPU): candidate filtering, choice of the
fastest tile, cache round trip and reuse by ``autotune.plan``."""
import json

from paper_2606_29702_gb300 import autotune, jet, specs


class FakePlan:
    made = []

    def __init__(self, spec, widths, precision, tile=None, **kw):
        if tile is not None and tile > 40:
            raise jet.JetError(3, "does not fit")
        self.tile = tile
        FakePlan.made.append(tile)

    def close(self):
        pass


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setattr(jet, "Plan", FakePlan)
    path = str(tmp_path / "cache.json")
    sp = specs.burgers(0.01)
    times = {8: 3.0, 16: 1.5, 24: 1.2, 32: 1.25, 40: 2.0}
    best, res = autotune.tune(sp, [2, 32, 32, 1], "bf16", None, None, path=path,
                              timer=lambda plan, p, x, s, reps: times[plan.tile])
    assert best == 24
    assert set(res) == set(times)  # 48..64 rejected by the plan
    with open(path) as f:
        cache = json.load(f)
    key = autotune.shape_key(sp, [2, 32, 32, 1], "bf16")
    assert cache[key]["tile"] == 24
    assert autotune.tuned_tile(sp, [2, 32, 32, 1], "bf16", path) == 24
    assert autotune.tuned_tile(sp, [2, 64, 1], "bf16", path) is None
    FakePlan.made.clear()
    autotune.plan(sp, [2, 32, 32, 1], "bf16", path=path)
    assert FakePlan.made == [24]


def test_shape_key_distinguishes_shapes():
    a = autotune.shape_key(specs.burgers(0.01), [2, 32, 1], "bf16")
    b = autotune.shape_key(specs.allen_cahn(), [2, 32, 1], "bf16")
    c = autotune.shape_key(specs.burgers(0.01), [2, 32, 1], "bf16x3")
    assert len({a, b, c}) == 3
