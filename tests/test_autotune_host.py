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


class FakeShapedPlan:
    made = []

    def __init__(self, spec, widths, precision, tile=None, ctas=0, store=False, **kw):
        if ctas == 2 and tile > 16:
            raise jet.JetError(3, "two CTAs do not fit")
        self.key = (tile, ctas, store)
        FakeShapedPlan.made.append(self.key)

    def close(self):
        pass


def test_tune_picks_cta_shape_and_schedule(tmp_path, monkeypatch):
    monkeypatch.setattr(jet, "Plan", FakeShapedPlan)
    path = str(tmp_path / "cache.json")
    sp = specs.ks()
    # (tile, ctas, store) -> ms; the two-CTA tile-16 store form is fastest
    times = {(8, 1, False): 5.0, (8, 1, True): 4.0, (8, 2, False): 3.0, (8, 2, True): 2.5,
             (16, 1, False): 2.2, (16, 1, True): 2.4, (16, 2, False): 2.0, (16, 2, True): 1.1,
             (24, 1, False): 1.5, (24, 1, True): 1.6}
    best, res = autotune.tune(sp, [2, 64, 64, 1], "bf16", None, None, path=path, candidates=(8, 16, 24),
                              timer=lambda plan, p, x, s, reps: times[plan.key])
    assert best == 16 and res == {8: 2.5, 16: 1.1, 24: 1.5}
    assert autotune.tuned(sp, [2, 64, 64, 1], "bf16", path) == (16, "store", 2)
    FakeShapedPlan.made.clear()
    autotune.plan(sp, [2, 64, 64, 1], "bf16", path=path)
    assert FakeShapedPlan.made == [(16, 2, True)]
    # the SIMT forms are timed with the plan's own shape only
    FakeShapedPlan.made.clear()
    autotune.tune(sp, [2, 64, 64, 1], "fp32", None, None, path=path, candidates=(8,),
                  timer=lambda plan, p, x, s, reps: 1.0)
    assert FakeShapedPlan.made == [(8, 0, False)]
