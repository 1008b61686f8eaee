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


class FakeBatchPlan:
    """Default tile 64 (one CTA) or 32 (two CTAs); width 256 does not fit two."""
    made = []

    def __init__(self, spec, widths, precision, tile=None, ctas=0, **kw):
        if ctas == 2 and widths[1] == 256:
            raise jet.JetError(3, "two CTAs do not fit")
        if tile is not None and tile % 16:
            raise jet.JetError(3, "not a whole number of sub-tiles")
        self.key = (tile or (32 if ctas == 2 else 64), ctas)
        FakeBatchPlan.made.append(self.key)

    def info(self):
        return {"tile_points": self.key[0]}

    def close(self):
        pass


def test_batch_tuning_times_whole_batches(tmp_path, monkeypatch):
    """tune_batch times the whole batch under every option that fits all
    members (one CTA shape for all, tiles scaled from each default and rounded
    down to a tile the plan accepts), caches the fastest under the batch's key,
    and batch_plans reuses it without timing."""
    monkeypatch.setattr(jet, "Plan", FakeBatchPlan)
    path = str(tmp_path / "cache.json")
    b, a = specs.burgers(0.01), specs.allen_cahn()
    members = [(b, [2, 32, 32, 1], None), (a, [2, 64, 1], None)]
    timed = []

    def timer(plans, params, X, reps):
        keys = tuple(p.key for p in plans)
        timed.append(keys)
        return {64: 2.0, 32: 1.0, 16: 3.0}[keys[0][0]] + (0.5 if keys[0][1] == 2 else 0.0)

    best, res = autotune.tune_batch(members, "bf16", None, path=path, timer=timer)
    # (1, 0.5) -> 32-point tiles, the fastest; (2, 0.5) rounds 16 to a size the plan takes
    assert best == (1, 0.5) and set(res) == set(autotune.BATCH_OPTIONS)
    assert ((32, 1), (32, 1)) in timed and ((16, 2), (16, 2)) in timed
    timed.clear()
    plans = autotune.batch_plans(members, "bf16", None, path=path, timer=timer)
    assert timed == [] and [p.key for p in plans] == [(32, 1), (32, 1)]
    # a member too wide for two CTAs removes those options
    wide = members + [(b, [2, 256, 256, 1], None)]
    best, res = autotune.tune_batch(wide, "bf16", None, path=path, timer=timer)
    assert set(res) == {(1, 1.0), (1, 0.5)} and best == (1, 0.5)
    assert autotune.batch_key(wide, "bf16") != autotune.batch_key(members, "bf16")
