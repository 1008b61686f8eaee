"""Tile autotuner for the fused jet kernels.

For a plan shape (residual spec, layer widths, precision) it builds plans with
each candidate tile size (points per tile, which fixes the MMA N extent of the
tensor-core kernel and the per-CTA chunking of the work list), weight-gradient
schedule and CTA shape (one CTA of 16 warps or two of 8 warps per SM), times
the parameter-gradient call with CUDA events on representative points, and
keeps the fastest.  Results are cached in a JSON file keyed by the shape, so that
later plans of the same shape reuse the choice without timing.

The cache path is ``$JET_TUNE_CACHE`` when set, else ``jet_tune_cache.json``
in the system temporary directory.
"""

import json
import os
import tempfile

from . import jet

DEFAULT_CANDIDATES = (8, 16, 24, 32, 40, 48, 56, 64, 80, 96, 112, 128, 160, 192, 256)


def cache_path():
    return os.environ.get("JET_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "jet_tune_cache.json"))


def shape_key(spec, widths, precision):
    chans = ",".join("".join(str(k) for k in a) for a in spec.closure())
    return "%s|d%d|o%d|%s|%s|%s" % (spec.name, spec.d_in, spec.n_out, "x".join(map(str, widths)), precision, chans)


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=None):
    path = path or cache_path()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_plan(plan, params, X, source, reps):
    import torch
    plan.backward(params, X, source)  # warm-up (also first-launch costs)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.backward(params, X, source)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


STORE_BUDGET = 96 << 30


def tune(spec, widths, precision, params, X, source=None, candidates=DEFAULT_CANDIDATES, reps=3, path=None,
         timer=None, schedules=None, ctas=None):
    """Time every (tile size, weight-gradient schedule, CTA shape) triple;
    cache and return (best_tile, {tile: ms}) -- the ms of each tile's fastest
    schedule and shape.

    Schedules of the tensor-core forms: "tile" (weight gradient flushed per
    tile, bounded memory) and "store" (layer inputs and adjoints in HBM, one
    weight-gradient GEMM per layer); CTA shapes 1 (16 warps) and 2 (two CTAs
    of 8 warps per SM).  The SIMT forms have one schedule and shape.
    """
    timer = timer or _time_plan
    tc = precision in ("bf16", "bf16x3", "tf32")
    if schedules is None:
        schedules = ("tile", "store") if tc else ("tile",)
    if ctas is None:
        ctas = (1, 2) if tc else (0,)
    results, choice = {}, {}
    for P in candidates:
        for sc in schedules:
            for nc in ctas:
                kw = dict(store=True, mem_budget=STORE_BUDGET) if sc == "store" else {}
                try:
                    plan = jet.Plan(spec, widths, precision, tile=P, ctas=nc, **kw)
                except jet.JetError:
                    continue  # does not fit shared memory / TMEM for this shape
                try:
                    ms = float(timer(plan, params, X, source, reps))
                finally:
                    plan.close()
                if P not in results or ms < results[P]:
                    results[P], choice[P] = ms, (sc, nc)
    if not results:
        raise RuntimeError("no candidate tile size fits this shape")
    best = min(results, key=lambda k: (results[k], k))
    cache = load_cache(path)
    cache[shape_key(spec, widths, precision)] = {"tile": int(best), "schedule": choice[best][0],
                                                 "ctas": int(choice[best][1]),
                                                 "ms": {str(k): v for k, v in results.items()}}
    save_cache(cache, path)
    return best, results


def tuned(spec, widths, precision, path=None):
    """Cached (tile, schedule, ctas) for the shape, or None."""
    e = load_cache(path).get(shape_key(spec, widths, precision))
    return None if e is None else (int(e["tile"]), e.get("schedule", "tile"), int(e.get("ctas", 0)))


def tuned_tile(spec, widths, precision, path=None):
    """Cached tile size for the shape, or None."""
    t = tuned(spec, widths, precision, path)
    return None if t is None else t[0]


def plan(spec, widths, precision, path=None, **kw):
    """A plan that uses the cached tile size and schedule of its shape when there is one."""
    t = tuned(spec, widths, precision, path)
    if t is None:
        return jet.Plan(spec, widths, precision, **kw)
    if t[1] == "store":
        kw.setdefault("store", True)
        kw.setdefault("mem_budget", STORE_BUDGET)
    kw.setdefault("ctas", t[2])
    return jet.Plan(spec, widths, precision, tile=t[0], **kw)


BATCH_PREFIX = "batch|"
# options of a batched ensemble: (CTA shape, fraction of each member's default
# tile).  A batch runs one CTA shape and the per-tile weight-gradient schedule.
BATCH_OPTIONS = ((1, 1.0), (1, 0.5), (2, 1.0), (2, 0.5))


def batch_key(members, precision):
    """Cache key of a batch: its member shapes (in order) and precision."""
    import hashlib
    sig = "\n".join(shape_key(spec, widths, precision) for spec, widths, _ in members)
    return BATCH_PREFIX + hashlib.sha1(sig.encode()).hexdigest()[:20]


def _member_plans(members, precision, ctas, scale):
    """One plan per member: CTA shape `ctas`, tile = `scale` x the shape's
    default tile (rounded down to a size the plan accepts, else the default)."""
    plans = []
    try:
        for spec, widths, _ in members:
            base = jet.Plan(spec, widths, precision, ctas=ctas)  # raises if the shape does not fit
            P = base.info()["tile_points"]
            if scale >= 1.0:
                plans.append(base)
                continue
            base.close()
            plan = None
            t = int(P * scale) // 8 * 8
            while plan is None and t >= 8:
                try:
                    plan = jet.Plan(spec, widths, precision, tile=t, ctas=ctas)
                except jet.JetError:
                    t -= 8
            plans.append(plan or jet.Plan(spec, widths, precision, ctas=ctas))
    except jet.JetError:
        for p in plans:
            p.close()
        raise
    return plans


def _time_batch(plans, params, X, reps):
    import torch
    b = jet.Batch(plans)
    try:
        b.backward(params, X)  # warm-up (also first-launch costs)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            b.backward(params, X)
        e.record()
        torch.cuda.synchronize()
        return a.elapsed_time(e) / reps
    finally:
        b.close()


def tune_batch(members, precision, X, reps=3, path=None, timer=None, options=BATCH_OPTIONS):
    """Time the batched backward of all members (one persistent launch) under
    every option, cache the fastest under the batch key and return
    (best option, {option: ms}).  members: list of (spec, widths, params);
    X: each member's points."""
    timer = timer or _time_batch
    params = [p for _, _, p in members]
    results = {}
    for ctas, scale in options:
        try:
            plans = _member_plans(members, precision, ctas, scale)
        except jet.JetError:
            continue  # some member does not fit this CTA shape
        try:
            results[(ctas, scale)] = float(timer(plans, params, X, reps))
        finally:
            for p in plans:
                p.close()
    if not results:
        raise RuntimeError("no batch option fits every member")
    best = min(results, key=lambda k: (results[k], -k[1], k[0]))
    cache = load_cache(path)
    cache[batch_key(members, precision)] = {"ctas": best[0], "scale": best[1],
                                            "ms": {"%d,%g" % k: v for k, v in results.items()}}
    save_cache(cache, path)
    return best, results


def batch_plans(members, precision, X, reps=3, path=None, timer=None):
    """Plans for a batched ensemble (jet.Batch) with tuned tiles: the batch's
    cached option, or tune_batch on the members' own points first."""
    e = load_cache(path).get(batch_key(members, precision))
    if e is None:
        (ctas, scale), _ = tune_batch(members, precision, X, reps=reps, path=path, timer=timer)
    else:
        ctas, scale = int(e["ctas"]), float(e["scale"])
    return _member_plans(members, precision, ctas, scale)
