"""Tile autotuner for the fused jet kernels.

For a plan shape (residual spec, layer widths, precision) it builds plans with
each candidate tile size (points per tile, which fixes the MMA N extent of the
tensor-core kernel and the per-CTA chunking of the work list), times the
parameter-gradient call with CUDA events on representative points, and keeps
the fastest.  Results are cached in a JSON file keyed by the shape, so that
later plans of the same shape reuse the choice without timing.

The cache path is ``$JET_TUNE_CACHE`` when set, else ``jet_tune_cache.json``
in the system temporary directory.
"""

import json
import os
import tempfile

from . import jet

DEFAULT_CANDIDATES = (8, 16, 24, 32, 40, 48, 56, 64)


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


def tune(spec, widths, precision, params, X, source=None, candidates=DEFAULT_CANDIDATES, reps=3, path=None,
         timer=None):
    """Time every candidate tile size; cache and return (best_tile, {tile: ms})."""
    timer = timer or _time_plan
    results = {}
    for P in candidates:
        try:
            plan = jet.Plan(spec, widths, precision, tile=P)
        except jet.JetError:
            continue  # does not fit shared memory / TMEM for this shape
        try:
            results[P] = float(timer(plan, params, X, source, reps))
        finally:
            plan.close()
    if not results:
        raise RuntimeError("no candidate tile size fits this shape")
    best = min(results, key=lambda k: (results[k], k))
    cache = load_cache(path)
    cache[shape_key(spec, widths, precision)] = {"tile": int(best), "ms": {str(k): v for k, v in results.items()}}
    save_cache(cache, path)
    return best, results


def tuned_tile(spec, widths, precision, path=None):
    """Cached tile size for the shape, or None."""
    e = load_cache(path).get(shape_key(spec, widths, precision))
    return None if e is None else int(e["tile"])


def plan(spec, widths, precision, path=None, **kw):
    """A plan that uses the cached tile size of its shape when there is one."""
    return jet.Plan(spec, widths, precision, tile=tuned_tile(spec, widths, precision, path), **kw)
