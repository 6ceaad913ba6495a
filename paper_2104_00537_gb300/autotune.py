"""Autotuner for the engine's launch choices (cell size and interaction variant).

For a set of cases it times a few Symplectic steps of each candidate
configuration on the device (CUDA events inside libsph) and keeps the fastest.
Results are cached in a JSON file keyed by (GPU name, case count bucket,
particle count bucket) so that later runs on the same kind of GPU and workload
skip the search.
"""
import json
import math
import os

CANDIDATES = [(1, 4), (1, 5), (2, 4), (0, 4), (1, 3), (1, 0), (2, 0), (1, 1), (0, 0)]  # (cell_mode, pi_variant)


def cache_path() -> str:
    base = os.environ.get("SPH_AUTOTUNE_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache")),
        "sph_gb300_autotune.json")
    return base


def bucket_key(gpu_name: str, cases) -> str:
    n = sum(c.n for c in cases)
    return "%s|cases~2^%d|particles~2^%d" % (gpu_name, int(math.log2(max(1, len(cases)))),
                                            int(math.log2(max(1, n))))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def tune(cases, make_engine, gpu_name: str, steps=3, warmup=2, candidates=CANDIDATES,
         use_cache=True):
    """Return ((cell_mode, pi_variant), {config: ms_per_step}) for these cases.

    make_engine(cases) must build an engine from the cases (whose params carry
    cell_mode); the engine's timing option gives the device time per step."""
    key = bucket_key(gpu_name, cases)
    cache = _load() if use_cache else {}
    if key in cache:
        best = tuple(cache[key]["best"])
        return best, cache[key].get("times", {})
    times = {}
    saved = [c.params.get("cell_mode", 0) for c in cases]
    for cm, var in candidates:
        for c in cases:
            c.params["cell_mode"] = cm
        e = make_engine(cases)
        e.set_options(pi_variant=var)
        e.step(warmup)
        e.set_options(pi_variant=var, timing=1)
        e.timing(reset=True)
        e.step(steps)
        t = e.timing(reset=True)
        e.destroy()
        times["%d,%d" % (cm, var)] = t["step_ms"] / steps
    for c, cm in zip(cases, saved):
        c.params["cell_mode"] = cm
    best_s = min(times, key=times.get)
    best = tuple(int(x) for x in best_s.split(","))
    if use_cache:
        cache[key] = {"best": list(best), "times": times}
        _store(cache)
    return best, times
