"""Autotuner for the engine's launch choices: cell size, pair loop and block size.

For a set of cases it times a few Symplectic steps of each candidate
configuration on the device (CUDA events inside libsph) and keeps the fastest.
The search has two stages: the cell size (cells of 2h, h or 2h/3, i.e. the
cells a target's support spans per axis) crossed with the interaction
variant, then, for the winner if it walks a neighbour list, the thread-block
size of that walk.  Results are cached in a JSON file keyed by (GPU name,
case count bucket, particle count bucket) so that later runs on the same kind
of GPU and workload skip the search.
"""
import json
import math
import os

# (cell_mode, pi_variant)
CANDIDATES = [(1, 4), (1, 5), (2, 4), (2, 5), (0, 4), (1, 3), (1, 0), (2, 0), (1, 1), (0, 0)]
# threads per block of the list walk (pi_variant 3-5)
BLOCKS = (128, 256, 512)


def cache_path() -> str:
    base = os.environ.get("SPH_AUTOTUNE_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache")),
        "sph_gb300_autotune.json")
    return base


def bucket_key(gpu_name: str, cases, pair_once=0) -> str:
    n = sum(c.n for c in cases)
    return "%s|cases~2^%d|particles~2^%d%s" % (gpu_name, int(math.log2(max(1, len(cases)))),
                                              int(math.log2(max(1, n))),
                                              "|pair_once" if pair_once else "")


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


def _time(cases, make_engine, cm, var, block, steps, warmup, pair_once=0):
    """ms per step of one configuration; inf if it cannot run (for instance a
    neighbour list that overflows at this cell size: the library reports it)."""
    for c in cases:
        c.params["cell_mode"] = cm
    try:
        e = make_engine(cases)
    except RuntimeError:
        return float("inf")
    try:
        e.set_options(pi_variant=var, pi_block=block, pair_once=pair_once)
        e.step(warmup)
        e.set_options(pi_variant=var, pi_block=block, timing=1, pair_once=pair_once)
        e.timing(reset=True)
        e.step(steps)
        t = e.timing(reset=True)
    except RuntimeError:
        return float("inf")
    finally:
        e.destroy()
    return t["step_ms"] / steps


def tune(cases, make_engine, gpu_name: str, steps=3, warmup=2, candidates=CANDIDATES,
         blocks=BLOCKS, use_cache=True, pair_once=0):
    """Return ((cell_mode, pi_variant, pi_block), {config: ms_per_step}).

    make_engine(cases) must build an engine from the cases (whose params carry
    cell_mode); the engine's timing option gives the device time per step.
    pair_once: the candidates are timed with each pair evaluated once (where a
    list walk applies).  The cases' cell_mode is restored afterwards."""
    key = bucket_key(gpu_name, cases, pair_once)
    cache = _load() if use_cache else {}
    if key in cache and len(cache[key].get("best", ())) == 3:
        return tuple(cache[key]["best"]), cache[key].get("times", {})
    times = {}
    saved = [c.params.get("cell_mode", 0) for c in cases]
    try:
        for cm, var in candidates:
            times["%d,%d,128" % (cm, var)] = _time(cases, make_engine, cm, var, 0, steps, warmup,
                                                   pair_once)
        best_s = min(times, key=times.get)
        cm, var, _ = (int(x) for x in best_s.split(","))
        if var in (3, 4, 5):
            for b in blocks:
                k = "%d,%d,%d" % (cm, var, b)
                if k not in times:
                    times[k] = _time(cases, make_engine, cm, var, b, steps, warmup, pair_once)
    finally:
        for c, cm0 in zip(cases, saved):
            c.params["cell_mode"] = cm0
    best_s = min(times, key=times.get)
    best = tuple(int(x) for x in best_s.split(","))
    if use_cache:
        cache[key] = {"best": list(best), "times": times}
        _store(cache)
    return best, times
