"""Autotuner of the kernel shapes (written for this library).

The library exposes seven shape knobs (`ladder_set_tuning`): the full
search's band height (candidate rows per lane task), its warp tiles per CTA
and whether its last CTA per CTU also takes the CTU's decisions,
the dependent search's band height, the piece size large dependent CUs are
split into, the dependent search's grid size and whether it stages its
windows in shared memory.  None of them changes a result; they trade
load balance (how many tiles a launch has, how long the longest one is)
against per-candidate overhead, and the best setting depends on the
workload: one 1080p ladder frame has too few CTUs to fill the GPU with long
tiles, a batch of 32 frames has plenty.

`tune()` times a caller-supplied step (one batch of the real workload) for
each candidate setting by coordinate descent: knobs are tried one at a time,
each against the best values found so far, and a knob keeps its new value
only if the step gets faster by more than the noise margin.  The dependent
search's piece size, band height and form (staged in shared memory or read
through L1) are tried jointly (every combination): the best band depends on
the piece size through the shared memory a tile needs, and the best form
on both, so one knob at a time can stop at a setting that is worse than
one it never tried.  Each timing is
the median of `reps` runs bracketed by CUDA events on the step's stream.
Results are cached in a JSON file keyed by the device name and a
caller-chosen workload key, so a later run with the same shape only applies
the stored setting.
"""
from __future__ import annotations

import json
import os
import statistics
import time

SPACE = {
    "fs_band": (13, 9),
    "fs_group": (0, 1, 2, 3),
    "fs_fuse": (1, 0),
    ("dep_range", "dep_band", "dep_staged"): tuple((rg, bd, st) for st in (1, 0, 2) for rg in (16, 32)
                                                   for bd in (0, 17, 9)),
    "dep_ctas_per_sm": (0, 1, 2),
}
DEFAULTS = {"fs_band": 13, "fs_group": 0, "fs_fuse": 1, "dep_range": 16, "dep_band": 0, "dep_ctas_per_sm": 0,
            "dep_staged": 1, "dep_inherit": 1}


def knob_values(name: str) -> tuple:
    """Every value the search may give knob `name` (alone or in a joint
    pair); a knob outside the search keeps its default (dep_inherit: summing
    a CU's SADs from its sub-CUs' only removes work, so it stays on)."""
    for key, values in SPACE.items():
        if key == name:
            return tuple(values)
        if isinstance(key, tuple) and name in key:
            i = key.index(name)
            return tuple(sorted({v[i] for v in values}))
    if name in DEFAULTS:
        return (DEFAULTS[name],)
    raise KeyError(name)


def default_cache_path() -> str:
    return os.environ.get("LADDER_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ladder_tuning.json"))


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def workload_key(ladder, tag: str) -> str:
    """Key of a workload: geometry of the ladder plus a caller tag (e.g. the
    number of frames per batch)."""
    g = ladder.geometry
    rungs = "_".join(f"{w}x{h}" for (w, h) in ladder.rungs)
    return (f"bd{g.bit_depth}-ctu{g.ctu_size}-R{g.ref_search_range}-r{g.dep_refine_range}-ref{g.ref_rung}-"
            f"{rungs}-{tag}")


def time_step(run_step, stream, reps=5, warmup=2) -> float:
    """Median device time (ms) of run_step() on `stream`."""
    import torch
    for _ in range(warmup):
        run_step()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_step()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def tune(ladder, run_step, *, tag: str, stream=None, space=None, reps=5, warmup=2, margin=0.02,
         cache_path=None, use_cache=True, log=None, timer=None, device=None) -> dict:
    """Chooses the knob values for `ladder` on the workload `run_step`.

    Returns {"knobs": {...}, "ms": best step time, "trials": [...],
    "cached": bool, "seconds": tuning time}; the ladder is left set to the
    chosen values.  `timer(run_step)` (default: CUDA events on `stream`,
    median of `reps`) and `device` (default: the current CUDA device's name)
    can be replaced, e.g. to test the search on the host."""
    from .ladder import LadderError

    if timer is None or device is None:
        import torch
        stream = stream or torch.cuda.current_stream()
        device = device or torch.cuda.get_device_name()
        timer = timer or (lambda fn: time_step(fn, stream, reps, warmup))
    path = cache_path or default_cache_path()
    key = f"{device}|{workload_key(ladder, tag)}"
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            ladder.set_tuning(**hit["knobs"])
            return {"knobs": dict(hit["knobs"]), "ms": hit["ms"], "trials": [], "cached": True, "seconds": 0.0}

    t0 = time.perf_counter()
    space = space or SPACE
    best = dict(DEFAULTS)
    ladder.set_tuning(**best)
    best_ms = timer(run_step)
    trials = [(dict(best), best_ms)]
    for name, values in space.items():
        names = name if isinstance(name, tuple) else (name,)
        for v in values:
            v = v if isinstance(name, tuple) else (v,)
            if all(best[n] == x for n, x in zip(names, v)):
                continue
            cand = dict(best, **dict(zip(names, v)))
            try:
                ladder.set_tuning(**cand)
            except LadderError:
                continue  # a shape this geometry does not have
            ms = timer(run_step)
            trials.append((dict(cand), ms))
            if log:
                log(f"tune {cand} {ms:.4f} ms")
            if ms < best_ms * (1.0 - margin):
                best, best_ms = cand, ms
        ladder.set_tuning(**best)
    seconds = time.perf_counter() - t0
    if use_cache:
        data = _load(path)
        data[key] = {"knobs": best, "ms": best_ms, "when": time.strftime("%Y-%m-%d %H:%M:%S")}
        _save(path, data)
    return {"knobs": best, "ms": best_ms, "trials": trials, "cached": False, "seconds": seconds}
