"""Autotuner of the diameter kernels' tile and block shapes.

The FP32 pair kernel's tile size (vertices per tile), threads per CTA and
persistent CTAs per SM, and the spatial cell size that orders vertices into
tiles, trade culling granularity against per-item overhead differently for a
single large mask and for a batch of small crops.  tune() measures a staged
search on the caller's own workload (CUDA events around whole passes), picks
the fastest configuration and remembers it per size bucket; apply() restores
it.  The library's own defaults are used when nothing is cached.
"""
import json
import math
import os
import statistics

from . import rad

# (tile, threads) pairs the library instantiates
SHAPES = ((64, 64), (64, 128), (128, 64), (128, 128), (128, 256), (256, 64), (256, 128))
CELL_SHIFTS = (3, 4, 5)
CTAS_PER_SM = (2, 4, 8, 16)

DEFAULT_CACHE = os.environ.get("RAD_TUNING_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "rad_gb300", "tuning.json"))


def bucket(n_rois, total_vertices):
    """Size bucket of a workload: ROI count and vertex count, both by powers of two."""
    r = max(0, math.ceil(math.log2(max(1, n_rois))))
    v = max(0, math.ceil(math.log2(max(2, total_vertices))))
    return f"rois2^{r}_verts2^{v}"


def _timer_cuda():
    import torch

    def time_ms(run, reps):
        run()  # re-capture after a tuning change
        run()
        stream = torch.cuda.current_stream()
        out = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    return time_ms


def tune(run, label, reps=5, cache_path=DEFAULT_CACHE, time_ms=None, set_tuning=None, get_tuning=None,
         margin=0.01):
    """Staged search; returns (best config dict, list of (config, ms)).

    run: callable doing one whole pass of the workload (e.g. a rad_extract or
    rad_batch_run).  time_ms / set_tuning / get_tuning default to CUDA events
    and the library; tests substitute fakes.  A candidate replaces the best
    only when it is faster by `margin` (relative), and the winner is timed
    again against the starting configuration with twice the repetitions, so
    timing noise does not move the configuration."""
    time_ms = time_ms or _timer_cuda()
    set_tuning = set_tuning or rad.set_tuning
    get_tuning = get_tuning or rad.get_tuning
    start = dict(get_tuning())
    table = []
    seen = {}

    def trial(cfg):
        key = tuple(sorted(cfg.items()))
        if key in seen:  # every configuration is measured once
            return seen[key]
        set_tuning(**cfg)
        ms = time_ms(run, reps)
        table.append((dict(cfg), ms))
        seen[key] = ms
        return ms

    def better(ms, ref):
        return ms < ref * (1.0 - margin)

    best = dict(start)
    best_ms = trial(best)
    for cs in CELL_SHIFTS:
        if cs == best["cell_shift"]:
            continue
        cfg = dict(best, cell_shift=cs)
        ms = trial(cfg)
        if better(ms, best_ms):
            best, best_ms = cfg, ms
    for tile, threads in SHAPES:
        if (tile, threads) == (best["tile"], best["threads"]):
            continue
        cfg = dict(best, tile=tile, threads=threads)
        ms = trial(cfg)
        if better(ms, best_ms):
            best, best_ms = cfg, ms
    for c in CTAS_PER_SM:
        if c == best["ctas_per_sm"]:
            continue
        cfg = dict(best, ctas_per_sm=c)
        ms = trial(cfg)
        if better(ms, best_ms):
            best, best_ms = cfg, ms
    if best != start:  # confirm against the start with more repetitions
        set_tuning(**start)
        ms_start = time_ms(run, 2 * reps)
        set_tuning(**best)
        ms_best = time_ms(run, 2 * reps)
        if not better(ms_best, ms_start):
            best, best_ms = dict(start), ms_start
        else:
            best_ms = ms_best
    set_tuning(**best)
    if cache_path:
        store(label, best, best_ms, cache_path)
    return best, table


def load(cache_path=DEFAULT_CACHE):
    try:
        with open(cache_path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(label, cfg, ms, cache_path=DEFAULT_CACHE):
    data = load(cache_path)
    data[label] = {"config": cfg, "ms": ms}
    os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)


def apply(label, cache_path=DEFAULT_CACHE, set_tuning=None):
    """Set the cached configuration of `label`; returns it (or None)."""
    entry = load(cache_path).get(label)
    if not entry:
        return None
    (set_tuning or rad.set_tuning)(**entry["config"])
    return entry["config"]
