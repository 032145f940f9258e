"""Autotuner of the library's launch choices for one workload.

The library exposes per-context choices that change only how the work is
laid out on the GPU, never the results:

* ``pass_kernels``: the kernels of the sequential-order passes
  (``wavefront``: one interpolation and one gather kernel per wavefront and
  pass; ``groups``: a persistent launch with a CTA group per particle; FP32
  fields) -- bitwise the same;
* ``volume_split``: the CTAs per particle of the volume integrals (slabs of
  cell planes; 0: one resident wave) -- the same sums, grouped differently;
* ``gather_ctas``: resident wavefront-gather CTAs per SM (0: as many as fit);
* ``gather_stage``: the candidates of a spreading tile that a gather CTA
  stages in shared memory -- the tile's bin capacity on chip; larger tiles
  read their candidates from memory, a smaller capacity lets more CTAs share
  an SM (0: the largest).  Both gather choices leave every sum unchanged.

:func:`tune` times a caller-supplied step (the call sequence of the
workload) on the device -- CUDA events on the current stream, warm-up steps
first, the median of several repeats -- by coordinate descent over the space
(each choice in turn, the others held at their best so far; two sweeps), and
leaves the fastest combination set on the context(s).  The step is run for
real, so the tuning steps advance the workload's state like any other step.

:func:`tune_cached` keeps the choices in a JSON file keyed by the device, the
field precision, the particles' diameter range and the grid size, so a
workload of the same kind reuses them without timing.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

SPACE = {"pass_kernels": ("wavefront", "groups"), "volume_split": (0, 4, 8, 16),
         "gather_ctas": (0, 2, 3, 4), "gather_stage": (0, 128, 192)}

DEFAULT = {"pass_kernels": "wavefront", "volume_split": 0, "gather_ctas": 0, "gather_stage": 0}


def apply(ctxs, choice: dict):
    for c in ctxs:
        if "pass_kernels" in choice:
            c.set_pass_kernels(choice["pass_kernels"])
        if "volume_split" in choice:
            c.set_volume_split(choice["volume_split"])
        if "gather_ctas" in choice or "gather_stage" in choice:
            c.set_gather(choice.get("gather_ctas", 0), choice.get("gather_stage", 0))


def time_step(step, warmup: int = 2, reps: int = 5, steps_per_rep: int = 2) -> float:
    """Median device time (ms) of one step over `reps` repeats."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    out = []
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps_per_rep):
            step()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b) / steps_per_rep)
    return statistics.median(out)


def tune(ctxs, step, space: dict | None = None, sweeps: int = 2, **timing) -> dict:
    """Coordinate descent over `space` (default :data:`SPACE`) on the
    contexts `ctxs` with `step`; set and return the fastest choice.

    Returns {"choice": {...}, "ms": best, "table": [(choice, ms), ...]} with
    one table row per distinct combination timed.
    """
    space = SPACE if space is None else space
    best = {k: (DEFAULT[k] if DEFAULT.get(k) in v else v[0]) for k, v in space.items()}
    seen: dict[tuple, float] = {}

    def measure(choice):
        key = tuple(sorted(choice.items()))
        if key not in seen:
            apply(ctxs, choice)
            seen[key] = time_step(step, **timing)
        return seen[key]

    best_ms = measure(best)
    for _ in range(sweeps):
        changed = False
        for k, values in space.items():
            for v in values:
                cand = dict(best, **{k: v})
                ms = measure(cand)
                if ms < best_ms:
                    best, best_ms, changed = cand, ms, True
        if not changed:
            break
    apply(ctxs, best)
    table = [(dict(k), ms) for k, ms in seen.items()]
    return {"choice": best, "ms": best_ms, "table": table}


def cache_key(device, prec: int, d_cells, grid_n) -> str:
    """(device, precision, diameter range in cells, grid size) -> cache key.
    Diameters are bucketed to 4 cells and the grid to the next multiple of
    32 cells, so nearby workloads share an entry."""
    name = torch.cuda.get_device_name(device)
    cap = "%d.%d" % torch.cuda.get_device_capability(device)
    dlo, dhi = min(d_cells), max(d_cells)
    lo, hi = 4 * int(dlo // 4), 4 * int(-(-dhi // 4))
    n = 32 * int(-(-max(grid_n) // 32))
    return "%s|sm_%s|%s|D%d-%d|N%d" % (name, cap, "f64" if prec == 0 else "f32", lo, hi, n)


def default_cache_path() -> str:
    return os.environ.get("GBIB_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gbib", "autotune.json"))


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_cached(key: str, ctxs, step, path: str | None = None, space: dict | None = None, **timing) -> dict:
    """The choices cached under `key` (applied without timing), else
    :func:`tune`'s, stored under `key`.  Returns tune's result plus
    {"cached": bool, "key": key}."""
    path = default_cache_path() if path is None else path
    cache = load_cache(path)
    if key in cache:
        choice = cache[key]["choice"]
        apply(ctxs, choice)
        return {"choice": choice, "ms": cache[key].get("ms"), "table": [], "cached": True, "key": key}
    res = tune(ctxs, step, space=space, **timing)
    cache[key] = {"choice": res["choice"], "ms": res["ms"]}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return dict(res, cached=False, key=key)
