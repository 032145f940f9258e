"""Autotuner of the library's launch choices for one workload.

The library exposes two choices per context that change only how the work is
laid out on the GPU, never the results:

* the kernels of the sequential-order passes (``wavefront``: one
  interpolation and one gather kernel per wavefront and pass; ``groups``: a
  persistent launch with a CTA group per particle) -- bitwise the same;
* the CTAs per particle of the volume integrals (slabs of cell planes; 0:
  one resident wave) -- the same sums, grouped differently.

:func:`tune` times a caller-supplied step (the call sequence of the
workload) for every combination on the device -- CUDA events on the current
stream, warm-up steps first, the median of several repeats -- and leaves the
fastest combination set on the context(s).  The step is run for real, so the
tuning steps advance the workload's state like any other step.
"""
from __future__ import annotations

import itertools
import statistics

import torch

SPACE = {"pass_kernels": ("wavefront", "groups"), "volume_split": (0, 4, 8, 16)}


def apply(ctxs, choice: dict):
    for c in ctxs:
        if "pass_kernels" in choice:
            c.set_pass_kernels(choice["pass_kernels"])
        if "volume_split" in choice:
            c.set_volume_split(choice["volume_split"])


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


def tune(ctxs, step, space: dict | None = None, **timing) -> dict:
    """Try every combination of `space` (default :data:`SPACE`) on the
    contexts `ctxs` with `step`; set and return the fastest.

    Returns {"choice": {...}, "ms": best, "table": [(choice, ms), ...]}.
    """
    space = SPACE if space is None else space
    keys = list(space)
    table = []
    for values in itertools.product(*(space[k] for k in keys)):
        choice = dict(zip(keys, values))
        apply(ctxs, choice)
        table.append((choice, time_step(step, **timing)))
    best, ms = min(table, key=lambda t: t[1])
    apply(ctxs, best)
    return {"choice": best, "ms": ms, "table": table}
