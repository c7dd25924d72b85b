"""Schedule and launch-shape autotuner for libppe plans.

ppe_set_tuning exposes two kinds of choices:
  * the spectral schedule of the solve (LEGACY three passes on the
    [kz][j][kx] spectrum, FUSED cluster pass per kx plane, PENCIL bulk-copy-
    staged passes on the [kx][kz][j] spectrum), which changes which kernels
    run, so it is scored by the whole projection's device time (the sum of the
    per-kernel CUDA-event times of ppe_profile);
  * tile sizes (lines per CTA of the right-hand-side kernel and of the x
    transforms, columns per CTA of the z and y passes, planes per marching
    chunk), which change no result bit and only the time of their own kernel,
    so each is scored by that kernel alone.
`autotune` searches them coordinate by coordinate on the caller's own fields
(the schedule first, since it decides which kernels the tile sizes drive),
applies the best and remembers it in a JSON cache keyed by grid, precision,
face rule and GPU name, so that later plans of the same size class start from
it (`apply_cached`).
"""
from __future__ import annotations

import json
import os
import threading

from . import ppe

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ppe_gb300", "tuning.json")

STEP = "step"  # score: the sum of all kernel times of the projection

# which kernel each field of ppe_tuning drives, and the values tried (in this
# order: the schedule decides which kernels the later fields drive)
SEARCH = {
    "spectral": (STEP, (0, 1, 2)),
    "y_solve": (STEP, (1, 0)),
    "rhs_lines": ("k_rhs_march", (1, 2, 4, 8)),
    "rhs_planes": ("k_rhs_march", (4, 8, 16, 32)),
    "x_lines": ("k_xinv", (4, 8, 16, 32, 64)),
    "z_cols": ("k_zfft_fwd", (2, 4, 8, 16)),
    "y_cols": ("k_ysolve", (2, 4, 8, 16, 32)),
}

_lock = threading.Lock()


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:  # pragma: no cover
        return "unknown"


def cache_key(plan: "ppe.Plan", gpu: str | None = None) -> str:
    return (f"{plan.nx}x{plan.ny}x{plan.nz}|prec{plan.precision}|face{plan.opts.face_rule}|"
            f"{gpu if gpu is not None else _gpu_name()}")


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    with _lock:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def apply_cached(plan: "ppe.Plan", path: str = DEFAULT_CACHE, gpu: str | None = None) -> bool:
    """Apply a cached tuning for this plan's size class; True if one was found."""
    entry = load_cache(path).get(cache_key(plan, gpu))
    if not entry:
        return False
    try:
        plan.set_tuning(**entry["tuning"])
    except ppe.PPEError:
        return False
    return True


def _kernel_us(plan, run, kernel: str, reps: int) -> float:
    plan.profile(True)
    plan.profile_read()
    run(reps)
    kt = plan.profile_read()
    plan.profile(False)
    if kernel == STEP:
        return 1e3 * sum(ms for _, ms in kt.values()) / reps if kt else float("inf")
    if kernel not in kt:
        return float("inf")
    launches, ms = kt[kernel]
    return 1e3 * ms / launches


def autotune(plan: "ppe.Plan", run, reps: int = 3, path: str | None = DEFAULT_CACHE,
             search: dict | None = None) -> dict:
    """Tune `plan` in place.  `run(k)` must perform k projections with this plan
    (the caller's fields, so that the timing is that of the real workload).
    Returns {"tuning": best shapes, "kernel_us": time of each tuned kernel}."""
    search = SEARCH if search is None else search
    run(1)  # warm-up and first-use costs
    best = plan.get_tuning()
    times = {}
    for field, (kernel, values) in search.items():
        scores = []
        for v in values:
            trial = dict(best)
            trial[field] = v
            try:
                plan.set_tuning(**trial)
            except ppe.PPEError:
                continue  # out of range, too much shared memory, or a schedule this plan lacks
            if kernel == STEP:
                run(1)  # first use of a schedule (graph rebuild, first launches)
            scores.append((_kernel_us(plan, run, kernel, reps), v))
        if scores:
            t, v = min(scores)
            best[field] = v
            times[field] = {"kernel": kernel, "us": t, "tried": {str(b): a for a, b in scores}}
        plan.set_tuning(**best)
    result = {"tuning": best, "kernel_us": times}
    if path:
        cache = load_cache(path)
        cache[cache_key(plan)] = result
        save_cache(cache, path)
    return result


# Queue of the persistent batched form (ppe_batch_options): elements per
# queue item (tile runs), grids per window of the stage-major order, stages
# between windows, resident CTAs per SM (0: as many as fit).
BATCH_SEARCH = {
    "grain": (65536, 16384, 262144, 1048576),
    "window": (0, 32, 16, 8),
    "stagger": (1, 2, 4, 8),
    "ctas_per_sm": (0, 2),
}


def tune_batch(measure, search=None, start=None):
    """Coordinate search over the persistent batch's options.  `measure(opts)`
    builds the batch with the option dict `opts` (keys of BATCH_SEARCH), times
    its launches and returns milliseconds per batch (or None if the options are
    refused).  Each field is tried in turn with the others held at the best so
    far.  Returns (best options, best ms, {option tuple: ms} of every trial)."""
    search = search or BATCH_SEARCH
    best = dict(start or {k: v[0] for k, v in search.items()})
    trials = {}

    def key(o):
        return tuple(o[k] for k in search)

    def score(o):
        k = key(o)
        if k not in trials:
            trials[k] = measure(dict(o))
        return trials[k]

    best_ms = score(best)
    for field, values in search.items():
        for v in values:
            cand = dict(best, **{field: v})
            ms = score(cand)
            if ms is not None and (best_ms is None or ms < best_ms):
                best, best_ms = cand, ms
    return best, best_ms, {",".join(f"{k}={v}" for k, v in zip(search, t)): ms for t, ms in trials.items()}
